// Longitude transform of lambda-pencil rows: the FFT that follows the first
// transposition (Sec. II-A: the spectral transform is an FFT in longitude and a
// Legendre transform in latitude; Sec. II-B: the z -> lambda all-to-all makes
// every longitude row local).  For a row x_0 .. x_{N-1} it returns
//     F_m = (1/N) sum_j x_j exp(-2 pi i j m / N),  m = 0 .. K-1,
// as two float arrays (real and imaginary parts), the wavenumber fields the
// second transposition then moves.
//
// A real row of N = 2H values is read as H complex values z_k = x_2k + i x_2k+1
// (the row itself, reinterpreted), transformed by an H-point complex FFT, and
// split into the even- and odd-index transforms to give X_m for m = 0 .. H.
// The H-point FFT is a self-sorting (Stockham) FFT in shared memory: after
// the stages of radices p_1 .. p_t (product L so far, r = H / L) the buffer
// holds at k + r f the L-point DFT, at frequency f, of the samples
// z_k, z_{k+r}, z_{k+2r}, ...; one stage of radix p maps (k + r' q, f) for
// q < p, r' = r / p, through twiddles w_{pL}^{f q} and a p-point DFT onto
// (k, f + L s) for s < p.  Radices 16, 8, 4, 2, 3 and 5 (16 and 8 as two
// levels of 4 x 4 and 4 x 2 in registers); twiddles e^{-2 pi i t / N}
// from a table built on the host in double precision and rounded once.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <cuda_runtime.h>

#include "zfpx_internal.h"
#include "zfpx_fft.cuh"

namespace zfpx {
namespace {

using namespace fft;

constexpr int kMaxWarps = 8;                    // rows (one per warp) per CTA
constexpr int kRowBytesBudget = 40 * 1024;      // shared memory for the rows of one CTA (several CTAs per SM)

// One warp per row: the warp's two H-value buffers in shared memory, no
// barrier wider than the warp, so warps of a CTA never wait for each other.
// The bound keeps registers at 85 or fewer, so that shared memory, not
// registers, limits the warps per SM.
__global__ void __launch_bounds__(32 * kMaxWarps, 3) rfft_lon_kernel(const float *__restrict__ in, float *__restrict__ re,
                                                                float *__restrict__ im, const float2 *__restrict__ tw,
                                                                FftGeom g)
{
    extern __shared__ __align__(16) float2 fsm[];
    const int H = g.H, lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float2 *const buf = fsm + (size_t)wid * 2 * H;
    for (int64_t gr = (int64_t)blockIdx.x * nw + wid; gr < g.nrows; gr += (int64_t)gridDim.x * nw) {
        const int64_t y = gr % g.ny, z = gr / g.ny;
        // the row in, as H complex values (8-byte aligned pairs)
        const float2 *src = reinterpret_cast<const float2 *>(in + z * g.is2 + y * g.is1);
        load_row_async(buf, src, H, lane);
        wait_rows();
        __syncwarp();
        rfft_row(buf, buf + H, tw, g, lane, re + z * g.os2 + y * g.os1, im + z * g.os2 + y * g.os1);
    }
}

// e^{-2 pi i t / N}, t < N, per (device, N); built once, never freed.
std::mutex g_tw_mu;
std::map<std::pair<int, int>, float2 *> g_tw;

int twiddles_impl(int N, const float2 **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ZFPX_ECUDA;
    std::lock_guard<std::mutex> lk(g_tw_mu);
    auto key = std::make_pair(dev, N);
    auto it = g_tw.find(key);
    if (it != g_tw.end()) { *out = it->second; return ZFPX_OK; }
    std::vector<float2> h(N);
    const double two_pi = 6.283185307179586476925286766559;
    for (int t = 0; t < N; t++) {
        const double a = two_pi * (double)t / (double)N;
        h[t] = make_float2((float)std::cos(a), (float)-std::sin(a));
    }
    float2 *d = nullptr;
    if (cudaMalloc(&d, sizeof(float2) * N) != cudaSuccess) return ZFPX_ECUDA;
    if (cudaMemcpy(d, h.data(), sizeof(float2) * N, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return ZFPX_ECUDA;
    }
    g_tw[key] = d;
    *out = d;
    return ZFPX_OK;
}

// H = 16^a 8^b 4^c 2^d 3^e 5^f -> radices, largest first; false if another
// prime divides H
bool factor_half_impl(int H, FftGeom &g)
{
    g.nst = 0;
    int h = H;
    for (int p : {16, 8, 4, 2, 3, 5})
        while (h % p == 0) {
            if (g.nst == kMaxStages) return false;
            g.radix[g.nst++] = p;
            h /= p;
        }
    return h == 1;
}

}  // namespace

int fft_twiddles(int N, const float2 **out) { return twiddles_impl(N, out); }

bool fft_plan_half(int H, FftGeom &g)
{
    if (!factor_half_impl(H, g)) return false;
    for (int s = 0, r = H; s < g.nst; s++) {
        g.rp[s] = make_fastdiv((uint32_t)(r / g.radix[s]));
        r /= g.radix[s];
    }
    return true;
}
}  // namespace zfpx

using namespace zfpx;

extern "C" {

int zfpx_rfft_lon(const float *d_in, const int64_t n[3], const int64_t stride[3], int K, float *d_re, float *d_im,
                  const int64_t ostride[3], void *stream)
{
    if (!d_in || !d_re || !d_im || !n || !stride || !ostride) return ZFPX_EINVAL;
    const int64_t N = n[0];
    if (N < 2 || N % 2 || N > 2 * kMaxHalf || n[1] < 1 || n[2] < 1) return ZFPX_EINVAL;
    if (K < 1 || K > N / 2 + 1) return ZFPX_EINVAL;
    if (stride[0] != 1 || ostride[0] != 1 || stride[1] < 0 || stride[2] < 0 || ostride[1] < 0 || ostride[2] < 0)
        return ZFPX_EINVAL;
    if (((uintptr_t)d_in & 7u) || (stride[1] & 1) || (stride[2] & 1)) return ZFPX_EINVAL;
    if (((uintptr_t)d_re & 3u) || ((uintptr_t)d_im & 3u)) return ZFPX_EINVAL;
    FftGeom g{};
    g.N = (int)N; g.H = (int)(N / 2); g.K = K;
    if (!fft_plan_half(g.H, g)) return ZFPX_EINVAL;
    const int warps = std::max(1, std::min(kMaxWarps, kRowBytesBudget / (int)(2 * sizeof(float2) * g.H)));
    g.nrows = n[1] * n[2]; g.ny = n[1];
    g.is1 = stride[1]; g.is2 = stride[2]; g.os1 = ostride[1]; g.os2 = ostride[2];
    const float2 *tw = nullptr;
    int rc = fft_twiddles(g.N, &tw);
    if (rc) return rc;
    const size_t smem = 2 * sizeof(float2) * (size_t)warps * g.H;
    if (cudaFuncSetAttribute(rfft_lon_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return ZFPX_ECUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rfft_lon_kernel, 32 * warps, smem) != cudaSuccess)
        return ZFPX_ECUDA;
    const int64_t groups = (g.nrows + warps - 1) / warps;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(groups, (int64_t)num_sms() * std::max(1, per_sm)));
    rfft_lon_kernel<<<grid, 32 * warps, smem, (cudaStream_t)stream>>>(d_in, d_re, d_im, tw, g);
    count_launch();
    return check_launch();
}

}  // extern "C"
