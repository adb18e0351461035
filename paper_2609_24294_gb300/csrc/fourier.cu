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

namespace zfpx {
namespace {

constexpr int kMaxWarps = 8;                    // rows (one per warp) per CTA
constexpr int kMaxStages = 16;
constexpr int kMaxHalf = 4096;                  // N <= 8192
constexpr int kRowBytesBudget = 40 * 1024;      // shared memory for the rows of one CTA (several CTAs per SM)

// n / d for n d < 2^32 as one multiply-high by m = ceil(2^32 / d) (exact in
// that range: m d - 2^32 < d); d = 1 has m = 0 and returns n.
struct FastDiv {
    uint32_t d, m;
    __device__ __forceinline__ uint32_t div(uint32_t n) const { return m ? __umulhi(n, m) : n; }
};
inline FastDiv make_fastdiv(uint32_t d)
{
    return FastDiv{d, d == 1 ? 0u : (uint32_t)((((uint64_t)1 << 32) + d - 1) / d)};
}

struct FftGeom {
    int N, H, K, nst;
    int radix[kMaxStages];
    FastDiv rp[kMaxStages];   // r / p of each stage
    int64_t nrows, ny;
    int64_t is1, is2;         // input row strides (floats)
    int64_t os1, os2;         // output row strides (floats)
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// multiply by -i
__device__ __forceinline__ float2 cmul_mi(float2 a) { return make_float2(a.y, -a.x); }

__device__ __forceinline__ void dft4(float2 a0, float2 a1, float2 a2, float2 a3, float2 &v0, float2 &v1, float2 &v2,
                                     float2 &v3)
{
    // w_4 = -i: v_s = sum_q a_q (-i)^{s q}
    const float2 a = cadd(a0, a2), b = csub(a0, a2);
    const float2 c = cadd(a1, a3), d = cmul_mi(csub(a1, a3));
    v0 = cadd(a, c);
    v1 = cadd(b, d);
    v2 = csub(a, c);
    v3 = csub(b, d);
}

// v_s = sum_q u_q w_P^{s q}, with w[j] = w_P^j.  P = 8 and 16 as two levels:
// q = B a + b, s = c + 4 d (B = P / 4): a 4-point DFT over a for every b, the
// twiddle w_P^{b c}, then a B-point DFT over b for every c.
template <int P>
__device__ __forceinline__ void small_dft(const float2 (&u)[P], float2 (&v)[P], const float2 (&w)[P])
{
    if constexpr (P == 2) {
        v[0] = cadd(u[0], u[1]);
        v[1] = csub(u[0], u[1]);
    } else if constexpr (P == 4) {
        dft4(u[0], u[1], u[2], u[3], v[0], v[1], v[2], v[3]);
    } else if constexpr (P == 8 || P == 16) {
        constexpr int B = P / 4;
        float2 t[B][4];
#pragma unroll
        for (int b = 0; b < B; b++) {
            dft4(u[b], u[B + b], u[2 * B + b], u[3 * B + b], t[b][0], t[b][1], t[b][2], t[b][3]);
#pragma unroll
            for (int c = 1; c < 4; c++)
                if (b) t[b][c] = cmul(t[b][c], w[(b * c) % P]);
        }
#pragma unroll
        for (int c = 0; c < 4; c++) {
            if constexpr (B == 2) {
                v[c] = cadd(t[0][c], t[1][c]);
                v[c + 4] = csub(t[0][c], t[1][c]);
            } else {
                dft4(t[0][c], t[1][c], t[2][c], t[3][c], v[c], v[c + 4], v[c + 8], v[c + 12]);
            }
        }
    } else {
        // P = 3 or 5
#pragma unroll
        for (int s = 0; s < P; s++) {
            float2 acc = u[0];
#pragma unroll
            for (int q = 1; q < P; q++) acc = cadd(acc, cmul(u[q], w[(s * q) % P]));
            v[s] = acc;
        }
    }
}

// FIRST: the first stage (L = 1, so f = 0 and every twiddle is 1).
template <int P, bool FIRST>
__device__ __forceinline__ void fft_stage(const float2 *x, float2 *y, const float2 *__restrict__ tw, int N, int H,
                                          int L, int lane, FastDiv drp)
{
    const int Lp = L * P, r = H / L, rp = (int)drp.d, nb = H / P;
    float2 w[P];
#pragma unroll
    for (int j = 0; j < P; j++) w[j] = __ldg(tw + (int64_t)j * (N / P));
    const int tstep = N / Lp;                   // w_{pL}^{t} = e^{-2 pi i t / (pL)} = tw[t N / (pL)]
    for (int b = lane; b < nb; b += 32) {
        const int f = (int)drp.div(b), k = b - f * rp;
        float2 u[P], v[P];
#pragma unroll
        for (int q = 0; q < P; q++) {
            const float2 a = x[k + rp * q + r * f];
            u[q] = (FIRST || !q) ? a : cmul(a, __ldg(tw + f * q * tstep));
        }
        small_dft<P>(u, v, w);
#pragma unroll
        for (int s = 0; s < P; s++) y[k + rp * (f + L * s)] = v[s];
    }
}

// One warp per row: the warp's two H-value buffers in shared memory, no
// barrier wider than the warp, so warps of a CTA never wait for each other.
// The bound keeps registers at 85 or fewer, so that shared memory, not
// registers, limits the warps per SM.
__global__ void __launch_bounds__(32 * kMaxWarps, 3) rfft_lon_kernel(const float *__restrict__ in, float *__restrict__ re,
                                                                float *__restrict__ im, const float2 *__restrict__ tw,
                                                                FftGeom g)
{
    extern __shared__ float2 fsm[];
    const int H = g.H, lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const float scale = 1.0f / (float)g.N;
    float2 *const buf = fsm + (size_t)wid * 2 * H;
    for (int64_t gr = (int64_t)blockIdx.x * nw + wid; gr < g.nrows; gr += (int64_t)gridDim.x * nw) {
        const int64_t y = gr % g.ny, z = gr / g.ny;
        float2 *X = buf, *Y = buf + H;
        // the row in, as H complex values (8-byte aligned pairs)
        const float2 *src = reinterpret_cast<const float2 *>(in + z * g.is2 + y * g.is1);
#pragma unroll 4
        for (int k = lane; k < H; k += 32) X[k] = __ldg(src + k);
        __syncwarp();
        int L = 1;
        for (int s = 0; s < g.nst; s++) {
            const int p = g.radix[s];
            if (s == 0) {
                if (p == 16) fft_stage<16, true>(X, Y, tw, g.N, H, L, lane, g.rp[s]);
                else if (p == 8) fft_stage<8, true>(X, Y, tw, g.N, H, L, lane, g.rp[s]);
                else if (p == 4) fft_stage<4, true>(X, Y, tw, g.N, H, L, lane, g.rp[s]);
                else if (p == 2) fft_stage<2, true>(X, Y, tw, g.N, H, L, lane, g.rp[s]);
                else if (p == 3) fft_stage<3, true>(X, Y, tw, g.N, H, L, lane, g.rp[s]);
                else fft_stage<5, true>(X, Y, tw, g.N, H, L, lane, g.rp[s]);
            } else {
                if (p == 16) fft_stage<16, false>(X, Y, tw, g.N, H, L, lane, g.rp[s]);
                else if (p == 8) fft_stage<8, false>(X, Y, tw, g.N, H, L, lane, g.rp[s]);
                else if (p == 4) fft_stage<4, false>(X, Y, tw, g.N, H, L, lane, g.rp[s]);
                else if (p == 2) fft_stage<2, false>(X, Y, tw, g.N, H, L, lane, g.rp[s]);
                else if (p == 3) fft_stage<3, false>(X, Y, tw, g.N, H, L, lane, g.rp[s]);
                else fft_stage<5, false>(X, Y, tw, g.N, H, L, lane, g.rp[s]);
            }
            __syncwarp();
            float2 *t = X; X = Y; Y = t;
            L *= p;
        }
        // X now holds Z_f at f.  X_m = E_m + e^{-2 pi i m / N} O_m with
        // E_m = (Z_m + conj Z_{H-m}) / 2, O_m = (Z_m - conj Z_{H-m}) / (2i).
        float *ore = re + z * g.os2 + y * g.os1, *oim = im + z * g.os2 + y * g.os1;
#pragma unroll 2
        for (int m = lane; m < g.K; m += 32) {
            const float2 zm = X[m == H ? 0 : m];
            const float2 zc = X[m == 0 ? 0 : H - m];
            const float2 E = make_float2(0.5f * (zm.x + zc.x), 0.5f * (zm.y - zc.y));
            const float2 O = make_float2(0.5f * (zm.y + zc.y), -0.5f * (zm.x - zc.x));
            const float2 Xm = cadd(E, cmul(O, __ldg(tw + m)));
            ore[m] = Xm.x * scale;
            oim[m] = Xm.y * scale;
        }
        __syncwarp();
    }
}

// e^{-2 pi i t / N}, t < N, per (device, N); built once, never freed.
std::mutex g_tw_mu;
std::map<std::pair<int, int>, float2 *> g_tw;

int twiddles(int N, const float2 **out)
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
bool factor_half(int H, FftGeom &g)
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
    if (!factor_half(g.H, g)) return ZFPX_EINVAL;
    const int warps = std::max(1, std::min(kMaxWarps, kRowBytesBudget / (int)(2 * sizeof(float2) * g.H)));
    for (int s = 0, r = g.H; s < g.nst; s++) {
        g.rp[s] = make_fastdiv((uint32_t)(r / g.radix[s]));
        r /= g.radix[s];
    }
    g.nrows = n[1] * n[2]; g.ny = n[1];
    g.is1 = stride[1]; g.is2 = stride[2]; g.os1 = ostride[1]; g.os2 = ostride[2];
    const float2 *tw = nullptr;
    int rc = twiddles(g.N, &tw);
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
