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
// (k, f + L s) for s < p.  Radices 4, 2, 3 and 5; twiddles e^{-2 pi i t / N}
// from a table built on the host in double precision and rounded once.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <cuda_runtime.h>

#include "zfpx_internal.h"

namespace zfpx {
namespace {

constexpr int kFftThreads = 256;
constexpr int kMaxStages = 16;
constexpr int kMaxHalf = 4096;                  // N <= 8192
constexpr int kRowBytesBudget = 40 * 1024;      // shared memory for the rows of one CTA (several CTAs per SM)

constexpr int kMaxRows = 16;

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
    FastDiv nb[kMaxStages];   // H / p of each stage
    FastDiv rp[kMaxStages];   // r / p of each stage
    FastDiv dH, dK;
    int R;                    // rows per CTA pass (<= kMaxRows)
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

template <int P>
__device__ __forceinline__ void small_dft(float2 (&u)[5], float2 (&v)[5], const float2 (&w)[5])
{
    if (P == 2) {
        v[0] = cadd(u[0], u[1]);
        v[1] = csub(u[0], u[1]);
    } else if (P == 4) {
        // w_4 = -i: v_s = sum_q u_q (-i)^{s q}
        const float2 a = cadd(u[0], u[2]), b = csub(u[0], u[2]);
        const float2 c = cadd(u[1], u[3]), d = cmul_mi(csub(u[1], u[3]));
        v[0] = cadd(a, c);
        v[1] = cadd(b, d);
        v[2] = csub(a, c);
        v[3] = csub(b, d);
    } else {
        // P = 3 or 5: v_s = sum_q u_q w_P^{(s q) mod P}
#pragma unroll
        for (int s = 0; s < P; s++) {
            float2 acc = u[0];
#pragma unroll
            for (int q = 1; q < P; q++) acc = cadd(acc, cmul(u[q], w[(s * q) % P]));
            v[s] = acc;
        }
    }
}

template <int P>
__device__ __forceinline__ void fft_stage(const float2 *X, float2 *Y, const float2 *__restrict__ tw, int N, int H,
                                          int L, int nr, FastDiv dnb, FastDiv drp)
{
    const int Lp = L * P, r = H / L, rp = (int)drp.d, nb = (int)dnb.d;
    float2 w[5];
#pragma unroll
    for (int j = 0; j < 5; j++) w[j] = j < P ? __ldg(tw + (int64_t)j * (N / P)) : make_float2(0.f, 0.f);
    const int tstep = N / Lp;                   // w_{pL}^{t} = e^{-2 pi i t / (pL)} = tw[t N / (pL)]
    for (int idx = threadIdx.x; idx < nr * nb; idx += blockDim.x) {
        const int row = (int)dnb.div(idx), b = idx - row * nb;
        const int f = (int)drp.div(b), k = b - f * rp;
        const float2 *x = X + row * H;
        float2 *y = Y + row * H;
        float2 u[5], v[5];
#pragma unroll
        for (int q = 0; q < P; q++) {
            const float2 a = x[k + rp * q + r * f];
            u[q] = q ? cmul(a, __ldg(tw + f * q * tstep)) : a;
        }
        small_dft<P>(u, v, w);
#pragma unroll
        for (int s = 0; s < P; s++) y[k + rp * (f + L * s)] = v[s];
    }
}

__global__ void __launch_bounds__(kFftThreads) rfft_lon_kernel(const float *__restrict__ in, float *__restrict__ re,
                                                                float *__restrict__ im, const float2 *__restrict__ tw,
                                                                FftGeom g)
{
    extern __shared__ float2 fsm[];
    __shared__ int64_t s_in[kMaxRows], s_out[kMaxRows];
    const int H = g.H;
    const float scale = 1.0f / (float)g.N;
    for (int64_t r0 = (int64_t)blockIdx.x * g.R; r0 < g.nrows; r0 += (int64_t)gridDim.x * g.R) {
        const int nr = (int)min((int64_t)g.R, g.nrows - r0);
        float2 *X = fsm, *Y = fsm + g.R * H;
        if ((int)threadIdx.x < nr) {
            const int64_t gr = r0 + threadIdx.x, y = gr % g.ny, z = gr / g.ny;
            s_in[threadIdx.x] = z * g.is2 + y * g.is1;
            s_out[threadIdx.x] = z * g.os2 + y * g.os1;
        }
        __syncthreads();
        // rows in, as H complex values each (8-byte aligned pairs)
#pragma unroll 4
        for (int idx = threadIdx.x; idx < nr * H; idx += blockDim.x) {
            const int q = (int)g.dH.div(idx), k = idx - q * H;
            X[idx] = __ldg(reinterpret_cast<const float2 *>(in + s_in[q]) + k);
        }
        __syncthreads();
        int L = 1;
        for (int s = 0; s < g.nst; s++) {
            const int p = g.radix[s];
            if (p == 4) fft_stage<4>(X, Y, tw, g.N, H, L, nr, g.nb[s], g.rp[s]);
            else if (p == 2) fft_stage<2>(X, Y, tw, g.N, H, L, nr, g.nb[s], g.rp[s]);
            else if (p == 3) fft_stage<3>(X, Y, tw, g.N, H, L, nr, g.nb[s], g.rp[s]);
            else fft_stage<5>(X, Y, tw, g.N, H, L, nr, g.nb[s], g.rp[s]);
            __syncthreads();
            float2 *t = X; X = Y; Y = t;
            L *= p;
        }
        // X now holds Z_f at f.  X_m = E_m + e^{-2 pi i m / N} O_m with
        // E_m = (Z_m + conj Z_{H-m}) / 2, O_m = (Z_m - conj Z_{H-m}) / (2i).
#pragma unroll 2
        for (int idx = threadIdx.x; idx < nr * g.K; idx += blockDim.x) {
            const int q = (int)g.dK.div(idx), m = idx - q * g.K;
            const float2 zm = X[q * H + (m == H ? 0 : m)];
            const float2 zc = X[q * H + (m == 0 ? 0 : H - m)];
            const float2 E = make_float2(0.5f * (zm.x + zc.x), 0.5f * (zm.y - zc.y));
            const float2 O = make_float2(0.5f * (zm.y + zc.y), -0.5f * (zm.x - zc.x));
            const float2 Xm = cadd(E, cmul(O, __ldg(tw + m)));
            const int64_t o = s_out[q] + m;
            re[o] = Xm.x * scale;
            im[o] = Xm.y * scale;
        }
        __syncthreads();
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

// H = 4^a 2^b 3^c 5^d -> radices (4s first); false if another prime divides H
bool factor_half(int H, FftGeom &g)
{
    g.nst = 0;
    int h = H;
    for (int p : {4, 2, 3, 5})
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
    g.R = std::max(1, std::min(kMaxRows, kRowBytesBudget / (int)(2 * sizeof(float2) * g.H)));
    g.dH = make_fastdiv((uint32_t)g.H);
    g.dK = make_fastdiv((uint32_t)K);
    for (int s = 0, r = g.H; s < g.nst; s++) {
        g.nb[s] = make_fastdiv((uint32_t)(g.H / g.radix[s]));
        g.rp[s] = make_fastdiv((uint32_t)(r / g.radix[s]));
        r /= g.radix[s];
    }
    g.nrows = n[1] * n[2]; g.ny = n[1];
    g.is1 = stride[1]; g.is2 = stride[2]; g.os1 = ostride[1]; g.os2 = ostride[2];
    const float2 *tw = nullptr;
    int rc = twiddles(g.N, &tw);
    if (rc) return rc;
    const size_t smem = 2 * sizeof(float2) * (size_t)g.R * g.H;
    if (cudaFuncSetAttribute(rfft_lon_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return ZFPX_ECUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rfft_lon_kernel, kFftThreads, smem) != cudaSuccess)
        return ZFPX_ECUDA;
    const int64_t groups = (g.nrows + g.R - 1) / g.R;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(groups, (int64_t)num_sms() * std::max(1, per_sm)));
    rfft_lon_kernel<<<grid, kFftThreads, smem, (cudaStream_t)stream>>>(d_in, d_re, d_im, tw, g);
    count_launch();
    return check_launch();
}

}  // extern "C"
