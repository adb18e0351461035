// Device pieces of the longitude FFT (fourier.cu), shared with the fused
// decode + FFT kernel (rfft_fused.cu): the radix stages of the self-sorting
// H-point complex FFT and the split of its result into the N = 2H-point real
// transform's wavenumbers (see fourier.cu for the method).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace zfpx {
namespace fft {

constexpr int kMaxStages = 16;
constexpr int kMaxHalf = 4096;                  // N <= 8192

// n / d for n d < 2^32 as one multiply-high by m = ceil(2^32 / d) (exact in
// that range: m d - 2^32 < d); d = 1 has m = 0 and returns n.
struct FastDiv {
    uint32_t d, m;
    __device__ __forceinline__ uint32_t div(uint32_t n) const { return m ? __umulhi(n, m) : n; }
};
__host__ inline FastDiv make_fastdiv(uint32_t d)
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


// A row of H complex values (8-byte aligned) into shared memory by
// asynchronous copies, every copy of the lane in flight at once (16 bytes each
// when both addresses are on 16 bytes and H is even, else 8), as one commit
// group; wait_rows() waits for the lane's groups.
__device__ __forceinline__ void load_row_async(float2 *dst, const float2 *src, int H, int lane)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(dst);
    if (((((uint32_t)(uintptr_t)src) | s) & 15u) == 0 && (H & 1) == 0) {
        for (int k = lane; k < H / 2; k += 32)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s + 16u * (uint32_t)k), "l"(src + 2 * k)
                         : "memory");
    } else {
        for (int k = lane; k < H; k += 32)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s + 8u * (uint32_t)k), "l"(src + k)
                         : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void wait_rows() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// One row: X holds the H complex values z_k = x_2k + i x_2k+1 on entry; Y is
// scratch of H values; writes X_m / N, m < K, to ore / oim.  One warp.
__device__ __forceinline__ void rfft_row(float2 *X, float2 *Y, const float2 *__restrict__ tw, const FftGeom &g,
                                         int lane, float *ore, float *oim)
{
    const int H = g.H;
    const float scale = 1.0f / (float)g.N;
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

}  // namespace fft

// Host side (fourier.cu): e^{-2 pi i t / N}, t < N, per (device, N), built once
// and never freed; and the radix plan of H (false if H has a prime factor other
// than 2, 3, 5).
int fft_twiddles(int N, const float2 **out);
bool fft_plan_half(int H, fft::FftGeom &g);

}  // namespace zfpx
