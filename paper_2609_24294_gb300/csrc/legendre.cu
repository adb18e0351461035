// The Legendre transform: the latitude half of the spectral transform, run on
// theta-pencils after the second transposition (Sec. II-A: associated
// Legendre functions on Gauss-Legendre latitudes; Sec. II-B: the lambda ->
// theta all-to-all makes every latitude column local).  For the wavenumber
// fields F_m(mu_j) (real and imaginary parts, [lev][lat][m]) it returns
//     a_l^m = sum_j w_j Pbar_l^m(mu_j) F_m(mu_j),   0 <= m <= l <= T,
// with Pbar normalised to int Pbar^2 dmu = 1 (Condon-Shortley phase), mu_j the
// Gauss-Legendre nodes north to south and w_j their weights.
//
// Pbar_l^m(-mu) = (-1)^(l+m) Pbar_l^m(mu) and the nodes and weights are
// symmetric, so with S_j = F(mu_j) + F(-mu_j) and A_j = F(mu_j) - F(-mu_j)
// over the northern half (j < nlat/2)
//     a_l^m = sum_{j < nlat/2} w_j Pbar_l^m(mu_j) (l + m even ? S_j : A_j),
// half the work of the full sum.  For each order m and parity p of l + m this
// is a product (rows l of that parity) x (nlat/2) times (nlat/2) x (2 nlev)
// (columns: the real parts of all levels, then the imaginary parts).
//
// The plan holds the table w_j Pbar_l^m(mu_j), j < nlat/2, built on the host
// in double precision (Newton iteration for the nodes, the three-term
// recurrences for Pbar) and rounded once to float; values below the double
// range near the poles for large m are 0.  A fold kernel writes S and A per
// order (a transpose through shared memory, into the caller's workspace);
// a tiled single-precision GEMM kernel (64 x 64 outputs per CTA, 16-deep
// k steps through double-buffered shared memory, 8 x 4 per thread) forms the
// products and scatters them into the triangular output.  Tensor cores are not used: the
// transform needs float32 accuracy, which TF32 and BF16 do not give.
#include <algorithm>
#include <cmath>
#include <vector>
#include <cuda_runtime.h>

#include "zfpx_internal.h"

struct LegItem {
    int32_t m, p, r0, nr;   // order, parity of l + m, first row (of that parity), rows in this tile
    int32_t ldm;            // row length of this (m, p) table block: its row count rounded up to 4
    int32_t pad;
    int64_t aoff;           // float offset of the (m, p) table block ([nlat/2][ldm], latitude-major)
};

struct zfpx_legendre_s {
    int nlat = 0, T = 0, nh = 0, device = 0;
    float *d_table = nullptr;
    LegItem *d_items = nullptr;
    int nitems = 0;
};

namespace zfpx {
namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16;

struct LegGeom {
    int nlat, nh, T, nlev;
    int ldc;                 // columns of the folded operand per row (2 nlev rounded up to 4)
    int nct;                 // column tiles
    int64_t is1, is2;        // input strides: latitude, level (floats; longitude/wavenumber stride 1)
    int64_t os;              // output level stride (floats)
};

__host__ __device__ __forceinline__ int64_t tri_offset(int m, int T)
{
    return (int64_t)m * (T + 1) - (int64_t)m * (m - 1) / 2;
}

// G[m][p][j][c], c = part * nlev + lev: S (p = 0) and A (p = 1) of part
// `part` of F at level lev, latitude pair (j, nlat - 1 - j), order m.
// Block (32, 8) over 32 orders x 32 levels of one (j, part).
__global__ void __launch_bounds__(256) legendre_fold_kernel(const float *__restrict__ re, const float *__restrict__ im,
                                                            float *__restrict__ G, LegGeom g)
{
    __shared__ float sS[32][33], sA[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int m0 = blockIdx.x * 32, lev0 = blockIdx.y * 32;
    const int j = blockIdx.z >> 1, part = blockIdx.z & 1;
    const float *F = part ? im : re;
    const int jn = g.nlat - 1 - j;
    for (int i = ty; i < 32; i += 8) {
        const int lev = lev0 + i, m = m0 + tx;
        float a = 0.f, b = 0.f;
        if (lev < g.nlev && m <= g.T) {
            a = __ldg(F + lev * g.is2 + (int64_t)j * g.is1 + m);
            b = __ldg(F + lev * g.is2 + (int64_t)jn * g.is1 + m);
        }
        sS[i][tx] = a + b;
        sA[i][tx] = a - b;
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        const int m = m0 + i, lev = lev0 + tx;
        if (m <= g.T && lev < g.nlev) {
            const int64_t row = ((int64_t)m * 2 * g.nh + j) * g.ldc + part * g.nlev + lev;
            G[row] = sS[tx][i];
            G[row + (int64_t)g.nh * g.ldc] = sA[tx][i];
        }
    }
}

// 64 x 64 outputs per CTA of 128 threads (2 x 2 warps of 32 x 32), each thread
// 8 rows x 4 columns; 16-deep k
// steps, the next step's tiles loaded into registers while the current one is
// multiplied out of the other shared-memory buffer (one barrier per step).
// A tiles come from the latitude-major table block ([j][row], rows of one
// parity contiguous), B tiles from the folded operand ([j][column]): both are
// float4 rows copied into shared memory as they are.
constexpr int kGemmThreads = 128;

__global__ void __launch_bounds__(kGemmThreads) legendre_gemm_kernel(const float *__restrict__ table,
                                                                     const float *__restrict__ G,
                                                                     const LegItem *__restrict__ items, LegGeom g,
                                                                     float *__restrict__ are, float *__restrict__ aim)
{
    __shared__ __align__(16) float As[2][kBK][kBM];
    __shared__ __align__(16) float Bs[2][kBK][kBN];
    const int tid = threadIdx.x;
    const LegItem it = items[blockIdx.x / g.nct];
    const int c0 = (blockIdx.x % g.nct) * kBN;
    const float *A = table + it.aoff;
    const float *B = G + ((int64_t)it.m * 2 + it.p) * g.nh * g.ldc;
    const int N = 2 * g.nlev;
    // warp w holds rows 32 (w >> 1) .. + 31 and columns 32 (w & 1) .. + 31; lane
    // (ly, lx) rows 8 ly .. + 7 and columns 4 lx .. + 3 of those.  A warp whose
    // rows or columns all lie past the tile's edge skips the multiply-adds.
    const int w = tid >> 5, lane = tid & 31;
    const int r_base = 32 * (w >> 1) + 8 * (lane >> 3), c_base = 32 * (w & 1) + 4 * (lane & 7);
    const bool active = 32 * (w >> 1) < it.nr && c0 + 32 * (w & 1) < N;
    // loaders: two float4 of A and two of B per thread; element e = tid + 128 h
    // covers k-row e / 16 and the four rows / columns 4 (e % 16) .. + 3
    float4 ra[2], rb[2];
    auto load = [&](int k0) {
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int e = tid + kGemmThreads * h, kr = e >> 4, q4 = (e & 15) * 4;
            const bool kin = k0 + kr < g.nh;
            ra[h] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (kin && it.r0 + q4 < it.ldm)
                ra[h] = __ldg(reinterpret_cast<const float4 *>(A + (int64_t)(k0 + kr) * it.ldm + it.r0 + q4));
            rb[h] = make_float4(0.f, 0.f, 0.f, 0.f);
            const int c = c0 + q4;
            if (kin && c < N) {
                rb[h] = __ldg(reinterpret_cast<const float4 *>(B + (int64_t)(k0 + kr) * g.ldc + c));
                if (c + 1 >= N) rb[h].y = 0.f;
                if (c + 2 >= N) rb[h].z = 0.f;
                if (c + 3 >= N) rb[h].w = 0.f;
            }
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int e = tid + kGemmThreads * h, kr = e >> 4, q4 = (e & 15) * 4;
            *reinterpret_cast<float4 *>(&As[buf][kr][q4]) = ra[h];
            *reinterpret_cast<float4 *>(&Bs[buf][kr][q4]) = rb[h];
        }
    };
    float acc[8][4] = {};
    load(0);
    store(0);
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < g.nh; k0 += kBK) {
        const bool more = k0 + kBK < g.nh;
        if (more) load(k0 + kBK);
        if (active)
#pragma unroll
        for (int k = 0; k < kBK; k++) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][k][r_base]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][k][r_base + 4]);
            const float4 b = *reinterpret_cast<const float4 *>(&Bs[buf][k][c_base]);
            const float ai[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w}, bj[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 8; i++)
#pragma unroll
                for (int jj = 0; jj < 4; jj++) acc[i][jj] = fmaf(ai[i], bj[jj], acc[i][jj]);
        }
        if (more) store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
    const int64_t base = tri_offset(it.m, g.T) + it.p;     // l = m + p + 2 (r0 + row)
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int row = r_base + i;
        if (row >= it.nr) continue;
        const int64_t o = base + 2 * (int64_t)(it.r0 + row);
#pragma unroll
        for (int jj = 0; jj < 4; jj++) {
            const int c = c0 + c_base + jj;
            if (c >= N) continue;
            const int part = c >= g.nlev, lev = part ? c - g.nlev : c;
            (part ? aim : are)[(int64_t)lev * g.os + o] = acc[i][jj];
        }
    }
}

// Gauss-Legendre nodes (north to south) and weights: Newton's iteration on
// P_n from the initial guesses cos(pi (i + 3/4) / (n + 1/2)), the upper half
// mirrored.
void gauss_legendre(int n, std::vector<double> &mu, std::vector<double> &w)
{
    const double pi = 3.14159265358979323846264338327950288;
    mu.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; i++) {
        double x = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; k++) {
                const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = x; p0 = 1.0; }
            dp = n * (x * p1 - p0) / -((1.0 - x) * (1.0 + x));
            const double dx = p1 / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        // recompute the derivative at the converged node for the weight
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; k++) {
            const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        if (n == 1) { p1 = x; p0 = 1.0; }
        dp = n * (x * p1 - p0) / -((1.0 - x) * (1.0 + x));
        mu[i] = x;
        mu[n - 1 - i] = -x;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - x) * (1.0 + x) * dp * dp);   // 1 - x^2 without cancellation
    }
}

}  // namespace
}  // namespace zfpx

using namespace zfpx;

extern "C" {

int zfpx_legendre_create(zfpx_legendre *out, int nlat, int T)
{
    if (!out) return ZFPX_EINVAL;
    *out = nullptr;
    if (nlat < 2 || nlat % 2 || nlat > 1 << 15 || T < 0 || T + 1 > nlat) return ZFPX_EINVAL;   // grid z = nlat
    auto *p = new zfpx_legendre_s();
    p->nlat = nlat; p->T = T; p->nh = nlat / 2;
    if (cudaGetDevice(&p->device) != cudaSuccess) { delete p; return ZFPX_ECUDA; }
    std::vector<double> mu, w;
    gauss_legendre(nlat, mu, w);
    const int nh = p->nh;
    std::vector<double> s(nh);
    for (int j = 0; j < nh; j++) s[j] = std::sqrt(std::max(0.0, 1.0 - mu[j] * mu[j]));
    // blocks: for m = 0..T, parity 0 then 1, a [nh][ldm] block whose column i
    // is the row l = m + p + 2 i (ldm = that parity's row count rounded up to 4)
    int64_t total = 0;
    for (int m = 0; m <= T; m++)
        for (int par = 0; par < 2; par++) {
            const int cnt = (T - m - par) >= 0 ? (T - m - par) / 2 + 1 : 0;
            total += (int64_t)nh * ((cnt + 3) / 4 * 4);
        }
    std::vector<float> tab((size_t)total, 0.0f);
    std::vector<LegItem> items;
    std::vector<double> pmm(nh, std::sqrt(0.5)), P0(nh), P1(nh), P2(nh);
    std::vector<std::vector<double>> rows;
    int64_t blk = 0;
    for (int m = 0; m <= T; m++) {
        if (m > 0) {
            const double f = -std::sqrt((2.0 * m + 1.0) / (2.0 * m));
            for (int j = 0; j < nh; j++) pmm[j] *= f * s[j];
        }
        const int L = T - m + 1;
        rows.assign(L, std::vector<double>(nh));
        rows[0] = pmm;
        if (L > 1)
            for (int j = 0; j < nh; j++) rows[1][j] = std::sqrt(2.0 * m + 3.0) * mu[j] * pmm[j];
        for (int i = 2; i < L; i++) {
            const double l = m + i;
            const double a = std::sqrt((4.0 * l * l - 1.0) / (l * l - (double)m * m));
            const double b = std::sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
            for (int j = 0; j < nh; j++) rows[i][j] = a * (mu[j] * rows[i - 1][j] - b * rows[i - 2][j]);
        }
        for (int par = 0; par < 2; par++) {
            const int cnt = par < L ? (L - 1 - par) / 2 + 1 : 0;
            const int ldm = (cnt + 3) / 4 * 4;
            for (int c = 0; c < cnt; c++)
                for (int j = 0; j < nh; j++)
                    tab[(size_t)(blk + (int64_t)j * ldm + c)] = (float)(w[j] * rows[par + 2 * c][j]);
            for (int r0 = 0; r0 < cnt; r0 += kBM)
                items.push_back(LegItem{m, par, r0, std::min(kBM, cnt - r0), ldm, 0, blk});
            blk += (int64_t)nh * ldm;
        }
    }
    p->nitems = (int)items.size();
    if (cudaMalloc(&p->d_table, tab.size() * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&p->d_items, items.size() * sizeof(LegItem)) != cudaSuccess ||
        cudaMemcpy(p->d_table, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->d_items, items.data(), items.size() * sizeof(LegItem), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(p->d_table);
        cudaFree(p->d_items);
        delete p;
        return ZFPX_ECUDA;
    }
    *out = p;
    return ZFPX_OK;
}

int zfpx_gauss_legendre(int n, double *mu, double *w)
{
    if (n < 1 || n > (1 << 15) || !mu || !w) return ZFPX_EINVAL;
    std::vector<double> m, ww;
    gauss_legendre(n, m, ww);
    for (int i = 0; i < n; i++) { mu[i] = m[i]; w[i] = ww[i]; }
    return ZFPX_OK;
}

void zfpx_legendre_destroy(zfpx_legendre p)
{
    if (!p) return;
    cudaFree(p->d_table);
    cudaFree(p->d_items);
    delete p;
}

size_t zfpx_legendre_workspace_bytes(zfpx_legendre p, int64_t nlev)
{
    if (!p || nlev < 1) return 0;
    const int64_t ldc = (2 * nlev + 3) / 4 * 4;
    return (size_t)((int64_t)(p->T + 1) * 2 * p->nh * ldc * (int64_t)sizeof(float));
}

int zfpx_legendre_forward(zfpx_legendre p, const float *d_re, const float *d_im, const int64_t n[3],
                          const int64_t stride[3], float *d_are, float *d_aim, int64_t out_stride, void *d_work,
                          size_t work_bytes, void *stream)
{
    if (!p || !d_re || !d_im || !n || !stride || !d_are || !d_aim || !d_work) return ZFPX_EINVAL;
    if (n[0] < p->T + 1 || n[1] != p->nlat || n[2] < 1 || n[2] > (1 << 20)) return ZFPX_EINVAL;
    if (stride[0] != 1 || stride[1] < 0 || stride[2] < 0) return ZFPX_EINVAL;
    if (out_stride < (int64_t)(p->T + 1) * (p->T + 2) / 2) return ZFPX_EINVAL;
    if (((uintptr_t)d_re & 3u) || ((uintptr_t)d_im & 3u) || ((uintptr_t)d_are & 3u) || ((uintptr_t)d_aim & 3u) ||
        ((uintptr_t)d_work & 15u))
        return ZFPX_EINVAL;
    if (work_bytes < zfpx_legendre_workspace_bytes(p, n[2])) return ZFPX_ESIZE;
    LegGeom g{};
    g.nlat = p->nlat; g.nh = p->nh; g.T = p->T; g.nlev = (int)n[2];
    g.ldc = (2 * g.nlev + 3) / 4 * 4;
    g.nct = (2 * g.nlev + kBN - 1) / kBN;
    g.is1 = stride[1]; g.is2 = stride[2]; g.os = out_stride;
    float *G = static_cast<float *>(d_work);
    const dim3 fgrid((p->T + 1 + 31) / 32, (g.nlev + 31) / 32, 2 * p->nh);
    legendre_fold_kernel<<<fgrid, dim3(32, 8), 0, (cudaStream_t)stream>>>(d_re, d_im, G, g);
    count_launch();
    int rc = check_launch();
    if (rc) return rc;
    const int64_t nblk = (int64_t)p->nitems * g.nct;
    if (nblk > 0x7fffffff) return ZFPX_EINVAL;
    legendre_gemm_kernel<<<(unsigned)nblk, kGemmThreads, 0, (cudaStream_t)stream>>>(p->d_table, G, p->d_items, g, d_are,
                                                                                 d_aim);
    count_launch();
    return check_launch();
}

}  // extern "C"
