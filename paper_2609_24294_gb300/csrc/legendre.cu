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
// range near the poles for large m are 0.  Both operands are stored K-major
// (the latitude index j contiguous): the table as rows l of each (m, p)
// block, and the folded operand, which a fold kernel writes per call into the
// caller's workspace, as rows (m, p, column).
//
// The products run on the tensor cores (tcgen05.mma, kind::tf32) with float32
// accuracy from a three-term split: a = a_hi + a_lo with a_hi = a truncated
// to TF32 (what the MMA reads of a float32 operand) and a_lo = a - a_hi rounded
// to TF32, and a b = a_hi b_hi + a_hi b_lo + a_lo b_hi, accumulated in float32
// in tensor memory; the dropped a_lo b_lo and the TF32 rounding of the lo
// parts leave about 2^-21 of sum |a b| per product, far below the float32
// dot-product bound the transform is held to.  A CTA of four warps computes a
// 128-row x Nt-column tile of one (m, p) block: one lane of warp 0 keeps TMA
// loads of 32-deep K slices of both operands (128-byte swizzled) up to four
// stages ahead, the other three warps derive the lo tiles in place, one of
// their threads issues the MMAs (three per 8-deep K step) and commits them to
// the stage's mbarrier, which frees the stage for the next load; after the
// last slice each warp reads its 32 rows of the accumulator from tensor
// memory and scatters them into the triangular output.  Every wait is
// bounded; a wait that runs out sets the plan's status word and the CTA
// stops.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <vector>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "zfpx_internal.h"

struct LegItem {
    int32_t m, p, r0, nr;   // order, parity of l + m, first row (of that parity), rows in this tile
    int64_t arow;           // first table row of this (m, p) block (rows of the K-major table tensor)
};

struct zfpx_legendre_s {
    int nlat = 0, T = 0, nh = 0, nhs = 0, device = 0;
    int64_t table_rows = 0;
    float *d_table = nullptr;   // K-major: [table_rows][nhs] floats, columns >= nh zero
    float *d_table_lo = nullptr;   // the table's TF32 low parts (tf32_lo), same layout
    LegItem *d_items = nullptr;
    int *d_status = nullptr;    // 0, or the code of a wait that ran out
    int nitems = 0;
    CUtensorMap tmap_table;     // TMA view of the table: {nh, table_rows}, boxes {32, 128}
    CUtensorMap tmap_table_lo;  // the same view of its low parts
};

namespace zfpx {
namespace {

constexpr int kBM = 128;        // rows per CTA tile (the MMA's M)
constexpr int kBK = 32;         // K per stage: one 128-byte swizzle row of float32
constexpr long long kSpinLimit = 1ll << 26;   // about a second of polling

struct LegGeom {
    int nlat, nh, nhs, T, nlev;
    int N;                   // columns: 2 nlev
    int nt, ntiles;          // columns per tile (a multiple of 16, <= 256), tiles
    int ncp;                 // column rows per (m, p) in the workspace: ntiles * nt
    int64_t is1, is2;        // input strides: latitude, level (floats; wavenumber stride 1)
    int64_t os;              // output level stride (floats)
};

__host__ __device__ __forceinline__ int64_t tri_offset(int m, int T)
{
    return (int64_t)m * (T + 1) - (int64_t)m * (m - 1) / 2;
}

// G[((m * 2 + p) * ncp + c) * nhs + j], c = part * nlev + lev: S (p = 0) and A
// (p = 1) of part `part` of F at level lev, latitude pair (j, nlat - 1 - j),
// order m; columns j in [nh, nhs) are written as zeros.  Block (32, 8) over 32
// orders x 32 latitudes of one (level, part).
__global__ void __launch_bounds__(256) legendre_fold_kernel(const float *__restrict__ re, const float *__restrict__ im,
                                                            float *__restrict__ G, LegGeom g)
{
    __shared__ float sS[32][33], sA[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int m0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    const int lev = blockIdx.z >> 1, part = blockIdx.z & 1;
    const float *F = (part ? im : re) + lev * g.is2;
    for (int i = ty; i < 32; i += 8) {
        const int j = j0 + i, m = m0 + tx;
        float a = 0.f, b = 0.f;
        if (j < g.nh && m <= g.T) {
            a = __ldg(F + (int64_t)j * g.is1 + m);
            b = __ldg(F + (int64_t)(g.nlat - 1 - j) * g.is1 + m);
        }
        sS[i][tx] = a + b;                            // [j][m]
        sA[i][tx] = a - b;
    }
    __syncthreads();
    const int c = part * g.nlev + lev;
    for (int i = ty; i < 32; i += 8) {
        const int m = m0 + i, j = j0 + tx;
        if (m <= g.T && j < g.nhs) {
            const int64_t row = ((int64_t)m * 2 * g.ncp + c) * g.nhs + j;
            G[row] = sS[tx][i];
            G[row + (int64_t)g.ncp * g.nhs] = sA[tx][i];
        }
    }
}

// The same fold for fields whose rows start on 16 bytes (latitude and level
// strides multiples of 4, 16-byte aligned bases): tiles of 128 orders x 32
// latitudes, every load and store a 16-byte vector (four orders in, four
// latitudes out).  Block (32, 8).
__global__ void __launch_bounds__(256) legendre_fold4_kernel(const float *__restrict__ re,
                                                             const float *__restrict__ im, float *__restrict__ G,
                                                             LegGeom g)
{
    __shared__ float sS[32][129], sA[32][129];          // [latitude][order]
    const int tx = threadIdx.x, ty = threadIdx.y, t = ty * 32 + tx;
    const int m0 = blockIdx.x * 128, j0 = blockIdx.y * 32;
    const int lev = blockIdx.z >> 1, part = blockIdx.z & 1;
    const float *F = (part ? im : re) + lev * g.is2;
    const int m = m0 + 4 * tx;
    for (int i = ty; i < 32; i += 8) {
        const int j = j0 + i;
        float a[4] = {0.f, 0.f, 0.f, 0.f}, b[4] = {0.f, 0.f, 0.f, 0.f};
        if (j < g.nh) {
            const float *rn = F + (int64_t)j * g.is1, *rs = F + (int64_t)(g.nlat - 1 - j) * g.is1;
            if (m + 3 <= g.T) {
                const float4 u = __ldg(reinterpret_cast<const float4 *>(rn + m));
                const float4 v = __ldg(reinterpret_cast<const float4 *>(rs + m));
                a[0] = u.x; a[1] = u.y; a[2] = u.z; a[3] = u.w;
                b[0] = v.x; b[1] = v.y; b[2] = v.z; b[3] = v.w;
            } else {
#pragma unroll
                for (int q = 0; q < 4; q++)
                    if (m + q <= g.T) {
                        a[q] = __ldg(rn + m + q);
                        b[q] = __ldg(rs + m + q);
                    }
            }
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            sS[i][4 * tx + q] = a[q] + b[q];
            sA[i][4 * tx + q] = a[q] - b[q];
        }
    }
    __syncthreads();
    const int c = part * g.nlev + lev;
    const int jj = 4 * (t & 7), j = j0 + jj;              // latitudes j .. j + 3 (nhs is a multiple of 4)
    if (j >= g.nhs) return;
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const int k = (t >> 3) + 32 * r, mm = m0 + k;
        if (mm > g.T) break;
        const int64_t row = ((int64_t)mm * 2 * g.ncp + c) * g.nhs + j;
        *reinterpret_cast<float4 *>(G + row) = make_float4(sS[jj][k], sS[jj + 1][k], sS[jj + 2][k], sS[jj + 3][k]);
        *reinterpret_cast<float4 *>(G + row + (int64_t)g.ncp * g.nhs) =
            make_float4(sA[jj][k], sA[jj + 1][k], sA[jj + 2][k], sA[jj + 3][k]);
    }
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory descriptor of a K-major, 128-byte-swizzled operand
// tile starting at `saddr` (8-row groups 1024 bytes apart)
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);           // start address / 16
    d |= (uint64_t)1u << 16;                             // leading byte offset (not used by swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;                   // stride byte offset / 16
    d |= (uint64_t)1u << 46;                             // descriptor version
    d |= (uint64_t)2u << 61;                             // 128-byte swizzle
    return d;
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    for (long long i = 0; i < kSpinLimit; i++) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                 :: "r"(dst), "l"(map), "r"(x), "r"(y), "r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_expect(uint32_t mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mbar), "r"(bytes) : "memory");
}

// The 3 x TF32 split of a float32 a: hi = a with its 13 low mantissa bits
// cleared (what the tensor core reads of a), lo = a - hi (exact) rounded to
// TF32, to nearest with ties away from zero, by adding half of the last kept
// bit to the magnitude bits and clearing the rest (the rounding of PTX's
// cvt.rna.tf32.f32, as integer operations).
__host__ __device__ inline float tf32_lo(float a)
{
#ifdef __CUDA_ARCH__
    const float l = a - __uint_as_float(__float_as_uint(a) & 0xffffe000u);
    return __uint_as_float((__float_as_uint(l) + 0x1000u) & 0xffffe000u);
#else
    uint32_t u;
    std::memcpy(&u, &a, 4);
    u &= 0xffffe000u;
    float h;
    std::memcpy(&h, &u, 4);
    const float l = a - h;
    std::memcpy(&u, &l, 4);
    u = (u + 0x1000u) & 0xffffe000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
#endif
}

// lo = tf32_lo(a) over n 16-byte chunks, by the `nthr` threads numbered t
__device__ __forceinline__ void split_lo(const uint8_t *raw, uint8_t *lo, int nchunks, int t, int nthr)
{
    for (int i = t; i < nchunks; i += nthr) {
        const float4 a = reinterpret_cast<const float4 *>(raw)[i];
        float v[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int q = 0; q < 4; q++) {
            v[q] = tf32_lo(v[q]);
        }
        reinterpret_cast<float4 *>(lo)[i] = make_float4(v[0], v[1], v[2], v[3]);
    }
}

// Persistent and warp-specialised: one CTA per SM walks the tiles t =
// blockIdx.x, blockIdx.x + gridDim.x, ... (a tile: 128 rows x nt columns of one
// (m, p) block).  Roles:
//   warp 0 (one lane)  TMA producer: the K slices of every tile in turn, up to
//                      `stages` ahead, a stage refilled once the MMAs that read
//                      it have completed (mma_bar);
//   warps 1-11         wait for a slice (full_bar), derive the data tile's lo
//                      part (the table's comes by TMA), meet at a named
//                      barrier; one of their threads issues the slice's
//                      MMAs into the tile's accumulator and commits them to the
//                      stage, and after a tile's last slice to acc_full;
//   warps 12-15        epilogue: once a tile's accumulator is complete, each
//                      reads the 32 rows of its TMEM lane quadrant, scatters
//                      them into the triangular output and frees the
//                      accumulator (acc_empty).
// Two accumulators of 256 columns (all of the SM's tensor memory) alternate
// between tiles, so a tile's epilogue overlaps the next tile's MMAs.
// Dynamic shared memory: `stages` x {A raw, A lo, B raw, B lo}, 1024-aligned.
constexpr int kMaxStages = 4;
constexpr int kConsumers = 352;                 // warps 1-11
constexpr int kMmaThreads = 512;                // 16 warps
constexpr int kAccCols = 256;

// A bounded wait that also gives up once another role has failed.
__device__ __forceinline__ bool role_wait(uint32_t mbar, uint32_t parity, volatile int *fail)
{
    for (long long i = 0; i < kSpinLimit; i++) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
        if (ok) return true;
        if ((i & 1023) == 1023 && *fail) return false;
    }
    return false;
}

__global__ void __launch_bounds__(kMmaThreads, 1)
legendre_mma_kernel(const __grid_constant__ CUtensorMap tmap_a, const __grid_constant__ CUtensorMap tmap_alo,
                    const __grid_constant__ CUtensorMap tmap_b,
                    const LegItem *__restrict__ items, LegGeom g, int stages, int ntiles_total,
                    float *__restrict__ are, float *__restrict__ aim, int *__restrict__ status)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kMaxStages], mma_bar[kMaxStages], acc_full[2], acc_empty[2];
    __shared__ uint32_t tmem_base;
    __shared__ int fail;
    volatile int *vfail = &fail;
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nt = g.nt;
    const uint32_t a_bytes = kBM * 128, b_bytes = (uint32_t)nt * 128;
    const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;
    auto a_raw = [&](int s) { return smem + s * stage_bytes; };
    auto a_lo = [&](int s) { return smem + s * stage_bytes + a_bytes; };
    auto b_raw = [&](int s) { return smem + s * stage_bytes + 2 * a_bytes; };
    auto b_lo = [&](int s) { return smem + s * stage_bytes + 2 * a_bytes + b_bytes; };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_base)), "n"(2 * kAccCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        fail = 0;
        for (int s = 0; s < stages; s++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&full_bar[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mma_bar[s])));
        }
        for (int a = 0; a < 2; a++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&acc_full[a])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" :: "r"(smem_u32(&acc_empty[a])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" :: "l"(&tmap_a) : "memory");
        asm volatile("prefetch.tensormap [%0];" :: "l"(&tmap_alo) : "memory");
        asm volatile("prefetch.tensormap [%0];" :: "l"(&tmap_b) : "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const int nk = (g.nh + kBK - 1) / kBK;

    if (warp == 0) {
        // ---- producer
        if (tid == 0) {
            int i = 0;                                   // slice count over all tiles of this CTA
            for (int t = blockIdx.x; t < ntiles_total && !*vfail; t += gridDim.x) {
                const LegItem it = items[t / g.ntiles];
                const int ct = t % g.ntiles;
                const int arow = (int)(it.arow + it.r0);
                const int brow = (int)(((int64_t)it.m * 2 + it.p) * g.ncp + (int64_t)ct * nt);
                for (int k = 0; k < nk; k++, i++) {
                    const int s = i % stages;
                    if (i >= stages && !role_wait(smem_u32(&mma_bar[s]), (uint32_t)(i / stages - 1) & 1u, vfail)) {
                        *vfail = 1;
                        break;
                    }
                    const uint32_t fb = smem_u32(&full_bar[s]);
                    mbar_expect(fb, 2 * a_bytes + b_bytes);
                    tma_load_2d(smem_u32(a_raw(s)), &tmap_a, k * kBK, arow, fb);
                    tma_load_2d(smem_u32(a_lo(s)), &tmap_alo, k * kBK, arow, fb);
                    tma_load_2d(smem_u32(b_raw(s)), &tmap_b, k * kBK, brow, fb);
                }
            }
        }
    } else if (warp <= 11) {
        // ---- lo tiles and MMAs
        const int c = tid - 32;
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(nt >> 3) << 17) |
                               ((uint32_t)(kBM >> 4) << 24);
        int i = 0, j = 0;                                // slices, tiles of this CTA
        bool stop = false;
        for (int t = blockIdx.x; t < ntiles_total && !stop; t += gridDim.x, j++) {
            const int acc = j & 1;
            const uint32_t d = tmem + (uint32_t)(acc * kAccCols);
            // the accumulator's previous tile must have been read out
            if (tid == 32 && j >= 2 && !role_wait(smem_u32(&acc_empty[acc]), (uint32_t)(j / 2 - 1) & 1u, vfail))
                *vfail = 1;
            for (int k = 0; k < nk; k++, i++) {
                const int s = i % stages;
                if (!role_wait(smem_u32(&full_bar[s]), (uint32_t)(i / stages) & 1u, vfail)) *vfail = 1;
                split_lo(b_raw(s), b_lo(s), (int)(b_bytes / 16), c, kConsumers);   // the table's come with it
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                // the named barrier, reducing every consumer's view of the failure
                // flag so that all of them take the same branch
                uint32_t any_fail;
                asm volatile("{\n\t.reg .pred q, r;\n\tsetp.ne.b32 q, %1, 0;\n\t"
                             "bar.red.or.pred r, 1, %2, q;\n\tselp.u32 %0, 1, 0, r;\n\t}"
                             : "=r"(any_fail) : "r"((uint32_t)*vfail), "n"(kConsumers) : "memory");
                if (any_fail) { stop = true; break; }
                if (tid == 32) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t ah = smem_u32(a_raw(s)), al = smem_u32(a_lo(s));
                    const uint32_t bh = smem_u32(b_raw(s)), bl = smem_u32(b_lo(s));
#pragma unroll
                    for (int q = 0; q < kBK / 8; q++) {     // 8-deep K steps, 32 bytes apart in the swizzle row
                        const uint64_t dah = sw128_desc(ah + 32 * q), dal = sw128_desc(al + 32 * q);
                        const uint64_t dbh = sw128_desc(bh + 32 * q), dbl = sw128_desc(bl + 32 * q);
#pragma unroll
                        for (int e = 0; e < 3; e++) {
                            const uint64_t da = e == 2 ? dal : dah, db = e == 1 ? dbl : dbh;
                            const uint32_t accum = (k > 0 || q > 0 || e > 0) ? 1u : 0u;
                            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                         "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                                         :: "r"(d), "l"(da), "l"(db), "r"(idesc), "r"(accum));
                        }
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 :: "r"(smem_u32(&mma_bar[s])) : "memory");
                    if (k == nk - 1)
                        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                     :: "r"(smem_u32(&acc_full[acc])) : "memory");
                }
            }
        }
    } else {
        // ---- epilogue: warp 12 + q reads TMEM lanes 32 q .. 32 q + 31 (its warp
        // index mod 4 is q, the lane quadrant tcgen05.ld lets it reach)
        const int q = warp - 12, lane = tid & 31;
        int j = 0;
        for (int t = blockIdx.x; t < ntiles_total; t += gridDim.x, j++) {
            const int acc = j & 1;
            const bool got = role_wait(smem_u32(&acc_full[acc]), (uint32_t)(j / 2) & 1u, vfail);
            if (!__all_sync(0xffffffffu, got)) { *vfail = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const LegItem it = items[t / g.ntiles];
            const int ct = t % g.ntiles;
            const int row = 32 * q + lane;
            const bool live = row < it.nr;
            const int64_t o = tri_offset(it.m, g.T) + it.p + 2 * (int64_t)(it.r0 + row);
            for (int c0 = 0; c0 < nt; c0 += 16) {
                uint32_t v[16];
                const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * kAccCols + c0);
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                             : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                               "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                             : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (live) {
#pragma unroll
                    for (int e = 0; e < 16; e++) {
                        const int col = ct * nt + c0 + e;
                        if (col < g.N) {
                            const int part = col >= g.nlev, lev = part ? col - g.nlev : col;
                            (part ? aim : are)[(int64_t)lev * g.os + o] = __uint_as_float(v[e]);
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(&acc_empty[acc])) : "memory");
        }
    }
    __syncthreads();
    if (*vfail && tid == 0) {
        atomicExch(status, 1);
        // let copies and MMAs still in flight land before the CTA leaves
        for (int s = 0; s < stages; s++) {
            mbar_wait(smem_u32(&full_bar[s]), 0u);
            mbar_wait(smem_u32(&mma_bar[s]), 0u);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "n"(2 * kAccCols));
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// TMA view of a K-major float32 matrix: `rows` rows of `k` values (`ld`
// floats apart, ld * 4 a multiple of 16), read as {32 x box_rows} boxes with
// 128-byte swizzle; values past k or rows read as zero.
int make_tmap(CUtensorMap *map, const float *base, int64_t k, int64_t rows, int64_t ld, int box_rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return ZFPX_ECUDA;
    const cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? ZFPX_OK : ZFPX_ECUDA;
}

// columns per tile for N = 2 nlev columns: the fewest tiles of at most 256
// columns, each a multiple of 16
void column_tiles(int N, int &nt, int &ntiles)
{
    ntiles = (N + 255) / 256;
    nt = ((N + ntiles - 1) / ntiles + 15) / 16 * 16;
}

size_t stage_bytes(int nt) { return 2 * kBM * 128 + 2 * (size_t)nt * 128; }

// as many stages (2 .. 4) as fit beside one CTA's static shared memory
int mma_stages(int nt)
{
    const size_t budget = 220 * 1024 - 1024;
    return (int)std::max<size_t>(2, std::min<size_t>(kMaxStages, budget / stage_bytes(nt)));
}

size_t mma_smem_bytes(int nt) { return 1024 + (size_t)mma_stages(nt) * stage_bytes(nt); }

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

namespace {

int legendre_create(zfpx_legendre *out, int nlat, int T)
{
    std::unique_ptr<zfpx_legendre_s> hold(new zfpx_legendre_s());
    zfpx_legendre_s *p = hold.get();
    p->nlat = nlat; p->T = T; p->nh = nlat / 2;
    p->nhs = (p->nh + 3) / 4 * 4;                        // row pitch: a multiple of 16 bytes
    if (cudaGetDevice(&p->device) != cudaSuccess) return ZFPX_ECUDA;
    const int nh = p->nh, nhs = p->nhs;
    // rows: for m = 0..T, parity 0 then 1, one row per l = m + p + 2 i, K-major
    int64_t rows = 0;
    for (int m = 0; m <= T; m++)
        for (int par = 0; par < 2; par++) rows += (T - m - par) >= 0 ? (T - m - par) / 2 + 1 : 0;
    p->table_rows = rows;
    // the two tables (high and low TF32 parts) must fit on the device
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return ZFPX_ECUDA;
    if ((double)std::max<int64_t>(rows, 1) * nhs * 2 * sizeof(float) > (double)total_b) return ZFPX_ENOMEM;
    std::vector<double> mu, w;
    gauss_legendre(nlat, mu, w);
    std::vector<double> s(nh);
    for (int j = 0; j < nh; j++) s[j] = std::sqrt(std::max(0.0, 1.0 - mu[j] * mu[j]));
    std::vector<float> tab((size_t)std::max<int64_t>(rows, 1) * nhs, 0.0f);
    std::vector<LegItem> items;
    std::vector<double> pmm(nh, std::sqrt(0.5));
    std::vector<std::vector<double>> prow;
    int64_t r = 0;
    for (int m = 0; m <= T; m++) {
        if (m > 0) {
            const double f = -std::sqrt((2.0 * m + 1.0) / (2.0 * m));
            for (int j = 0; j < nh; j++) pmm[j] *= f * s[j];
        }
        const int L = T - m + 1;
        prow.assign(L, std::vector<double>(nh));
        prow[0] = pmm;
        if (L > 1)
            for (int j = 0; j < nh; j++) prow[1][j] = std::sqrt(2.0 * m + 3.0) * mu[j] * pmm[j];
        for (int i = 2; i < L; i++) {
            const double l = m + i;
            const double a = std::sqrt((4.0 * l * l - 1.0) / (l * l - (double)m * m));
            const double b = std::sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
            for (int j = 0; j < nh; j++) prow[i][j] = a * (mu[j] * prow[i - 1][j] - b * prow[i - 2][j]);
        }
        for (int par = 0; par < 2; par++) {
            const int cnt = par < L ? (L - 1 - par) / 2 + 1 : 0;
            for (int c = 0; c < cnt; c++)
                for (int j = 0; j < nh; j++) tab[(size_t)(r + c) * nhs + j] = (float)(w[j] * prow[par + 2 * c][j]);
            for (int r0 = 0; r0 < cnt; r0 += kBM)
                items.push_back(LegItem{m, par, r0, std::min(kBM, cnt - r0), r});
            r += cnt;
        }
    }
    p->nitems = (int)items.size();
    std::vector<float> tab_lo(tab.size());
    for (size_t i = 0; i < tab.size(); i++) tab_lo[i] = tf32_lo(tab[i]);
    if (cudaMalloc(&p->d_table, tab.size() * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&p->d_table_lo, tab.size() * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&p->d_items, std::max<size_t>(items.size(), 1) * sizeof(LegItem)) != cudaSuccess ||
        cudaMalloc(&p->d_status, sizeof(int)) != cudaSuccess ||
        cudaMemcpy(p->d_table, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->d_table_lo, tab_lo.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->d_items, items.data(), items.size() * sizeof(LegItem), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess ||
        make_tmap(&p->tmap_table, p->d_table, nh, std::max<int64_t>(rows, 1), nhs, kBM) != ZFPX_OK ||
        make_tmap(&p->tmap_table_lo, p->d_table_lo, nh, std::max<int64_t>(rows, 1), nhs, kBM) != ZFPX_OK) {
        cudaFree(p->d_table);
        cudaFree(p->d_table_lo);
        cudaFree(p->d_items);
        cudaFree(p->d_status);
        return ZFPX_ECUDA;
    }
    *out = hold.release();
    return ZFPX_OK;
}

}  // namespace

extern "C" {

int zfpx_legendre_create(zfpx_legendre *out, int nlat, int T)
{
    if (!out) return ZFPX_EINVAL;
    *out = nullptr;
    if (nlat < 2 || nlat % 2 || nlat > 1 << 15 || T < 0 || T + 1 > nlat) return ZFPX_EINVAL;   // grid z = nlat
    // the host tables are built before any device memory is taken: a failed
    // host allocation leaves nothing behind
    try {
        return legendre_create(out, nlat, T);
    } catch (const std::bad_alloc &) {
        return ZFPX_ENOMEM;
    }
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
    cudaFree(p->d_table_lo);
    cudaFree(p->d_items);
    cudaFree(p->d_status);
    delete p;
}

size_t zfpx_legendre_workspace_bytes(zfpx_legendre p, int64_t nlev)
{
    if (!p || nlev < 1 || nlev > (1 << 20)) return 0;
    int nt, ntiles;
    column_tiles((int)(2 * nlev), nt, ntiles);
    return (size_t)((int64_t)(p->T + 1) * 2 * ntiles * nt * p->nhs * (int64_t)sizeof(float));
}

int zfpx_legendre_status(zfpx_legendre p)
{
    if (!p) return ZFPX_EINVAL;
    int v = 0;
    if (cudaMemcpy(&v, p->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return ZFPX_ECUDA;
    return v ? ZFPX_ETIMEOUT : ZFPX_OK;
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
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ZFPX_ECUDA;
    if (dev != p->device) return ZFPX_EINVAL;
    LegGeom g{};
    g.nlat = p->nlat; g.nh = p->nh; g.nhs = p->nhs; g.T = p->T; g.nlev = (int)n[2];
    g.N = 2 * g.nlev;
    column_tiles(g.N, g.nt, g.ntiles);
    g.ncp = g.nt * g.ntiles;
    g.is1 = stride[1]; g.is2 = stride[2]; g.os = out_stride;
    const int64_t grows = (int64_t)(p->T + 1) * 2 * g.ncp;
    if (grows > 0x7fffffff || p->table_rows > 0x7fffffff) return ZFPX_EINVAL;
    float *G = static_cast<float *>(d_work);
    CUtensorMap tmap_g;
    int rc = make_tmap(&tmap_g, G, p->nh, grows, p->nhs, g.nt);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (2 * g.nlev > 65535) return ZFPX_EINVAL;
    const bool vec4 = stride[1] % 4 == 0 && stride[2] % 4 == 0 && !((uintptr_t)d_re & 15u) && !((uintptr_t)d_im & 15u);
    if (vec4) {
        const dim3 fgrid((p->T + 1 + 127) / 128, (p->nhs + 31) / 32, 2 * g.nlev);
        legendre_fold4_kernel<<<fgrid, dim3(32, 8), 0, st>>>(d_re, d_im, G, g);
    } else {
        const dim3 fgrid((p->T + 1 + 31) / 32, (p->nhs + 31) / 32, 2 * g.nlev);
        legendre_fold_kernel<<<fgrid, dim3(32, 8), 0, st>>>(d_re, d_im, G, g);
    }
    count_launch();
    rc = check_launch();
    if (rc) return rc;
    const int64_t nblk = (int64_t)p->nitems * g.ntiles;
    if (nblk > 0x7fffffff) return ZFPX_EINVAL;
    if (nblk == 0) return ZFPX_OK;
    const size_t smem = mma_smem_bytes(g.nt);
    if (cudaFuncSetAttribute(legendre_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return ZFPX_ECUDA;
    const int grid = (int)std::min<int64_t>(nblk, num_sms());      // persistent: one CTA per SM
    legendre_mma_kernel<<<grid, kMmaThreads, smem, st>>>(p->tmap_table, p->tmap_table_lo, tmap_g, p->d_items, g,
                                                          mma_stages(g.nt), (int)nblk,
                                                          d_are, d_aim, p->d_status);
    count_launch();
    return check_launch();
}

}  // extern "C"
