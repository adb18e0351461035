// Batched compression of many fields on a grid of ragged rows in one
// persistent launch (encode) and one (decode): fields with different level
// counts, block dimensionality (1-D rows or 3-D row-quads) and rate (8 or 16)
// share the launch.  Grid: rows back to back, row r holding len[r] points
// (the octahedral reduced Gaussian grid has len = 20 + 4i, mirrored).
//
// Blocks (ZFP fixed rate, paper Sec. II-C): dims 1 = 4 consecutive points of
// one row of one level; dims 3 = 4 points x 4 consecutive rows x 4
// consecutive levels, covering x < max length of the row-quad, shorter rows
// repeating their last point and a missing last row / level repeating the
// last one.  Stream of a field: items (dims 3: level quads; dims 1: levels)
// in level order, inside an item the blocks in row (row-quad) order then along
// x; fields at 256-byte aligned offsets.
//
// Work list: every (field, item) is split into work units of consecutive
// blocks (3-D: 32, one per lane; 1-D: 32 lb1, lb1 per lane); units are sorted
// so that fields of one (dims, rate) class are contiguous, each class a queue
// that warps of the persistent grid claim units from (for_each_unit below).
// The class is uniform across a warp.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cstring>
#include <deque>
#include <map>
#include <unordered_map>
#include <new>
#include <tuple>
#include <vector>

#include "zfpx_internal.h"
#include "zfpx_block.cuh"
#include "zfpx_smem.cuh"
#include "zfpx_enc3.cuh"

namespace zfpx {
namespace {

using namespace blk;

struct FieldDevB {
    const float *src;      // (level 0, first point of row row0)
    float *dst;
    int64_t src_ls, dst_ls;  // elements between levels
    int64_t out_off;       // byte offset of the field's stream
    int64_t b0;            // first global block of the row range (row-quad or row prefix)
    int64_t roff0;         // grid offset of row row0
    int32_t nlev, dims, rate, vec;
    int32_t row0, row1;    // rows [row0, row1)
};

struct ItemDevB {
    int64_t unit0;     // first chunk
    int64_t out_off;   // byte offset of the item's stream (absolute)
    int64_t nblocks;
    int32_t field, z0, nz, pad;
};

struct GridDev {
    const int64_t *row_off;   // nrows
    const int32_t *row_len;   // nrows
    const int64_t *qpre;      // nq + 1: first block of each row-quad (dims 3)
    const int64_t *rpre;      // nrows + 1: first block of each row (dims 1)
    int32_t nrows, nq;
};

// Items of one (dims, rate) kind: units [u0, u0 + n).  cum1 is the share of
// all work up to and including this group, which picks the SMs for which it
// is the home group.
struct GroupDev {
    int64_t u0, n;
    int32_t dims, rate;
    float cum1;
    int32_t pad;
};
constexpr int kMaxGroups = 4;

struct BatchGeom {
    const ItemDevB *items;
    const FieldDevB *fields;
    GridDev grid;
    int nitems;
    int64_t nunits;
    GroupDev groups[kMaxGroups];
    int ngroups;
    int lb1;              // 1-D units: 32 lb1 blocks, lb1 per lane
    int upc;              // units a warp claims at a time (one atomic per claim)
    uint32_t *ctr;        // ngroups work counters, zero at launch
};

__device__ __forceinline__ int item_of_unit(const ItemDevB *items, int n, int64_t u)
{
    int lo = 0, hi = n - 1;   // last item with unit0 <= u
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&items[mid].unit0) <= u) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// A 1-D plane table, built by the CTA when the batch holds 1-D items.
template <class Tab>
__device__ __forceinline__ void fill_plane4(const BatchGeom &bg, Tab &tab)
{
    bool any1 = false;
    for (int i = 0; i < bg.ngroups; i++) any1 |= bg.groups[i].dims == 1;
    if (!any1) return;
    plane4_fill(tab, threadIdx.x, blockDim.x);
    __syncthreads();
}

// Work distribution of the batch kernels.  A batch with no more units than
// the grid has warps gives each warp one unit.  Otherwise each (dims, rate)
// group is a queue of units claimed upc at a time (one atomic add per claim)
// by whole warps.  A CTA starts on
// its home group -- the SMs are split between groups in proportion to their
// work, so an SM mostly runs one kind's code and keeps it in its instruction
// cache -- and then helps the other groups until every queue is empty.
template <class Fn>
__device__ __forceinline__ void for_each_unit(const BatchGeom &bg, int lane, Fn &&fn)
{
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    if (bg.nunits <= nwarps) {                                   // a small batch: one unit per warp, no claims
        const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
        if (c < bg.nunits) {
            int gi = 0;
            while (gi + 1 < bg.ngroups && c >= bg.groups[gi + 1].u0) gi++;
            fn(bg.groups[gi], c, item_of_unit(bg.items, bg.nitems, c));
        }
        return;
    }
    uint32_t smid, nsmid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    asm volatile("mov.u32 %0, %%nsmid;" : "=r"(nsmid));
    const float x = ((float)smid + 0.5f) / (float)nsmid;
    int home = 0;
    while (home + 1 < bg.ngroups && x >= bg.groups[home].cum1) home++;
    for (int t = 0; t < bg.ngroups; t++) {
        const int gi = (home + t) % bg.ngroups;
        const GroupDev G = bg.groups[gi];
        uint32_t *ctr = bg.ctr + gi;
        const uint32_t C = (uint32_t)bg.upc;
        uint32_t u = 0;
        if (lane == 0) u = atomicAdd(ctr, C);
        u = __shfl_sync(0xffffffffu, u, 0);
        while ((int64_t)u < G.n) {
            uint32_t next = 0;                                   // claimed ahead: its latency hides behind fn
            if (lane == 0) next = atomicAdd(ctr, C);
            next = __shfl_sync(0xffffffffu, next, 0);
            // the claim's units in order; a unit's item is the last one starting at or before it
            const uint32_t ue = (uint32_t)min((int64_t)u + C, G.n);
            int ii = item_of_unit(bg.items, bg.nitems, G.u0 + u);
            for (uint32_t v = u; v < ue; v++) {
                const int64_t c = G.u0 + v;
                while (ii + 1 < bg.nitems && __ldg(&bg.items[ii + 1].unit0) <= c) ii++;
                fn(G, c, ii);
            }
            u = next;
        }
    }
}

__device__ __forceinline__ int upper_index(const int64_t *pre, int n, int64_t b)
{
    int lo = 0, hi = n - 1;   // last i with pre[i] <= b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(pre + mid) <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The same index for a block at most 31 past one whose index is `start` (a
// unit's first block, searched once by the whole warp): a forward walk,
// which on grids of rows several blocks long takes a step or two at most.
__device__ __forceinline__ int upper_index_from(const int64_t *pre, int n, int start, int64_t b)
{
    int i = start;
    while (i + 1 < n && __ldg(pre + i + 1) <= b) i++;
    return i;
}

// 64 values of a 3-D block of row-quad q, x block bxi, levels z0.. (rows past
// the field's row range, points past a row's end and levels past nz repeat
// the last one).  Row by row: each row's loads can start as soon as its own
// offset has arrived, which keeps the latency of a lone small batch low (a
// variant testing all four rows first was a little faster on big batches and
// a quarter slower on small ones).
__device__ __forceinline__ void gather_quad(const FieldDevB &f, const GridDev &g, int q, int bxi, int z0, int nz,
                                            float (&x)[64])
{
    const int x0 = 4 * bxi;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int r = min(4 * q + j, f.row1 - 1);
        const int64_t roff = __ldg(g.row_off + r) - f.roff0;
        const int len = __ldg(g.row_len + r);
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const float *row = f.src + (int64_t)(z0 + min(k, nz - 1)) * f.src_ls + roff;
            if (f.vec && x0 + 4 <= len) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(row + x0));
                x[16 * k + 4 * j] = v.x; x[16 * k + 4 * j + 1] = v.y;
                x[16 * k + 4 * j + 2] = v.z; x[16 * k + 4 * j + 3] = v.w;
            } else {
#pragma unroll
                for (int i = 0; i < 4; i++) x[16 * k + 4 * j + i] = __ldg(row + min(x0 + i, len - 1));
            }
        }
    }
}

// The inverse: only points inside the field's rows, the rows' lengths and
// the item's levels are written.
__device__ __forceinline__ void scatter_quad(const FieldDevB &f, const GridDev &g, int q, int bxi, int z0, int nz,
                                             const float (&x)[64])
{
    const int x0 = 4 * bxi;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int r = 4 * q + j;
        if (r >= f.row1) continue;
        const int64_t roff = __ldg(g.row_off + r) - f.roff0;
        const int len = __ldg(g.row_len + r);
        if (x0 >= len) continue;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (k >= nz) continue;
            float *row = f.dst + (int64_t)(z0 + k) * f.dst_ls + roff;
            if (f.vec && x0 + 4 <= len) {
                *reinterpret_cast<float4 *>(row + x0) =
                    make_float4(x[16 * k + 4 * j], x[16 * k + 4 * j + 1], x[16 * k + 4 * j + 2], x[16 * k + 4 * j + 3]);
            } else {
#pragma unroll
                for (int i = 0; i < 4; i++)
                    if (x0 + i < len) row[x0 + i] = x[16 * k + 4 * j + i];
            }
        }
    }
}

// Every lane of the warp calls it (the encoder's loops are warp-wide); the
// tile of `v` is zero on entry and left zero.
template <int RATE>
__device__ __forceinline__ void enc3_chunk(const FieldDevB &f, const GridDev &g, const ItemDevB &it, int64_t b0,
                                           int nact, int lane, const enc3::View &v, uint8_t *out)
{
    const bool valid = lane < nact;
    float x[64];
    {
        // lanes past the unit's last block load that block and code nothing
        const int64_t bg = b0 + (valid ? lane : nact - 1) + f.b0;
        const int q = upper_index_from(g.qpre, g.nq + 1, upper_index(g.qpre, g.nq + 1, b0 + f.b0), bg);
        const int bxi = (int)(bg - __ldg(g.qpre + q));
        gather_quad(f, g, q, bxi, it.z0, it.nz, x);
    }
    enc3::encode<RATE>(x, valid, v, lane);
    __syncwarp();
    enc3::store_stream<RATE>(v, lane, valid, out + it.out_off + (b0 + lane) * RATE * 8);
    __syncwarp();
}

// A 1-D unit: 32 lb1 consecutive blocks, lane l coding blocks b0 + l + 32 j
// (each step of j one coalesced load and store across the warp).  The
// blocks go in groups of kLoads1 per lane, all of a group's loads issued
// before any is coded, so a warp keeps that many 16-byte loads in flight.
constexpr int kLoads1 = 4;

template <int RATE>
__device__ __forceinline__ void enc1_unit(const FieldDevB &f, const GridDev &g, const ItemDevB &it, int64_t b0,
                                          int lb1, int lane, const Plane4Enc &tab, uint8_t *out)
{
    int r = upper_index(g.rpre, g.nrows + 1, b0 + f.b0);
    const float *src = f.src + (int64_t)it.z0 * f.src_ls - f.roff0;
#pragma unroll 1
    for (int j0 = 0; j0 < lb1; j0 += kLoads1) {
        float x[kLoads1][4];
#pragma unroll
        for (int k = 0; k < kLoads1; k++) {
            const int64_t b = b0 + 32 * (j0 + k) + lane;
            x[k][0] = x[k][1] = x[k][2] = x[k][3] = 0.0f;
            if (j0 + k >= lb1 || b >= it.nblocks) continue;
            const int64_t bg = b + f.b0;
            r = upper_index_from(g.rpre, g.nrows + 1, r, bg);
            const int x0 = 4 * (int)(bg - __ldg(g.rpre + r));
            const int len = __ldg(g.row_len + r);
            const float *row = src + __ldg(g.row_off + r);
            if (f.vec && x0 + 4 <= len) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(row + x0));
                x[k][0] = v.x; x[k][1] = v.y; x[k][2] = v.z; x[k][3] = v.w;
            } else {
#pragma unroll
                for (int i = 0; i < 4; i++) x[k][i] = __ldg(row + min(x0 + i, len - 1));
            }
        }
        uint64_t w[kLoads1];
        encode_blocks1<RATE, kLoads1>(x, tab, w);
#pragma unroll
        for (int k = 0; k < kLoads1; k++) {
            const int64_t b = b0 + 32 * (j0 + k) + lane;
            if (j0 + k >= lb1 || b >= it.nblocks) continue;
            if (RATE == 16) reinterpret_cast<uint64_t *>(out + it.out_off)[b] = w[k];
            else reinterpret_cast<uint32_t *>(out + it.out_off)[b] = (uint32_t)w[k];
        }
    }
}

template <int WARPS>
__global__ void __launch_bounds__(32 * WARPS)
batch_encode_kernel(BatchGeom bg, uint8_t *__restrict__ out)
{
    __shared__ enc3::Shared<16> sh[WARPS];             // rate-16 sized, shared by both rates
    __shared__ Plane4Enc tab;
    fill_plane4(bg, tab);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const enc3::View v = sh[wid].view();
    enc3::clear(v, lane, enc3::kWords<16>);
    __syncwarp();
    for_each_unit(bg, lane, [&](const GroupDev &G, int64_t c, int ii) {
        const ItemDevB it = bg.items[ii];
        const FieldDevB f = bg.fields[it.field];
        if (G.dims == 3) {
            const int64_t b0 = (c - it.unit0) * 32;
            const int nact = (int)min((int64_t)32, it.nblocks - b0);
            if (G.rate == 8) enc3_chunk<8>(f, bg.grid, it, b0, nact, lane, v, out);
            else enc3_chunk<16>(f, bg.grid, it, b0, nact, lane, v, out);
        } else {
            const int64_t b0 = (c - it.unit0) * 32 * bg.lb1;
            if (G.rate == 8) enc1_unit<8>(f, bg.grid, it, b0, bg.lb1, lane, tab, out);
            else enc1_unit<16>(f, bg.grid, it, b0, bg.lb1, lane, tab, out);
        }
    });
}

template <int RATE>
__device__ __forceinline__ void dec3_lane(const FieldDevB &f, const GridDev &g, const ItemDevB &it, int64_t b,
                                          int start, int lane, const uint8_t *in, uint32_t *t32, uint64_t *wpl)
{
    const uint4 *src4 = reinterpret_cast<const uint4 *>(in + it.out_off) + b * (RATE / 2);
#pragma unroll
    for (int i = 0; i < RATE / 2; i++) {
        const uint4 v = __ldg(src4 + i);
        t32[(4 * i) * 32 + lane] = v.x;
        t32[(4 * i + 1) * 32 + lane] = v.y;
        t32[(4 * i + 2) * 32 + lane] = v.z;
        t32[(4 * i + 3) * 32 + lane] = v.w;
    }
#pragma unroll
    for (int r = 0; r < kTileZeroRows<RATE>; r++) t32[(2 * RATE + r) * 32 + lane] = 0u;
    const int64_t bg = b + f.b0;
    const int q = upper_index_from(g.qpre, g.nq + 1, start, bg);
    const int bxi = (int)(bg - __ldg(g.qpre + q));
    float x[64];
    const StreamTile tile{t32, lane};
    SmemPlanes pl{wpl, lane};
    decode_block3_tile<RATE>(tile, x, pl);
    scatter_quad(f, g, q, bxi, it.z0, it.nz, x);
}

template <int RATE>
__device__ __forceinline__ void dec1_unit(const FieldDevB &f, const GridDev &g, const ItemDevB &it, int64_t b0,
                                          int lb1, int lane, const Plane4Dec &tab, const uint8_t *in)
{
    int r = upper_index(g.rpre, g.nrows + 1, b0 + f.b0);
    float *dst = f.dst + (int64_t)it.z0 * f.dst_ls - f.roff0;
#pragma unroll 1
    for (int j0 = 0; j0 < lb1; j0 += kLoads1) {
        uint64_t w[kLoads1];
#pragma unroll
        for (int k = 0; k < kLoads1; k++) {
            const int64_t b = b0 + 32 * (j0 + k) + lane;
            w[k] = 0;
            if (j0 + k >= lb1 || b >= it.nblocks) continue;
            if (RATE == 16) w[k] = __ldg(reinterpret_cast<const uint64_t *>(in + it.out_off) + b);
            else w[k] = __ldg(reinterpret_cast<const uint32_t *>(in + it.out_off) + b);
        }
        float xs[kLoads1][4];
        decode_blocks1<RATE, kLoads1>(w, tab, xs);
#pragma unroll
        for (int k = 0; k < kLoads1; k++) {
            const int64_t b = b0 + 32 * (j0 + k) + lane;
            if (j0 + k >= lb1 || b >= it.nblocks) continue;
            const float (&x)[4] = xs[k];
            const int64_t bg = b + f.b0;
            r = upper_index_from(g.rpre, g.nrows + 1, r, bg);
            const int x0 = 4 * (int)(bg - __ldg(g.rpre + r));
            const int len = __ldg(g.row_len + r);
            float *row = dst + __ldg(g.row_off + r);
            if (f.vec && x0 + 4 <= len) {
                *reinterpret_cast<float4 *>(row + x0) = make_float4(x[0], x[1], x[2], x[3]);
            } else {
#pragma unroll
                for (int i = 0; i < 4; i++)
                    if (x0 + i < len) row[x0 + i] = x[i];
            }
        }
    }
}

template <int WARPS>
__global__ void __launch_bounds__(32 * WARPS)
batch_decode_kernel(BatchGeom bg, const uint8_t *__restrict__ in)
{
    __shared__ uint32_t stile[WARPS][(2 * 16 + 2) * 32];
    __shared__ uint64_t splanes[WARPS][32 * 32];
    __shared__ Plane4Dec tab;
    fill_plane4(bg, tab);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for_each_unit(bg, lane, [&](const GroupDev &G, int64_t c, int ii) {
        const ItemDevB it = bg.items[ii];
        const FieldDevB f = bg.fields[it.field];
        if (G.dims == 3) {
            const int64_t b0 = (c - it.unit0) * 32;
            const int nact = (int)min((int64_t)32, it.nblocks - b0);
            if (lane < nact) {
                const int start = upper_index(bg.grid.qpre, bg.grid.nq + 1, b0 + f.b0);
                if (G.rate == 8) dec3_lane<8>(f, bg.grid, it, b0 + lane, start, lane, in, stile[wid], splanes[wid]);
                else dec3_lane<16>(f, bg.grid, it, b0 + lane, start, lane, in, stile[wid], splanes[wid]);
            }
        } else {
            const int64_t b0 = (c - it.unit0) * 32 * bg.lb1;
            if (G.rate == 8) dec1_unit<8>(f, bg.grid, it, b0, bg.lb1, lane, tab, in);
            else dec1_unit<16>(f, bg.grid, it, b0, bg.lb1, lane, tab, in);
        }
        __syncwarp();
    });
}

}  // namespace
}  // namespace zfpx

namespace zfpx {
namespace {

// Grid tables shared by every batch on one grid (host copies and device).
struct GridHost {
    int nrows = 0, nq = 0;
    std::vector<int64_t> roff, qpre, rpre;
    std::vector<int32_t> rlen;
    bool mult4 = true;
    int64_t *d_row_off = nullptr;
    int32_t *d_row_len = nullptr;
    int64_t *d_qpre = nullptr, *d_rpre = nullptr;

    int init(const int64_t *row_len, int n)
    {
        nrows = n;
        nq = (n + 3) / 4;
        roff.assign(n, 0);
        rlen.assign(n, 0);
        qpre.assign(nq + 1, 0);
        rpre.assign(n + 1, 0);
        int64_t o = 0;
        for (int r = 0; r < n; r++) {
            if (row_len[r] < 1 || row_len[r] > (1 << 30)) return ZFPX_EINVAL;
            roff[r] = o;
            o += row_len[r];
            rlen[r] = (int32_t)row_len[r];
            mult4 = mult4 && (row_len[r] % 4 == 0);
        }
        for (int q = 0; q < nq; q++) {
            int64_t mx = 0;
            for (int j = 0; j < 4 && 4 * q + j < n; j++) mx = std::max(mx, row_len[4 * q + j]);
            qpre[q + 1] = qpre[q] + (mx + 3) / 4;
        }
        for (int r = 0; r < n; r++) rpre[r + 1] = rpre[r] + (row_len[r] + 3) / 4;
        return ZFPX_OK;
    }
    GridDev dev() const { return GridDev{d_row_off, d_row_len, d_qpre, d_rpre, nrows, nq}; }
    void free_dev()
    {
        cudaFree(d_row_off); cudaFree(d_row_len); cudaFree(d_qpre); cudaFree(d_rpre);
        d_row_off = nullptr; d_row_len = nullptr; d_qpre = nullptr; d_rpre = nullptr;
    }
};

template <class T>
int upload(T **dptr, const std::vector<T> &h)
{
    if (h.empty()) return ZFPX_OK;
    if (cudaMalloc((void **)dptr, h.size() * sizeof(T)) != cudaSuccess) return ZFPX_ENOMEM;
    if (cudaMemcpy(*dptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) return ZFPX_ECUDA;
    return ZFPX_OK;
}

int upload_grid(GridHost &g)
{
    int rc = upload(&g.d_row_off, g.roff);
    if (!rc) rc = upload(&g.d_row_len, g.rlen);
    if (!rc) rc = upload(&g.d_qpre, g.qpre);
    if (!rc) rc = upload(&g.d_rpre, g.rpre);
    return rc;
}

int check_field(const GridHost &g, const zfpx_field &F)
{
    if (F.nlev < 1 || (F.dims != 1 && F.dims != 3) || !valid_codec_rate(F.rate)) return ZFPX_EINVAL;
    const int r0 = F.row0, r1 = (F.row0 == 0 && F.row1 == 0) ? g.nrows : F.row1;
    if (r0 < 0 || r1 > g.nrows || r0 >= r1) return ZFPX_EINVAL;
    if (F.dims == 3 && ((r0 & 3) || ((r1 & 3) && r1 != g.nrows))) return ZFPX_EINVAL;
    const int64_t span = g.roff[r1 - 1] + g.rlen[r1 - 1] - g.roff[r0];
    const int64_t dls = F.dst_lev_stride ? F.dst_lev_stride : F.lev_stride;
    if (F.nlev > 1 && (F.lev_stride < span || dls < span)) return ZFPX_EINVAL;
    return ZFPX_OK;
}

// Blocks of one item of field F (all items of a field have the same count).
int64_t field_item_blocks(const GridHost &g, const zfpx_field &F, int r0, int r1)
{
    if (F.dims == 3) return g.qpre[(r1 + 3) / 4] - g.qpre[r0 / 4];
    return g.rpre[r1] - g.rpre[r0];
}

int64_t field_stream_bytes(const GridHost &g, const zfpx_field &F, int r0, int r1)
{
    const int64_t per_block = F.dims == 3 ? 8 * F.rate : F.rate / 2;
    const int64_t items = F.dims == 3 ? (F.nlev + 3) / 4 : F.nlev;
    return items * field_item_blocks(g, F, r0, r1) * per_block;
}

// Blocks of one work unit: 32 for 3-D items (one per lane), 32 lb1 for 1-D.
constexpr int kDefaultLb1 = 16;
constexpr int kMaxLb1 = 64;
constexpr int kDefaultUpc = 4;
constexpr int kMaxUpc = 64;
inline int64_t unit_blocks(int dims, int lb1) { return dims == 3 ? 32 : 32 * (int64_t)lb1; }

// Field and item descriptors of a set of fields whose streams start at the
// given byte offsets; items grouped by (dims, rate) class.
void build_work(const GridHost &g, const zfpx_field *fields, const int64_t *stream_off, int nfields, int lb1,
                std::vector<FieldDevB> &fd, std::vector<ItemDevB> &items, int64_t &units,
                std::vector<GroupDev> &groups)
{
    fd.resize(nfields);
    for (int f = 0; f < nfields; f++) {
        const zfpx_field &F = fields[f];
        const int r0 = F.row0, r1 = (F.row0 == 0 && F.row1 == 0) ? g.nrows : F.row1;
        const int64_t dls = F.dst_lev_stride ? F.dst_lev_stride : F.lev_stride;
        const bool vec = g.mult4 && (F.lev_stride % 4 == 0 || F.nlev == 1) && (dls % 4 == 0 || F.nlev == 1) &&
                         !((uintptr_t)F.d_src & 15u) && !((uintptr_t)F.d_dst & 15u);
        FieldDevB d;
        d.src = F.d_src;
        d.dst = F.d_dst;
        d.src_ls = F.lev_stride;
        d.dst_ls = dls;
        d.out_off = stream_off[f];
        d.b0 = F.dims == 3 ? g.qpre[r0 / 4] : g.rpre[r0];
        d.roff0 = g.roff[r0];
        d.nlev = F.nlev; d.dims = F.dims; d.rate = F.rate; d.vec = vec ? 1 : 0;
        d.row0 = r0; d.row1 = r1;
        fd[f] = d;
    }
    std::vector<int> order(nfields);
    for (int f = 0; f < nfields; f++) order[f] = f;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return std::make_tuple(fields[a].dims, fields[a].rate) < std::make_tuple(fields[c].dims, fields[c].rate);
    });
    items.clear();
    units = 0;
    for (int f : order) {
        const zfpx_field &F = fields[f];
        const int r0 = fd[f].row0, r1 = fd[f].row1;
        const int64_t per_block = F.dims == 3 ? 8 * F.rate : F.rate / 2;
        const int64_t blocks = field_item_blocks(g, F, r0, r1);
        const int step = F.dims == 3 ? 4 : 1;
        int64_t ioff = stream_off[f];
        for (int z = 0; z < F.nlev; z += step) {
            ItemDevB it;
            it.unit0 = units;
            it.out_off = ioff;
            it.nblocks = blocks;
            it.field = f;
            it.z0 = z;
            it.nz = std::min(step, F.nlev - z);
            it.pad = 0;
            items.push_back(it);
            units += (blocks + unit_blocks(F.dims, lb1) - 1) / unit_blocks(F.dims, lb1);
            ioff += blocks * per_block;
        }
    }
    // one group per (dims, rate) run of items; work share by values coded
    // (a rate-16 value costs about 15 % more than a rate-8 one)
    groups.clear();
    std::vector<double> work;
    for (const ItemDevB &it : items) {
        const FieldDevB &F = fd[it.field];
        const int64_t ub = unit_blocks(F.dims, lb1);
        const int64_t n = (it.nblocks + ub - 1) / ub;
        if (groups.empty() || groups.back().dims != F.dims || groups.back().rate != F.rate) {
            GroupDev G;
            G.u0 = it.unit0; G.n = 0; G.dims = F.dims; G.rate = F.rate; G.cum1 = 1.0f; G.pad = 0;
            groups.push_back(G);
            work.push_back(0.0);
        }
        groups.back().n += n;
        work.back() += (double)n * (double)ub * (F.dims == 3 ? 64.0 : 4.0) * (F.rate == 16 ? 1.15 : 1.0);
    }
    double total = 0.0, acc = 0.0;
    for (double w : work) total += w;
    for (size_t i = 0; i < groups.size(); i++) {
        acc += work[i];
        groups[i].cum1 = i + 1 == groups.size() ? 2.0f : (float)(acc / total);
    }
}

BatchGeom make_geom(const FieldDevB *d_fields, const ItemDevB *d_items, const GridDev &grid, int nitems,
                    int64_t nunits, const std::vector<GroupDev> &groups, int lb1, int upc, uint32_t *d_ctr)
{
    BatchGeom g;
    g.lb1 = lb1;
    g.upc = upc;
    g.items = d_items;
    g.fields = d_fields;
    g.grid = grid;
    g.nitems = nitems;
    g.nunits = nunits;
    g.ngroups = (int)groups.size();
    for (int i = 0; i < g.ngroups; i++) g.groups[i] = groups[i];
    g.ctr = d_ctr;
    return g;
}

// Warps per CTA the batch kernels are built for: fewer warps per CTA let
// more CTAs share an SM's shared memory (the encoder's per-warp storage is
// about 15 KB).
bool batch_warps_ok(int warps) { return warps == 2 || warps == 3 || warps == 4 || warps == 8; }

template <int W>
const void *batch_kernel(bool encode)
{
    return encode ? (const void *)batch_encode_kernel<W> : (const void *)batch_decode_kernel<W>;
}

template <int W>
void launch_w(bool encode, int grid, const BatchGeom &g, const uint8_t *in, uint8_t *out, cudaStream_t st)
{
    if (encode) batch_encode_kernel<W><<<grid, 32 * W, 0, st>>>(g, out);
    else batch_decode_kernel<W><<<grid, 32 * W, 0, st>>>(g, in);
}

int launch_batch(const BatchGeom &g, int warps, int ctas_per_sm, bool encode, const uint8_t *in, uint8_t *out,
                 cudaStream_t st)
{
    if (g.nunits == 0) return ZFPX_OK;
    if (!batch_warps_ok(warps)) return ZFPX_EINVAL;
    const void *fn = warps == 2 ? batch_kernel<2>(encode) : warps == 3 ? batch_kernel<3>(encode)
                   : warps == 8 ? batch_kernel<8>(encode) : batch_kernel<4>(encode);
    const int fit = occupancy(fn, 32 * warps);
    const int per_sm = ctas_per_sm > 0 ? std::min(ctas_per_sm, fit) : fit;
    const int64_t want = (g.nunits + warps - 1) / warps;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms() * per_sm));
    if (warps == 2) launch_w<2>(encode, grid, g, in, out, st);
    else if (warps == 3) launch_w<3>(encode, grid, g, in, out, st);
    else if (warps == 8) launch_w<8>(encode, grid, g, in, out, st);
    else launch_w<4>(encode, grid, g, in, out, st);
    count_launch();
    return check_launch();
}

}  // namespace
}  // namespace zfpx

struct zfpx_batch_s {
    zfpx::GridHost grid;
    std::vector<zfpx_field> fields;
    std::vector<int64_t> field_off, field_bytes;
    int64_t total = 0;
    int nitems = 0;
    int64_t nunits = 0;
    int warps = 3, ctas_per_sm = 0;     // 0 = as many as fit
    int lb1 = zfpx::kDefaultLb1;        // 1-D blocks per lane of a unit
    int upc = zfpx::kDefaultUpc;        // units per work claim
    zfpx::FieldDevB *d_fields = nullptr;
    zfpx::ItemDevB *d_items = nullptr;
    std::vector<zfpx::GroupDev> groups;
    uint32_t *d_ctr = nullptr;          // work counters: encode 0..3, decode 4..7
};

using namespace zfpx;

extern "C" {

void zfpx_batch_destroy(zfpx_batch b)
{
    if (!b) return;
    b->grid.free_dev();
    cudaFree(b->d_fields);
    cudaFree(b->d_items);
    cudaFree(b->d_ctr);
    delete b;
}

// (Re)builds the batch's field and item tables for its current unit size.
static int batch_work(zfpx_batch b)
{
    std::vector<FieldDevB> fd;
    std::vector<ItemDevB> items;
    build_work(b->grid, b->fields.data(), b->field_off.data(), (int)b->fields.size(), b->lb1, fd, items, b->nunits,
               b->groups);
    b->nitems = (int)items.size();
    cudaFree(b->d_fields);
    cudaFree(b->d_items);
    b->d_fields = nullptr;
    b->d_items = nullptr;
    int rc = upload(&b->d_fields, fd);
    if (!rc) rc = upload(&b->d_items, items);
    return rc;
}

int zfpx_batch_create(zfpx_batch *out, const int64_t *row_len, int nrows, const zfpx_field *fields, int nfields)
{
    if (!out) return ZFPX_EINVAL;
    *out = nullptr;
    if (!row_len || nrows < 1 || !fields || nfields < 1) return ZFPX_EINVAL;
    zfpx_batch_s *b = new (std::nothrow) zfpx_batch_s;
    if (!b) return ZFPX_ENOMEM;
    int rc = b->grid.init(row_len, nrows);
    for (int f = 0; f < nfields && !rc; f++) rc = check_field(b->grid, fields[f]);
    if (rc) { delete b; return rc; }
    b->fields.assign(fields, fields + nfields);
    b->field_off.resize(nfields);
    b->field_bytes.resize(nfields);
    int64_t off = 0;
    for (int f = 0; f < nfields; f++) {
        const zfpx_field &F = fields[f];
        const int r0 = F.row0, r1 = (F.row0 == 0 && F.row1 == 0) ? nrows : F.row1;
        b->field_off[f] = off;
        b->field_bytes[f] = field_stream_bytes(b->grid, F, r0, r1);
        off = (off + b->field_bytes[f] + 255) / 256 * 256;
    }
    b->total = off;
    rc = upload_grid(b->grid);
    if (!rc) rc = batch_work(b);
    if (!rc && cudaMalloc((void **)&b->d_ctr, 2 * kMaxGroups * sizeof(uint32_t)) != cudaSuccess) rc = ZFPX_ENOMEM;
    if (rc) { zfpx_batch_destroy(b); return rc; }
    *out = b;
    return ZFPX_OK;
}

size_t zfpx_batch_bytes(zfpx_batch b) { return b ? (size_t)b->total : 0; }

int64_t zfpx_batch_field_offset(zfpx_batch b, int f)
{
    if (!b || f < 0 || f >= (int)b->fields.size()) return -1;
    return b->field_off[f];
}

size_t zfpx_batch_field_bytes(zfpx_batch b, int f)
{
    if (!b || f < 0 || f >= (int)b->fields.size()) return 0;
    return (size_t)b->field_bytes[f];
}

int zfpx_batch_set_launch(zfpx_batch b, int warps_per_cta, int ctas_per_sm)
{
    if (!b || !batch_warps_ok(warps_per_cta) || ctas_per_sm < 0) return ZFPX_EINVAL;
    b->warps = warps_per_cta;
    b->ctas_per_sm = ctas_per_sm;
    return ZFPX_OK;
}

int zfpx_batch_set_claim_units(zfpx_batch b, int units_per_claim)
{
    if (!b || units_per_claim < 1 || units_per_claim > kMaxUpc) return ZFPX_EINVAL;
    b->upc = units_per_claim;
    return ZFPX_OK;
}

int zfpx_batch_set_unit_blocks(zfpx_batch b, int blocks_per_lane_1d)
{
    if (!b || blocks_per_lane_1d < 1 || blocks_per_lane_1d > kMaxLb1) return ZFPX_EINVAL;
    if (blocks_per_lane_1d == b->lb1) return ZFPX_OK;
    // the tables in use by launches still in flight stay valid until they finish
    if (cudaDeviceSynchronize() != cudaSuccess) return ZFPX_ECUDA;
    b->lb1 = blocks_per_lane_1d;
    return batch_work(b);
}

// Geometry for one launch; its work counters are zeroed on the stream first.
static int batch_geom(zfpx_batch b, bool encode, cudaStream_t st, BatchGeom &g)
{
    uint32_t *ctr = b->d_ctr + (encode ? 0 : kMaxGroups);
    if (cudaMemsetAsync(ctr, 0, kMaxGroups * sizeof(uint32_t), st) != cudaSuccess) return ZFPX_ECUDA;
    g = make_geom(b->d_fields, b->d_items, b->grid.dev(), b->nitems, b->nunits, b->groups, b->lb1, b->upc, ctr);
    return ZFPX_OK;
}

int zfpx_batch_encode(zfpx_batch b, uint8_t *d_out, size_t cap, void *stream)
{
    if (!b || !d_out || ((uintptr_t)d_out & 15u)) return ZFPX_EINVAL;
    if ((int64_t)cap < b->total) return ZFPX_ESIZE;
    for (const zfpx_field &F : b->fields)
        if (!F.d_src || ((uintptr_t)F.d_src & 3u)) return ZFPX_EINVAL;
    BatchGeom g;
    const int rc = batch_geom(b, true, (cudaStream_t)stream, g);
    return rc ? rc : launch_batch(g, b->warps, b->ctas_per_sm, true, nullptr, d_out, (cudaStream_t)stream);
}

int zfpx_batch_decode(zfpx_batch b, const uint8_t *d_in, size_t len, void *stream)
{
    if (!b || !d_in || ((uintptr_t)d_in & 15u)) return ZFPX_EINVAL;
    if ((int64_t)len < b->total) return ZFPX_ESIZE;
    for (const zfpx_field &F : b->fields)
        if (!F.d_dst || ((uintptr_t)F.d_dst & 3u)) return ZFPX_EINVAL;
    BatchGeom g;
    const int rc = batch_geom(b, false, (cudaStream_t)stream, g);
    return rc ? rc : launch_batch(g, b->warps, b->ctas_per_sm, false, d_in, nullptr, (cudaStream_t)stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Serving: a request loop with continuous batching.
//
// Requests are row x level slabs of fields already resident in device memory
// (one zfpx_field each).  A request is admitted when its memory -- its
// compressed stream and its decoded copy -- fits in the server's arena, which
// is one device allocation made at creation and sized by the HBM budget;
// requests that can never fit are refused at submission.  Every pump() puts
// all requests admitted since the previous batch (first come, first served;
// at most max_batch) into one batch -- one encode launch and one decode
// launch -- on the next of `nstreams` streams, so batches launched while
// earlier ones are still running overlap on the device.  poll() reports the
// requests of finished batches; their results stay valid until released,
// which returns their memory to the arena.  The descriptors of a batch go
// through pinned staging buffers, one per stream, reused once the stream's
// previous batch has finished; nothing is allocated after creation.
// Not thread safe: one host thread drives a server.
namespace zfpx {
namespace {

struct ServerReq {
    zfpx_field f;            // d_dst / dst_lev_stride filled in at admission
    int r0, r1;
    int64_t span;            // points per level in the slab
    int64_t stream_bytes, values_bytes, mem_bytes;
    int64_t mem_off = -1;    // arena offset (stream, then values)
    int state = 0;           // 0 queued, 1 in flight, 2 done
    std::chrono::steady_clock::time_point t_submit;
};

struct ServerSlot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    uint8_t *h_stage = nullptr;   // pinned
    uint8_t *d_desc = nullptr;
    size_t cap = 0;
    bool busy = false;
    std::vector<int64_t> ids;
};

// first-fit allocator over the arena with coalescing
struct ArenaAlloc {
    std::map<int64_t, int64_t> free_;   // offset -> size
    int64_t total = 0, used = 0;
    void init(int64_t bytes) { free_.clear(); free_[0] = bytes; total = bytes; used = 0; }
    int64_t take(int64_t n)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                const int64_t off = it->first, rest = it->second - n;
                free_.erase(it);
                if (rest > 0) free_[off + n] = rest;
                used += n;
                return off;
            }
        }
        return -1;
    }
    void give(int64_t off, int64_t n)
    {
        used -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) { it->second += nx->second; free_.erase(nx); }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) { pv->second += it->second; free_.erase(it); }
        }
    }
};

constexpr int kItemsPerRequest = 160;   // descriptor room per admitted request (137 levels + margin)

}  // namespace
}  // namespace zfpx

struct zfpx_server_s {
    zfpx::GridHost grid;
    uint8_t *d_arena = nullptr;
    zfpx::ArenaAlloc arena;
    std::deque<int64_t> queue;
    std::unordered_map<int64_t, zfpx::ServerReq> reqs;
    std::vector<zfpx::ServerSlot> slots;
    int next_slot = 0;
    int64_t next_id = 1;
    int max_batch = 64;
    int warps = 3, ctas_per_sm = 0;
    int lb1 = zfpx::kDefaultLb1;
    int upc = zfpx::kDefaultUpc;
    int min_batch = 1;                  // batching window: launch at min_batch waiting requests
    double max_wait_s = 0.0;            // ... or once the oldest has waited this long
    std::deque<int64_t> completed;
    int64_t batches = 0;
};

extern "C" {

void zfpx_server_destroy(zfpx_server s)
{
    if (!s) return;
    for (auto &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.h_stage) cudaFreeHost(sl.h_stage);
        if (sl.d_desc) cudaFree(sl.d_desc);
    }
    cudaFree(s->d_arena);
    s->grid.free_dev();
    delete s;
}

int zfpx_server_create(zfpx_server *out, const int64_t *row_len, int nrows, size_t arena_bytes, int nstreams,
                       int max_batch)
{
    if (!out) return ZFPX_EINVAL;
    *out = nullptr;
    if (!row_len || nrows < 1 || arena_bytes < 4096 || nstreams < 1 || nstreams > 64 || max_batch < 1 ||
        max_batch > 4096)
        return ZFPX_EINVAL;
    zfpx_server_s *s = new (std::nothrow) zfpx_server_s;
    if (!s) return ZFPX_ENOMEM;
    int rc = s->grid.init(row_len, nrows);
    if (!rc) rc = upload_grid(s->grid);
    if (!rc && cudaMalloc((void **)&s->d_arena, arena_bytes) != cudaSuccess) rc = ZFPX_ENOMEM;
    s->arena.init((int64_t)arena_bytes / 256 * 256);
    s->max_batch = max_batch;
    const size_t cap = (size_t)max_batch * (sizeof(FieldDevB) + kItemsPerRequest * sizeof(ItemDevB)) + 768;
    s->slots.resize(nstreams);
    for (auto &sl : s->slots) {
        if (rc) break;
        sl.cap = cap;
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess)
            rc = ZFPX_ECUDA;
        else if (cudaMallocHost((void **)&sl.h_stage, cap) != cudaSuccess || cudaMalloc((void **)&sl.d_desc, cap) != cudaSuccess)
            rc = ZFPX_ENOMEM;
    }
    if (rc) { zfpx_server_destroy(s); return rc; }
    *out = s;
    return ZFPX_OK;
}

int zfpx_server_set_launch(zfpx_server s, int warps_per_cta, int ctas_per_sm)
{
    if (!s || !batch_warps_ok(warps_per_cta) || ctas_per_sm < 0) return ZFPX_EINVAL;
    s->warps = warps_per_cta;
    s->ctas_per_sm = ctas_per_sm;
    return ZFPX_OK;
}

int zfpx_server_set_batching(zfpx_server s, int min_requests, double max_wait_us)
{
    if (!s || min_requests < 1 || min_requests > s->max_batch || !(max_wait_us >= 0.0) || max_wait_us > 1e7)
        return ZFPX_EINVAL;
    s->min_batch = min_requests;
    s->max_wait_s = max_wait_us * 1e-6;
    return ZFPX_OK;
}

int zfpx_server_set_claim_units(zfpx_server s, int units_per_claim)
{
    if (!s || units_per_claim < 1 || units_per_claim > kMaxUpc) return ZFPX_EINVAL;
    s->upc = units_per_claim;                 // applies to batches launched from now on
    return ZFPX_OK;
}

int zfpx_server_set_unit_blocks(zfpx_server s, int blocks_per_lane_1d)
{
    if (!s || blocks_per_lane_1d < 1 || blocks_per_lane_1d > kMaxLb1) return ZFPX_EINVAL;
    s->lb1 = blocks_per_lane_1d;              // applies to batches launched from now on
    return ZFPX_OK;
}

int zfpx_server_submit(zfpx_server s, const zfpx_field *req, int64_t *id)
{
    if (!s || !req || !id || !req->d_src) return ZFPX_EINVAL;
    int rc = check_field(s->grid, *req);
    if (rc) return rc;
    if (((req->dims == 3 ? (req->nlev + 3) / 4 : req->nlev)) > kItemsPerRequest) return ZFPX_EINVAL;
    ServerReq r;
    r.f = *req;
    r.r0 = req->row0;
    r.r1 = (req->row0 == 0 && req->row1 == 0) ? s->grid.nrows : req->row1;
    r.span = s->grid.roff[r.r1 - 1] + s->grid.rlen[r.r1 - 1] - s->grid.roff[r.r0];
    r.stream_bytes = field_stream_bytes(s->grid, *req, r.r0, r.r1);
    r.values_bytes = 4 * r.span * req->nlev;
    r.mem_bytes = (r.stream_bytes + 255) / 256 * 256 + (r.values_bytes + 255) / 256 * 256;
    if (r.mem_bytes > s->arena.total) return ZFPX_ENOMEM_BUDGET;
    const int64_t rid = s->next_id++;
    r.t_submit = std::chrono::steady_clock::now();
    s->reqs.emplace(rid, r);
    s->queue.push_back(rid);
    *id = rid;
    return ZFPX_OK;
}

static void server_reap(zfpx_server s)
{
    for (auto &sl : s->slots) {
        if (!sl.busy) continue;
        if (cudaEventQuery(sl.done) != cudaSuccess) continue;
        for (int64_t rid : sl.ids) {
            s->reqs[rid].state = 2;
            s->completed.push_back(rid);
        }
        sl.ids.clear();
        sl.busy = false;
    }
}

int zfpx_server_pump(zfpx_server s, int *launched)
{
    if (!s) return ZFPX_EINVAL;
    if (launched) *launched = 0;
    server_reap(s);
    if (s->queue.empty()) return ZFPX_OK;
    // the batching window: wait for min_batch requests unless the oldest has waited max_wait
    if ((int)s->queue.size() < s->min_batch) {
        const double waited = std::chrono::duration<double>(std::chrono::steady_clock::now() -
                                                            s->reqs[s->queue.front()].t_submit).count();
        if (waited < s->max_wait_s) return ZFPX_OK;
    }
    // the next stream whose previous batch has finished
    int si = -1;
    for (int t = 0; t < (int)s->slots.size(); t++) {
        const int c = (s->next_slot + t) % (int)s->slots.size();
        if (!s->slots[c].busy) { si = c; break; }
    }
    if (si < 0) return ZFPX_OK;
    ServerSlot &sl = s->slots[si];
    // admit first come, first served while the arena has room
    std::vector<int64_t> ids;
    while (!s->queue.empty() && (int)ids.size() < s->max_batch) {
        ServerReq &r = s->reqs[s->queue.front()];
        const int64_t off = s->arena.take(r.mem_bytes);
        if (off < 0) break;
        r.mem_off = off;
        r.f.d_dst = reinterpret_cast<float *>(s->d_arena + off + (r.stream_bytes + 255) / 256 * 256);
        r.f.dst_lev_stride = r.span;
        r.state = 1;
        ids.push_back(s->queue.front());
        s->queue.pop_front();
    }
    if (ids.empty()) return ZFPX_OK;
    std::vector<zfpx_field> fields(ids.size());
    std::vector<int64_t> soff(ids.size());
    for (size_t i = 0; i < ids.size(); i++) {
        const ServerReq &r = s->reqs[ids[i]];
        fields[i] = r.f;
        soff[i] = r.mem_off;          // stream first, at the start of the request's memory
    }
    std::vector<FieldDevB> fd;
    std::vector<ItemDevB> items;
    std::vector<GroupDev> groups;
    int64_t units = 0;
    build_work(s->grid, fields.data(), soff.data(), (int)fields.size(), s->lb1, fd, items, units, groups);
    // descriptors: fields, items, then zeroed work counters (encode, decode)
    const size_t fbytes = fd.size() * sizeof(FieldDevB);
    const size_t ioff = (fbytes + 255) / 256 * 256;
    const size_t coff = (ioff + items.size() * sizeof(ItemDevB) + 255) / 256 * 256;
    const size_t total = coff + 2 * kMaxGroups * sizeof(uint32_t);
    if (total > sl.cap) return ZFPX_ESIZE;
    std::memcpy(sl.h_stage, fd.data(), fbytes);
    std::memcpy(sl.h_stage + ioff, items.data(), items.size() * sizeof(ItemDevB));
    std::memset(sl.h_stage + coff, 0, 2 * kMaxGroups * sizeof(uint32_t));
    if (cudaMemcpyAsync(sl.d_desc, sl.h_stage, total, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
        return ZFPX_ECUDA;
    uint32_t *ctr = reinterpret_cast<uint32_t *>(sl.d_desc + coff);
    const FieldDevB *dfd = reinterpret_cast<const FieldDevB *>(sl.d_desc);
    const ItemDevB *dit = reinterpret_cast<const ItemDevB *>(sl.d_desc + ioff);
    const BatchGeom ge = make_geom(dfd, dit, s->grid.dev(), (int)items.size(), units, groups, s->lb1, s->upc, ctr);
    const BatchGeom gd = make_geom(dfd, dit, s->grid.dev(), (int)items.size(), units, groups, s->lb1, s->upc,
                                   ctr + kMaxGroups);
    int rc = launch_batch(ge, s->warps, s->ctas_per_sm, true, nullptr, s->d_arena, sl.stream);
    if (!rc) rc = launch_batch(gd, s->warps, s->ctas_per_sm, false, s->d_arena, nullptr, sl.stream);
    if (!rc && cudaEventRecord(sl.done, sl.stream) != cudaSuccess) rc = ZFPX_ECUDA;
    if (rc) return rc;
    sl.ids = ids;
    sl.busy = true;
    s->next_slot = (si + 1) % (int)s->slots.size();
    s->batches++;
    if (launched) *launched = (int)ids.size();
    return ZFPX_OK;
}

int zfpx_server_poll(zfpx_server s, int64_t *done, int max, int *ndone)
{
    if (!s || !ndone || (max > 0 && !done)) return ZFPX_EINVAL;
    server_reap(s);
    int n = 0;
    while (n < max && !s->completed.empty()) {
        done[n++] = s->completed.front();
        s->completed.pop_front();
    }
    *ndone = n;
    return ZFPX_OK;
}

int zfpx_server_result(zfpx_server s, int64_t id, const uint8_t **d_stream, size_t *stream_bytes,
                       const float **d_values, size_t *values_bytes)
{
    if (!s) return ZFPX_EINVAL;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end() || it->second.state != 2) return ZFPX_EINVAL;
    const ServerReq &r = it->second;
    if (d_stream) *d_stream = s->d_arena + r.mem_off;
    if (stream_bytes) *stream_bytes = (size_t)r.stream_bytes;
    if (d_values) *d_values = r.f.d_dst;
    if (values_bytes) *values_bytes = (size_t)r.values_bytes;
    return ZFPX_OK;
}

int zfpx_server_copy_result(zfpx_server s, int64_t id, uint8_t *h_stream, size_t stream_cap, float *h_values,
                            size_t values_cap)
{
    if (!s) return ZFPX_EINVAL;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end() || it->second.state != 2) return ZFPX_EINVAL;
    const ServerReq &r = it->second;
    if ((h_stream && stream_cap < (size_t)r.stream_bytes) || (h_values && values_cap < (size_t)r.values_bytes))
        return ZFPX_ESIZE;
    if (h_stream && cudaMemcpy(h_stream, s->d_arena + r.mem_off, r.stream_bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
        return ZFPX_ECUDA;
    if (h_values && cudaMemcpy(h_values, r.f.d_dst, r.values_bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
        return ZFPX_ECUDA;
    return ZFPX_OK;
}

int zfpx_server_release(zfpx_server s, int64_t id)
{
    if (!s) return ZFPX_EINVAL;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end() || it->second.state != 2) return ZFPX_EINVAL;
    s->arena.give(it->second.mem_off, it->second.mem_bytes);
    s->reqs.erase(it);
    return ZFPX_OK;
}

int zfpx_server_stats(zfpx_server s, int64_t out[6])
{
    if (!s || !out) return ZFPX_EINVAL;
    int busy = 0;
    for (auto &sl : s->slots) busy += sl.busy ? 1 : 0;
    out[0] = (int64_t)s->queue.size();
    out[1] = busy;
    out[2] = s->arena.used;
    out[3] = s->arena.total;
    out[4] = s->batches;
    out[5] = (int64_t)s->completed.size();
    return ZFPX_OK;
}

// The request loop in native code: request i is submitted once `arrivals[i]`
// seconds have passed since the call began (all at once when arrivals is
// NULL); between arrivals the loop pumps (a batch on every free stream) and
// polls, releasing every finished request.  t_done[i] receives the time from
// the start at which the loop saw request i finished (-1 if it was refused as
// larger than the arena).  info, if not NULL: [wall seconds from the first
// arrival to the last completion, batches launched, most streams busy at once,
// requests refused].
int zfpx_server_run(zfpx_server s, const zfpx_field *reqs, int n, const double *arrivals, double *t_done,
                    double *info)
{
    if (!s || n < 0 || (n > 0 && (!reqs || !t_done))) return ZFPX_EINVAL;
    using clk = std::chrono::steady_clock;
    const clk::time_point t0 = clk::now();
    auto elapsed = [&]() { return std::chrono::duration<double>(clk::now() - t0).count(); };
    std::unordered_map<int64_t, int> index;
    index.reserve((size_t)n * 2 + 1);
    const int64_t batches0 = s->batches;
    int i = 0, done = 0, refused = 0, busy_max = 0;
    std::vector<int64_t> fin(256);
    double first = arrivals && n ? arrivals[0] : 0.0, last = 0.0;
    for (int k = 0; k < n; k++) {
        t_done[k] = -1.0;
        if (arrivals && arrivals[k] < first) first = arrivals[k];
    }
    while (done < n) {
        const double now = elapsed();
        while (i < n && (!arrivals || arrivals[i] <= now)) {
            int64_t id = 0;
            const int rc = zfpx_server_submit(s, &reqs[i], &id);
            if (rc == ZFPX_ENOMEM_BUDGET) {
                refused++;
                done++;
            } else if (rc) {
                return rc;
            } else {
                index[id] = i;
            }
            i++;
        }
        for (;;) {                                     // a batch on every free stream
            int launched = 0;
            const int rc = zfpx_server_pump(s, &launched);
            if (rc) return rc;
            if (!launched) break;
        }
        int busy = 0;
        for (auto &sl : s->slots) busy += sl.busy ? 1 : 0;
        busy_max = std::max(busy_max, busy);
        int nd = 0;
        const int rc = zfpx_server_poll(s, fin.data(), (int)fin.size(), &nd);
        if (rc) return rc;
        for (int k = 0; k < nd; k++) {
            auto it = index.find(fin[k]);
            if (it != index.end()) {
                t_done[it->second] = elapsed();
                last = t_done[it->second];
                index.erase(it);
                done++;
            }
            zfpx_server_release(s, fin[k]);
        }
    }
    if (info) {
        info[0] = n ? last - first : 0.0;
        info[1] = (double)(s->batches - batches0);
        info[2] = busy_max;
        info[3] = refused;
    }
    return ZFPX_OK;
}

}  // extern "C"
