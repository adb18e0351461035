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
// Work list: every (field, item) is split into chunks of 32 consecutive blocks
// (one per lane); chunks are sorted so that fields of one (dims, rate) class
// are contiguous, and each warp of the persistent grid takes a contiguous
// range of chunks.  The class is uniform across a warp.
#include <algorithm>
#include <climits>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "zfpx_internal.h"
#include "zfpx_block.cuh"

namespace zfpx {
namespace {

using namespace blk;

struct FieldDevB {
    const float *src;
    float *dst;
    int64_t lev_stride;
    int64_t out_off;   // byte offset of the field's stream
    int32_t nlev, dims, rate, vec;
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

struct BatchGeom {
    const ItemDevB *items;
    const FieldDevB *fields;
    GridDev grid;
    int nitems;
    int64_t nunits;
};

__device__ __forceinline__ int upper_index(const int64_t *pre, int n, int64_t b)
{
    int lo = 0, hi = n - 1;   // last i with pre[i] <= b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(pre + mid) <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

struct ItemWalk {
    const ItemDevB *items;
    int n, i;
    int64_t next0;
    __device__ __forceinline__ void start(const ItemDevB *it, int cnt, int64_t u)
    {
        items = it; n = cnt;
        int lo = 0, hi = cnt - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (it[mid].unit0 <= u) lo = mid; else hi = mid - 1;
        }
        i = lo;
        next0 = i + 1 < cnt ? it[i + 1].unit0 : LLONG_MAX;
    }
    __device__ __forceinline__ void advance(int64_t u)
    {
        while (u >= next0) {
            i++;
            next0 = i + 1 < n ? items[i + 1].unit0 : LLONG_MAX;
        }
    }
};

template <int RATE>
struct SmemWriterB {
    uint64_t *sm;
    uint64_t acc;
    int nb, w, lane;
    __device__ __forceinline__ void put(uint64_t bits, int len)
    {
        acc |= bits << nb;
        int t = nb + len;
        if (t >= 64) {
            sm[w * 32 + (lane ^ w)] = acc;
            w++;
            acc = nb ? (bits >> (64 - nb)) : 0ull;
            t -= 64;
        }
        nb = t;
    }
    __device__ __forceinline__ void finish()
    {
        if (nb > 0) { sm[w * 32 + (lane ^ w)] = acc; w++; }
        for (; w < RATE; w++) sm[w * 32 + (lane ^ w)] = 0ull;
    }
};

struct SmemPlanesB {
    uint64_t *sm;
    int lane;
    __device__ __forceinline__ void store(int k, uint64_t X) { sm[k * 32 + lane] = X; }
    __device__ __forceinline__ uint64_t load(int k) const { return sm[k * 32 + lane]; }
    __device__ __forceinline__ uint32_t *words() { return reinterpret_cast<uint32_t *>(sm); }
    __device__ __forceinline__ int word_index(int i) const { return (i >> 1) * 64 + 2 * lane + (i & 1); }
};

struct StreamTileB {
    const uint32_t *sm;
    int lane;
    __device__ __forceinline__ uint32_t get(int i) const { return sm[i * 32 + lane]; }
};

// 64 values of a 3-D block of row-quad q, x block bxi, levels z0.. (clamped)
__device__ __forceinline__ void gather_quad(const FieldDevB &f, const GridDev &g, int q, int bxi, int z0, int nz,
                                            float (&x)[64])
{
    const int x0 = 4 * bxi;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int r = min(4 * q + j, g.nrows - 1);
        const int64_t roff = __ldg(g.row_off + r);
        const int len = __ldg(g.row_len + r);
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const float *row = f.src + (int64_t)(z0 + min(k, nz - 1)) * f.lev_stride + roff;
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

__device__ __forceinline__ void scatter_quad(const FieldDevB &f, const GridDev &g, int q, int bxi, int z0, int nz,
                                             const float (&x)[64])
{
    const int x0 = 4 * bxi;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int r = 4 * q + j;
        if (r >= g.nrows) continue;
        const int64_t roff = __ldg(g.row_off + r);
        const int len = __ldg(g.row_len + r);
        if (x0 >= len) continue;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (k >= nz) continue;
            float *row = f.dst + (int64_t)(z0 + k) * f.lev_stride + roff;
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

template <int RATE>
__device__ __forceinline__ void enc3_chunk(const FieldDevB &f, const GridDev &g, const ItemDevB &it, int64_t b0,
                                           int nact, int lane, uint64_t *wsm, uint64_t *wpl, uint8_t *out)
{
    if (lane < nact) {
        const int64_t b = b0 + lane;
        const int q = upper_index(g.qpre, g.nq + 1, b);
        const int bxi = (int)(b - __ldg(g.qpre + q));
        float x[64];
        gather_quad(f, g, q, bxi, it.z0, it.nz, x);
        SmemWriterB<RATE> wr{wsm, 0ull, 0, 0, lane};
        SmemPlanesB pl{wpl, lane};
        encode_block3<RATE>(x, wr, pl);
    }
    __syncwarp();
    uint64_t *dst = reinterpret_cast<uint64_t *>(out + it.out_off) + b0 * RATE;
    for (int idx = lane; idx < nact * RATE; idx += 32) {
        const int l = idx / RATE, w = idx % RATE;
        dst[idx] = wsm[w * 32 + (l ^ w)];
    }
    __syncwarp();
}

template <int RATE>
__device__ __forceinline__ void enc1_chunk(const FieldDevB &f, const GridDev &g, const ItemDevB &it, int64_t b0,
                                           int nact, int lane, uint8_t *out)
{
    if (lane >= nact) return;
    const int64_t b = b0 + lane;
    const int r = upper_index(g.rpre, g.nrows + 1, b);
    const int x0 = 4 * (int)(b - __ldg(g.rpre + r));
    const int len = __ldg(g.row_len + r);
    const float *row = f.src + (int64_t)it.z0 * f.lev_stride + __ldg(g.row_off + r);
    float x[4];
    if (f.vec && x0 + 4 <= len) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(row + x0));
        x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    } else {
#pragma unroll
        for (int i = 0; i < 4; i++) x[i] = __ldg(row + min(x0 + i, len - 1));
    }
    const uint64_t w = encode_block1<RATE>(x);
    if (RATE == 16) reinterpret_cast<uint64_t *>(out + it.out_off)[b] = w;
    else reinterpret_cast<uint32_t *>(out + it.out_off)[b] = (uint32_t)w;
}

template <int WARPS>
__global__ void __launch_bounds__(32 * WARPS)
batch_encode_kernel(BatchGeom bg, uint8_t *__restrict__ out)
{
    __shared__ uint64_t sout[WARPS][16 * 32];
    __shared__ uint64_t splanes[WARPS][32 * 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t W = (int64_t)gridDim.x * WARPS;
    const int64_t gw = (int64_t)blockIdx.x * WARPS + wid;
    int64_t c = gw * bg.nunits / W;
    const int64_t c1 = (gw + 1) * bg.nunits / W;
    if (c >= c1) return;
    ItemWalk walk;
    walk.start(bg.items, bg.nitems, c);
    for (; c < c1; c++) {
        walk.advance(c);
        const ItemDevB it = bg.items[walk.i];
        const FieldDevB f = bg.fields[it.field];
        const int64_t b0 = (c - it.unit0) * 32;
        const int nact = (int)min((int64_t)32, it.nblocks - b0);
        if (f.dims == 3) {
            if (f.rate == 8) enc3_chunk<8>(f, bg.grid, it, b0, nact, lane, sout[wid], splanes[wid], out);
            else enc3_chunk<16>(f, bg.grid, it, b0, nact, lane, sout[wid], splanes[wid], out);
        } else {
            if (f.rate == 8) enc1_chunk<8>(f, bg.grid, it, b0, nact, lane, out);
            else enc1_chunk<16>(f, bg.grid, it, b0, nact, lane, out);
        }
    }
}

template <int RATE>
__device__ __forceinline__ void dec3_lane(const FieldDevB &f, const GridDev &g, const ItemDevB &it, int64_t b,
                                          int lane, const uint8_t *in, uint32_t *t32, uint64_t *wpl)
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
    for (int r = 0; r < 3; r++) t32[(2 * RATE + r) * 32 + lane] = 0u;
    const int q = upper_index(g.qpre, g.nq + 1, b);
    const int bxi = (int)(b - __ldg(g.qpre + q));
    float x[64];
    const StreamTileB tile{t32, lane};
    SmemPlanesB pl{wpl, lane};
    decode_block3_tile<RATE>(tile, x, pl);
    scatter_quad(f, g, q, bxi, it.z0, it.nz, x);
}

template <int RATE>
__device__ __forceinline__ void dec1_lane(const FieldDevB &f, const GridDev &g, const ItemDevB &it, int64_t b,
                                          const uint8_t *in)
{
    uint64_t w;
    if (RATE == 16) w = __ldg(reinterpret_cast<const uint64_t *>(in + it.out_off) + b);
    else w = __ldg(reinterpret_cast<const uint32_t *>(in + it.out_off) + b);
    float x[4];
    decode_block1<RATE>(w, x);
    const int r = upper_index(g.rpre, g.nrows + 1, b);
    const int x0 = 4 * (int)(b - __ldg(g.rpre + r));
    const int len = __ldg(g.row_len + r);
    float *row = f.dst + (int64_t)it.z0 * f.lev_stride + __ldg(g.row_off + r);
    if (f.vec && x0 + 4 <= len) {
        *reinterpret_cast<float4 *>(row + x0) = make_float4(x[0], x[1], x[2], x[3]);
    } else {
#pragma unroll
        for (int i = 0; i < 4; i++)
            if (x0 + i < len) row[x0 + i] = x[i];
    }
}

template <int WARPS>
__global__ void __launch_bounds__(32 * WARPS)
batch_decode_kernel(BatchGeom bg, const uint8_t *__restrict__ in)
{
    __shared__ uint32_t stile[WARPS][(2 * 16 + 3) * 32];
    __shared__ uint64_t splanes[WARPS][32 * 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t W = (int64_t)gridDim.x * WARPS;
    const int64_t gw = (int64_t)blockIdx.x * WARPS + wid;
    int64_t c = gw * bg.nunits / W;
    const int64_t c1 = (gw + 1) * bg.nunits / W;
    if (c >= c1) return;
    ItemWalk walk;
    walk.start(bg.items, bg.nitems, c);
    for (; c < c1; c++) {
        walk.advance(c);
        const ItemDevB it = bg.items[walk.i];
        const FieldDevB f = bg.fields[it.field];
        const int64_t b0 = (c - it.unit0) * 32;
        const int nact = (int)min((int64_t)32, it.nblocks - b0);
        if (lane >= nact) continue;
        const int64_t b = b0 + lane;
        if (f.dims == 3) {
            if (f.rate == 8) dec3_lane<8>(f, bg.grid, it, b, lane, in, stile[wid], splanes[wid]);
            else dec3_lane<16>(f, bg.grid, it, b, lane, in, stile[wid], splanes[wid]);
        } else {
            if (f.rate == 8) dec1_lane<8>(f, bg.grid, it, b, in);
            else dec1_lane<16>(f, bg.grid, it, b, in);
        }
    }
}

}  // namespace
}  // namespace zfpx

struct zfpx_batch_s {
    int dev = -1;
    int nrows = 0, nq = 0;
    std::vector<zfpx_field> fields;
    std::vector<int64_t> field_off;
    std::vector<int64_t> field_bytes;
    int64_t total = 0;
    int nitems = 0;
    int64_t nunits = 0;
    int warps = 4, ctas_per_sm = 0;     // 0 = as many as fit
    // device allocations
    int64_t *d_row_off = nullptr;
    int32_t *d_row_len = nullptr;
    int64_t *d_qpre = nullptr, *d_rpre = nullptr;
    zfpx::FieldDevB *d_fields = nullptr;
    zfpx::ItemDevB *d_items = nullptr;
};

using namespace zfpx;

namespace {
template <class T>
int upload(T **dptr, const std::vector<T> &h)
{
    if (h.empty()) return ZFPX_OK;
    if (cudaMalloc((void **)dptr, h.size() * sizeof(T)) != cudaSuccess) return ZFPX_ENOMEM;
    if (cudaMemcpy(*dptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) return ZFPX_ECUDA;
    return ZFPX_OK;
}
}  // namespace

extern "C" {

void zfpx_batch_destroy(zfpx_batch b)
{
    if (!b) return;
    cudaFree(b->d_row_off);
    cudaFree(b->d_row_len);
    cudaFree(b->d_qpre);
    cudaFree(b->d_rpre);
    cudaFree(b->d_fields);
    cudaFree(b->d_items);
    delete b;
}

int zfpx_batch_create(zfpx_batch *out, const int64_t *row_len, int nrows, const zfpx_field *fields, int nfields)
{
    if (!out) return ZFPX_EINVAL;
    *out = nullptr;
    if (!row_len || nrows < 1 || !fields || nfields < 1) return ZFPX_EINVAL;
    int64_t npts = 0;
    bool mult4 = true;
    for (int r = 0; r < nrows; r++) {
        if (row_len[r] < 1 || row_len[r] > (1 << 30)) return ZFPX_EINVAL;
        npts += row_len[r];
        mult4 = mult4 && (row_len[r] % 4 == 0);
    }
    for (int f = 0; f < nfields; f++) {
        const zfpx_field &F = fields[f];
        if (F.nlev < 1 || (F.dims != 1 && F.dims != 3) || !valid_codec_rate(F.rate)) return ZFPX_EINVAL;
        if (F.lev_stride < npts && F.nlev > 1) return ZFPX_EINVAL;
    }
    zfpx_batch_s *b = new (std::nothrow) zfpx_batch_s;
    if (!b) return ZFPX_ENOMEM;
    if (cudaGetDevice(&b->dev) != cudaSuccess) { delete b; return ZFPX_ECUDA; }
    b->nrows = nrows;
    b->nq = (nrows + 3) / 4;
    b->fields.assign(fields, fields + nfields);

    std::vector<int64_t> roff(nrows), qpre(b->nq + 1, 0), rpre(nrows + 1, 0);
    std::vector<int32_t> rlen(nrows);
    int64_t o = 0;
    for (int r = 0; r < nrows; r++) { roff[r] = o; o += row_len[r]; rlen[r] = (int32_t)row_len[r]; }
    for (int q = 0; q < b->nq; q++) {
        int64_t mx = 0;
        for (int j = 0; j < 4 && 4 * q + j < nrows; j++) mx = std::max(mx, row_len[4 * q + j]);
        qpre[q + 1] = qpre[q] + (mx + 3) / 4;
    }
    for (int r = 0; r < nrows; r++) rpre[r + 1] = rpre[r] + (row_len[r] + 3) / 4;

    // field layout and items; chunks ordered by (dims, rate) class, then field, then item
    std::vector<FieldDevB> fd(nfields);
    b->field_off.resize(nfields);
    b->field_bytes.resize(nfields);
    int64_t off = 0;
    for (int f = 0; f < nfields; f++) {
        const zfpx_field &F = fields[f];
        const int64_t per_block = F.dims == 3 ? 8 * F.rate : F.rate / 2;
        const int64_t items = F.dims == 3 ? (F.nlev + 3) / 4 : F.nlev;
        const int64_t blocks = F.dims == 3 ? qpre[b->nq] : rpre[nrows];
        b->field_off[f] = off;
        b->field_bytes[f] = items * blocks * per_block;
        off = (off + b->field_bytes[f] + 255) / 256 * 256;
        const bool vec = mult4 && (F.lev_stride % 4 == 0 || F.nlev == 1) && !((uintptr_t)F.d_src & 15u) &&
                         !((uintptr_t)F.d_dst & 15u);
        fd[f] = FieldDevB{F.d_src, F.d_dst, F.lev_stride, b->field_off[f], F.nlev, F.dims, F.rate, vec ? 1 : 0};
    }
    b->total = off;
    std::vector<int> order(nfields);
    for (int f = 0; f < nfields; f++) order[f] = f;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return std::make_tuple(fields[a].dims, fields[a].rate) < std::make_tuple(fields[c].dims, fields[c].rate);
    });
    std::vector<ItemDevB> items;
    int64_t units = 0;
    for (int f : order) {
        const zfpx_field &F = fields[f];
        const int64_t per_block = F.dims == 3 ? 8 * F.rate : F.rate / 2;
        const int64_t blocks = F.dims == 3 ? qpre[b->nq] : rpre[nrows];
        const int step = F.dims == 3 ? 4 : 1;
        int64_t ioff = b->field_off[f];
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
            units += (blocks + 31) / 32;
            ioff += blocks * per_block;
        }
    }
    b->nitems = (int)items.size();
    b->nunits = units;
    int rc = upload(&b->d_row_off, roff);
    if (!rc) rc = upload(&b->d_row_len, rlen);
    if (!rc) rc = upload(&b->d_qpre, qpre);
    if (!rc) rc = upload(&b->d_rpre, rpre);
    if (!rc) rc = upload(&b->d_fields, fd);
    if (!rc) rc = upload(&b->d_items, items);
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
    if (!b || (warps_per_cta != 4 && warps_per_cta != 8) || ctas_per_sm < 0) return ZFPX_EINVAL;
    b->warps = warps_per_cta;
    b->ctas_per_sm = ctas_per_sm;
    return ZFPX_OK;
}

static int batch_launch(zfpx_batch b, bool encode, const uint8_t *in, uint8_t *out, cudaStream_t st)
{
    BatchGeom g;
    g.items = b->d_items;
    g.fields = b->d_fields;
    g.grid = GridDev{b->d_row_off, b->d_row_len, b->d_qpre, b->d_rpre, b->nrows, b->nq};
    g.nitems = b->nitems;
    g.nunits = b->nunits;
    if (g.nunits == 0) return ZFPX_OK;
    const void *fn = nullptr;
    if (encode) fn = b->warps == 8 ? (const void *)batch_encode_kernel<8> : (const void *)batch_encode_kernel<4>;
    else fn = b->warps == 8 ? (const void *)batch_decode_kernel<8> : (const void *)batch_decode_kernel<4>;
    const int fit = occupancy(fn, 32 * b->warps);
    const int per_sm = b->ctas_per_sm > 0 ? std::min(b->ctas_per_sm, fit) : fit;
    const int64_t want = (g.nunits + b->warps - 1) / b->warps;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms() * per_sm));
    if (encode) {
        if (b->warps == 8) batch_encode_kernel<8><<<grid, 256, 0, st>>>(g, out);
        else batch_encode_kernel<4><<<grid, 128, 0, st>>>(g, out);
    } else {
        if (b->warps == 8) batch_decode_kernel<8><<<grid, 256, 0, st>>>(g, in);
        else batch_decode_kernel<4><<<grid, 128, 0, st>>>(g, in);
    }
    count_launch();
    return check_launch();
}

int zfpx_batch_encode(zfpx_batch b, uint8_t *d_out, size_t cap, void *stream)
{
    if (!b || !d_out || ((uintptr_t)d_out & 15u)) return ZFPX_EINVAL;
    if ((int64_t)cap < b->total) return ZFPX_ESIZE;
    for (const zfpx_field &F : b->fields)
        if (!F.d_src || ((uintptr_t)F.d_src & 3u)) return ZFPX_EINVAL;
    return batch_launch(b, true, nullptr, d_out, (cudaStream_t)stream);
}

int zfpx_batch_decode(zfpx_batch b, const uint8_t *d_in, size_t len, void *stream)
{
    if (!b || !d_in || ((uintptr_t)d_in & 15u)) return ZFPX_EINVAL;
    if ((int64_t)len < b->total) return ZFPX_ESIZE;
    for (const zfpx_field &F : b->fields)
        if (!F.d_dst || ((uintptr_t)F.d_dst & 3u)) return ZFPX_EINVAL;
    return batch_launch(b, false, d_in, nullptr, (cudaStream_t)stream);
}

}  // extern "C"
