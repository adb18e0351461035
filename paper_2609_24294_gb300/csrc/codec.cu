// Fused pack + ZFP fixed-rate encode, and fused decode + unpack, for sm_103a.
//
// The codec is ZFP's fixed-rate mode as the paper uses it (Sec. II-C: 4^d
// blocks coded independently by a lifting transform and precision
// reduction; Sec. IV-B: rate 8 and 16, fixed message size), in the readings
// stated in include/zfpx.h:
//   e_max = frexp exponent of max|x|; zero block if max|x| is 0, subnormal or
//   non-finite; q = trunc(x 2^(30-e_max)); five-step integer lifting along
//   x, y, z; coefficients in total-sequency order; negabinary; group-tested
//   bit planes from 31 down, cut at exactly 4^d r bits.
//
// Mapping to the GPU: one lane owns one block.  A warp takes 32 consecutive
// blocks of one message, so its compressed output (or input) is one
// contiguous run of 32 * 8r bytes, staged through shared memory in a
// [word][lane] layout (XOR-swizzled) and moved with coalesced 8-byte
// accesses.  The 64 coefficients of a block live in registers; their 32 bit
// planes are formed with two in-register 32x32 bit-matrix transposes
// (byte permutes for the 16- and 8-bit stages, masked shifts below), after
// which each plane is one 64-bit word and group testing is a find-first-set
// per newly significant coefficient.  Each warp processes a contiguous range
// of 32-block chunks, so the message lookup is a forward scan.
#include <atomic>
#include <climits>
#include <cuda_runtime.h>

#include "zfpx_internal.h"
#include "zfpx_block.cuh"
#include "zfpx_smem.cuh"
#include "zfpx_enc3.cuh"

namespace zfpx {
namespace {

using namespace blk;

constexpr int kWarps = 4;
constexpr int kThreads = 32 * kWarps;
// Launch shapes of the 3-D kernels, chosen by measurement on GB300: encoder
// CTAs of 2 warps (rate 8) and 3 warps (rate 16), whose shared memory packs
// the SMs best; decoder CTAs of 4 warps, except the rate-16 decoder, whose
// 3-warp CTAs fit six to an SM (two zero rows after its stream tile make the
// shared memory fit); the rate-8 decoder is compiled for five resident CTAs,
// which its shared memory allows and capping its registers to match pays for.
template <int RATE>
constexpr int kEnc3Warps = RATE == 16 ? 3 : 2;
template <int RATE>
constexpr int kEnc3MinBlocks = RATE == 16 ? 5 : 8;     // what the shared memory allows
template <int RATE>
constexpr int kDec3Warps = RATE == 16 ? 3 : 4;
template <int RATE>
constexpr int kDec3MinBlocks = RATE == 8 ? 5 : 6;

// ----------------------------------------------------------------- message walk
__device__ __forceinline__ int find_msg(const MsgDev *msgs, int nmsg, int64_t u)
{
    int lo = 0, hi = nmsg - 1;               // last message with unit0 <= u
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (msgs[mid].unit0 <= u) lo = mid; else hi = mid - 1;
    }
    return lo;
}

struct MsgWalk {
    const MsgDev *msgs;
    int nmsg, mi;
    int64_t next0;
    __device__ __forceinline__ void start(const MsgDev *m, int n, int64_t u)
    {
        msgs = m; nmsg = n;
        mi = find_msg(m, n, u);
        next0 = mi + 1 < n ? m[mi + 1].unit0 : LLONG_MAX;
    }
    __device__ __forceinline__ void advance(int64_t u)
    {
        while (u >= next0) {
            mi++;
            next0 = mi + 1 < nmsg ? msgs[mi + 1].unit0 : LLONG_MAX;
        }
    }
};

// Work split of the 3-D kernels: warp w of the grid codes the upw consecutive
// 32-block units starting at w * upw (the grid has ceil(units / (upw * warps))
// CTAs), and the hardware's CTA scheduler balances the CTAs over the SMs.  No
// counters in device memory: launches on any streams may overlap, and a CUDA
// graph replays a launch as it was recorded.
struct UnitRange {
    int64_t c, c1;
    __device__ __forceinline__ UnitRange(const LaunchGeom &g, int warps, int wid)
    {
        c = ((int64_t)blockIdx.x * warps + wid) * g.upw;
        c1 = min(c + (int64_t)g.upw, g.nunits);
    }
};

// ================================================================= 3-D kernels
// VEC: every block's rows start on 16 bytes (the view's row and level strides
// and every message's x origin are multiples of 4 values, the base aligned),
// so full rows move as 16-byte loads and stores.  Otherwise a separate
// instantiation reads and writes the rows of x-complete blocks as four scalar
// accesses each, unrolled, keeping the vector kernel's code as it is.
template <int RATE, bool VEC>
__global__ void __launch_bounds__(32 * kEnc3Warps<RATE>, kEnc3MinBlocks<RATE>)
encode3_kernel(const float *__restrict__ src, uint8_t *__restrict__ out, LaunchGeom g, int layout)
{
    __shared__ enc3::Shared<RATE> sh[kEnc3Warps<RATE>];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const enc3::View v = sh[wid].view();
    const UnitRange ur(g, kEnc3Warps<RATE>, wid);
    if (ur.c >= ur.c1) return;
    enc3::clear(v, lane, enc3::kWords<RATE>);
    __syncwarp();
    MsgWalk walk;
    walk.start(g.msgs, g.nmsg, ur.c);
    for (int64_t c = ur.c; c < ur.c1; c++) {
        walk.advance(c);
        const MsgDev &m = g.msgs[walk.mi];
        const int64_t unit0 = m.unit0, nblocks = m.nblocks, src_off = m.src_off;
        const int64_t boff = layout ? m.off[1] : m.off[0];
        const int nx = m.nx, ny = m.ny, nz = m.nz, bxn = m.bx, byn = m.by;
        const int64_t b0 = (c - unit0) * 32;
        const int nact = (int)min((int64_t)32, nblocks - b0);
        const bool valid = lane < nact;
        float x[64];
        {
            // lanes past the unit's last block load that block and code nothing
            const int b = (int)b0 + (valid ? lane : nact - 1);
            const int t = (int)divu((uint32_t)b, m.bxm, m.bxl), bxi = b - t * bxn;
            const int bzi = (int)divu((uint32_t)t, m.bym, m.byl), byi = t - bzi * byn;
            const int x0 = 4 * bxi, y0 = 4 * byi, z0 = 4 * bzi;
            const float *base = src + src_off;
            if (VEC && x0 + 4 <= nx) {
                // the common case: sixteen 16-byte row loads (rows past the
                // end of the box repeat its last row)
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const int64_t zo = (int64_t)min(z0 + k, nz - 1) * g.ss[2];
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        const float4 f = __ldg(reinterpret_cast<const float4 *>(
                            base + zo + (int64_t)min(y0 + j, ny - 1) * g.ss[1] + x0));
                        x[16 * k + 4 * j] = f.x; x[16 * k + 4 * j + 1] = f.y;
                        x[16 * k + 4 * j + 2] = f.z; x[16 * k + 4 * j + 3] = f.w;
                    }
                }
            } else if (!VEC && x0 + 4 <= nx) {
                // rows not on 16 bytes: four scalar loads per row
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const int64_t zo = (int64_t)min(z0 + k, nz - 1) * g.ss[2];
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        const float *row = base + zo + (int64_t)min(y0 + j, ny - 1) * g.ss[1] + (int64_t)x0 * g.ss[0];
#pragma unroll
                        for (int i = 0; i < 4; i++) x[16 * k + 4 * j + i] = __ldg(row + (int64_t)i * g.ss[0]);
                    }
                }
            } else {
                // partial in x: element loads through a local
                // array, kept rolled so the hot path's code stays compact
                float t[64];
#pragma unroll 1
                for (int r = 0; r < 64; r++) {
                    const int i = r & 3, j = (r >> 2) & 3, k = r >> 4;
                    t[r] = __ldg(base + (int64_t)min(z0 + k, nz - 1) * g.ss[2] +
                                 (int64_t)min(y0 + j, ny - 1) * g.ss[1] + (int64_t)min(x0 + i, nx - 1) * g.ss[0]);
                }
#pragma unroll
                for (int r = 0; r < 64; r++) x[r] = t[r];
            }
        }
        enc3::encode<RATE>(x, valid, v, lane);
        __syncwarp();
        enc3::store_stream<RATE>(v, lane, valid, out + boff + (b0 + lane) * RATE * 8);
        __syncwarp();
    }
}

template <int RATE, bool VEC>
__global__ void __launch_bounds__(32 * kDec3Warps<RATE>, kDec3MinBlocks<RATE>)
decode3_kernel(const uint8_t *__restrict__ in, float *__restrict__ dstf, LaunchGeom g, int layout)
{
    __shared__ uint32_t stile[kDec3Warps<RATE>][(2 * RATE + kTileZeroRows<RATE>) * 32];
    __shared__ uint64_t splanes[kDec3Warps<RATE>][32 * 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t *t32 = stile[wid];
    SmemPlanes pl{splanes[wid], lane};
    const StreamTile tile{t32, lane};
#pragma unroll
    for (int r = 0; r < kTileZeroRows<RATE>; r++) t32[(2 * RATE + r) * 32 + lane] = 0u;
    const UnitRange ur(g, kDec3Warps<RATE>, wid);
    if (ur.c >= ur.c1) return;
    MsgWalk walk;
    walk.start(g.msgs, g.nmsg, ur.c);
    for (int64_t c = ur.c; c < ur.c1; c++) {
        walk.advance(c);
        const MsgDev &m = g.msgs[walk.mi];
        const int64_t unit0 = m.unit0, nblocks = m.nblocks, dst_off = m.dst_off;
        const int64_t boff = layout ? m.off[1] : m.off[0];
        const int nx = m.nx, ny = m.ny, nz = m.nz, bxn = m.bx, byn = m.by;
        const int64_t b0 = (c - unit0) * 32;
        const int nact = (int)min((int64_t)32, nblocks - b0);
        if (lane < nact) {
            const int b = (int)b0 + lane;
            // this lane's block: RATE / 2 16-byte loads into its own tile column
            const uint4 *src4 = reinterpret_cast<const uint4 *>(in + boff) + (int64_t)b * (RATE / 2);
#pragma unroll
            for (int i = 0; i < RATE / 2; i++) {
                const uint4 v = __ldg(src4 + i);
                t32[(4 * i) * 32 + lane] = v.x;
                t32[(4 * i + 1) * 32 + lane] = v.y;
                t32[(4 * i + 2) * 32 + lane] = v.z;
                t32[(4 * i + 3) * 32 + lane] = v.w;
            }
            const int t = (int)divu((uint32_t)b, m.bxm, m.bxl), bxi = b - t * bxn;
            const int bzi = (int)divu((uint32_t)t, m.bym, m.byl), byi = t - bzi * byn;
            const int x0 = 4 * bxi, y0 = 4 * byi, z0 = 4 * bzi;
            float v[64];
            decode_block3_tile<RATE>(tile, v, pl);
            float *base = dstf + dst_off;
            if (VEC && x0 + 4 <= nx) {
#pragma unroll
                for (int k = 0; k < 4; k++) {
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        float *row = base + (int64_t)(z0 + k) * g.ds[2] + (int64_t)(y0 + j) * g.ds[1] + x0;
                        if (z0 + k < nz && y0 + j < ny)
                            *reinterpret_cast<float4 *>(row) = make_float4(v[16 * k + 4 * j], v[16 * k + 4 * j + 1],
                                                                           v[16 * k + 4 * j + 2], v[16 * k + 4 * j + 3]);
                    }
                }
            } else if (!VEC && x0 + 4 <= nx) {
                // rows not on 16 bytes: four scalar stores per row
#pragma unroll
                for (int k = 0; k < 4; k++) {
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        float *row = base + (int64_t)(z0 + k) * g.ds[2] + (int64_t)(y0 + j) * g.ds[1] + (int64_t)x0 * g.ds[0];
                        if (z0 + k < nz && y0 + j < ny) {
#pragma unroll
                            for (int i = 0; i < 4; i++) row[(int64_t)i * g.ds[0]] = v[16 * k + 4 * j + i];
                        }
                    }
                }
            } else {
                float t[64];
#pragma unroll
                for (int r = 0; r < 64; r++) t[r] = v[r];
#pragma unroll 1
                for (int r = 0; r < 64; r++) {
                    const int i = r & 3, j = (r >> 2) & 3, k = r >> 4;
                    if (x0 + i < nx && y0 + j < ny && z0 + k < nz)
                        base[(int64_t)(z0 + k) * g.ds[2] + (int64_t)(y0 + j) * g.ds[1] + (int64_t)(x0 + i) * g.ds[0]] = t[r];
                }
            }
        }
        __syncwarp();
    }
}

// ================================================================= 1-D kernels
// Blocks of 4 values along x; a block is 4r bits (32 or 64), kept in one
// register and moved with one coalesced 4- or 8-byte access per lane.
template <int RATE>
__global__ void __launch_bounds__(kThreads)
encode1_kernel(const float *__restrict__ src, uint8_t *__restrict__ out, LaunchGeom g, int layout, int vec)
{
    __shared__ Plane4Enc tab;
    plane4_fill(tab, threadIdx.x, blockDim.x);
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t W = (int64_t)gridDim.x * kWarps;
    const int64_t gw = (int64_t)blockIdx.x * kWarps + wid;
    int64_t c = gw * g.nunits / W;
    const int64_t c1 = (gw + 1) * g.nunits / W;
    if (c >= c1) return;
    MsgWalk walk;
    walk.start(g.msgs, g.nmsg, c);
    for (; c < c1; c++) {
        walk.advance(c);
        const MsgDev &m = g.msgs[walk.mi];
        const int64_t b0 = (c - m.unit0) * 32;
        const int nact = (int)min((int64_t)32, m.nblocks - b0);
        if (lane >= nact) continue;
        const int nx = m.nx, bxn = m.bx, byn = m.by;
        const int64_t boff = layout ? m.off[1] : m.off[0];
        const int b = (int)b0 + lane;
        const int t = (int)divu((uint32_t)b, m.bxm, m.bxl), bxi = b - t * bxn;
        const int z = (int)divu((uint32_t)t, m.bym, m.byl), y = t - z * byn;
        const int x0 = 4 * bxi;
        const float *row = src + m.src_off + (int64_t)z * g.ss[2] + (int64_t)y * g.ss[1];
        float r[4];
        if (vec && x0 + 4 <= nx) {
            const float4 f = __ldg(reinterpret_cast<const float4 *>(row + x0));
            r[0] = f.x; r[1] = f.y; r[2] = f.z; r[3] = f.w;
        } else {
#pragma unroll
            for (int i = 0; i < 4; i++) r[i] = __ldg(row + (int64_t)min(x0 + i, nx - 1) * g.ss[0]);
        }
        const uint64_t w = encode_block1<RATE>(r, tab);
        if (RATE == 16) reinterpret_cast<uint64_t *>(out + boff)[b] = w;
        else reinterpret_cast<uint32_t *>(out + boff)[b] = (uint32_t)w;
    }
}

template <int RATE>
__global__ void __launch_bounds__(kThreads)
decode1_kernel(const uint8_t *__restrict__ in, float *__restrict__ dstf, LaunchGeom g, int layout, int vec)
{
    __shared__ Plane4Dec tab;
    plane4_fill(tab, threadIdx.x, blockDim.x);
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t W = (int64_t)gridDim.x * kWarps;
    const int64_t gw = (int64_t)blockIdx.x * kWarps + wid;
    int64_t c = gw * g.nunits / W;
    const int64_t c1 = (gw + 1) * g.nunits / W;
    if (c >= c1) return;
    MsgWalk walk;
    walk.start(g.msgs, g.nmsg, c);
    for (; c < c1; c++) {
        walk.advance(c);
        const MsgDev &m = g.msgs[walk.mi];
        const int64_t b0 = (c - m.unit0) * 32;
        const int nact = (int)min((int64_t)32, m.nblocks - b0);
        if (lane >= nact) continue;
        const int nx = m.nx, bxn = m.bx, byn = m.by;
        const int64_t boff = layout ? m.off[1] : m.off[0];
        const int b = (int)b0 + lane;
        uint64_t w;
        if (RATE == 16) w = __ldg(reinterpret_cast<const uint64_t *>(in + boff) + b);
        else w = __ldg(reinterpret_cast<const uint32_t *>(in + boff) + b);
        float v[4];
        decode_block1<RATE>(w, v, tab);
        const int t = (int)divu((uint32_t)b, m.bxm, m.bxl), bxi = b - t * bxn;
        const int z = (int)divu((uint32_t)t, m.bym, m.byl), y = t - z * byn;
        const int x0 = 4 * bxi;
        float *row = dstf + m.dst_off + (int64_t)z * g.ds[2] + (int64_t)y * g.ds[1];
        if (vec && x0 + 4 <= nx) {
            *reinterpret_cast<float4 *>(row + x0) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
#pragma unroll
            for (int i = 0; i < 4; i++)
                if (x0 + i < nx) row[(int64_t)(x0 + i) * g.ds[0]] = v[i];
        }
    }
}

// ================================================================= 2-D kernels
// Blocks of 4 x 4 values over axes 0 and 1 of one level; one lane per block,
// a warp takes 32 consecutive blocks of one message (units split statically
// over the warps).  A block's stream is RATE / 4 64-bit words, staged in a
// swizzled [word][lane] shared tile and moved with coalesced 8-byte accesses.
template <int RATE>
__global__ void __launch_bounds__(kThreads)
encode2_kernel(const float *__restrict__ src, uint8_t *__restrict__ out, LaunchGeom g, int layout, int vec)
{
    constexpr int NW = RATE / 4;
    __shared__ uint64_t smem[kWarps][(NW + 2) * 32];
    __shared__ uint32_t splanes[kWarps][32 * 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t *wsm = smem[wid];
    SmemPlanes16 pl{splanes[wid], lane};
    const int64_t W = (int64_t)gridDim.x * kWarps;
    const int64_t gw = (int64_t)blockIdx.x * kWarps + wid;
    int64_t c = gw * g.nunits / W;
    const int64_t c1 = (gw + 1) * g.nunits / W;
    if (c >= c1) return;
    MsgWalk walk;
    walk.start(g.msgs, g.nmsg, c);
    for (; c < c1; c++) {
        walk.advance(c);
        const MsgDev &m = g.msgs[walk.mi];
        const int64_t b0 = (c - m.unit0) * 32;
        const int nact = (int)min((int64_t)32, m.nblocks - b0);
        const int64_t boff = layout ? m.off[1] : m.off[0];
        if (lane < nact) {
            const int nx = m.nx, ny = m.ny, bxn = m.bx, byn = m.by;
            const int b = (int)b0 + lane;
            const int t = (int)divu((uint32_t)b, m.bxm, m.bxl), bxi = b - t * bxn;
            const int z = (int)divu((uint32_t)t, m.bym, m.byl), byi = t - z * byn;
            const int x0 = 4 * bxi, y0 = 4 * byi;
            const float *base = src + m.src_off + (int64_t)z * g.ss[2];
            float x[16];
            if (vec && x0 + 4 <= nx) {
                // four 16-byte row loads (rows past the box repeat its last row)
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const float4 f = __ldg(reinterpret_cast<const float4 *>(
                        base + (int64_t)min(y0 + j, ny - 1) * g.ss[1] + x0));
                    x[4 * j] = f.x; x[4 * j + 1] = f.y; x[4 * j + 2] = f.z; x[4 * j + 3] = f.w;
                }
            } else {
#pragma unroll
                for (int r = 0; r < 16; r++) {
                    const int i = r & 3, j = r >> 2;
                    x[r] = __ldg(base + (int64_t)min(y0 + j, ny - 1) * g.ss[1] + (int64_t)min(x0 + i, nx - 1) * g.ss[0]);
                }
            }
            SmemWriter<NW> wr{wsm, 0ull, 0, 0, lane};
            encode_block2<RATE>(x, wr, pl);
        }
        __syncwarp();
        uint64_t *dst = reinterpret_cast<uint64_t *>(out + boff) + b0 * NW;
        for (int idx = lane; idx < nact * NW; idx += 32) {
            const int l = idx / NW, w = idx % NW;
            dst[idx] = wsm[w * 32 + (l ^ w)];
        }
        __syncwarp();
    }
}

template <int RATE>
__global__ void __launch_bounds__(kThreads)
decode2_kernel(const uint8_t *__restrict__ in, float *__restrict__ dstf, LaunchGeom g, int layout, int vec)
{
    constexpr int NW = RATE / 4;              // 64-bit words per block
    constexpr int ZR = 3;                     // zero rows after the stream
    __shared__ uint32_t stile[kWarps][(2 * NW + ZR) * 32];
    __shared__ uint32_t splanes[kWarps][32 * 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t *t32 = stile[wid];
    SmemPlanes16 pl{splanes[wid], lane};
    const StreamTile tile{t32, lane};
#pragma unroll
    for (int r = 0; r < ZR; r++) t32[(2 * NW + r) * 32 + lane] = 0u;
    const int64_t W = (int64_t)gridDim.x * kWarps;
    const int64_t gw = (int64_t)blockIdx.x * kWarps + wid;
    int64_t c = gw * g.nunits / W;
    const int64_t c1 = (gw + 1) * g.nunits / W;
    if (c >= c1) return;
    MsgWalk walk;
    walk.start(g.msgs, g.nmsg, c);
    for (; c < c1; c++) {
        walk.advance(c);
        const MsgDev &m = g.msgs[walk.mi];
        const int64_t b0 = (c - m.unit0) * 32;
        const int nact = (int)min((int64_t)32, m.nblocks - b0);
        if (lane >= nact) continue;
        const int nx = m.nx, ny = m.ny, bxn = m.bx, byn = m.by;
        const int64_t boff = layout ? m.off[1] : m.off[0];
        const int b = (int)b0 + lane;
        // this lane's block: NW / 2 16-byte loads into its own tile column
        const uint4 *src4 = reinterpret_cast<const uint4 *>(in + boff) + (int64_t)b * (NW / 2);
#pragma unroll
        for (int i = 0; i < NW / 2; i++) {
            const uint4 v = __ldg(src4 + i);
            t32[(4 * i) * 32 + lane] = v.x;
            t32[(4 * i + 1) * 32 + lane] = v.y;
            t32[(4 * i + 2) * 32 + lane] = v.z;
            t32[(4 * i + 3) * 32 + lane] = v.w;
        }
        float v[16];
        decode_block2_tile<RATE>(tile, v, pl);
        const int t = (int)divu((uint32_t)b, m.bxm, m.bxl), bxi = b - t * bxn;
        const int z = (int)divu((uint32_t)t, m.bym, m.byl), byi = t - z * byn;
        const int x0 = 4 * bxi, y0 = 4 * byi;
        float *base = dstf + m.dst_off + (int64_t)z * g.ds[2];
        if (vec && x0 + 4 <= nx) {
#pragma unroll
            for (int j = 0; j < 4; j++)
                if (y0 + j < ny)
                    *reinterpret_cast<float4 *>(base + (int64_t)(y0 + j) * g.ds[1] + x0) =
                        make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        } else {
#pragma unroll
            for (int r = 0; r < 16; r++) {
                const int i = r & 3, j = r >> 2;
                if (x0 + i < nx && y0 + j < ny)
                    base[(int64_t)(y0 + j) * g.ds[1] + (int64_t)(x0 + i) * g.ds[0]] = v[r];
            }
        }
    }
}

// ================================================================= launch
template <class K>
int grid_for(K kernel, int64_t nunits, int warps = kWarps)
{
    const int occ = occupancy((const void *)kernel, 32 * warps);
    const int64_t want = (nunits + warps - 1) / warps;
    const int64_t cap = (int64_t)num_sms() * occ;
    return (int)std::max<int64_t>(1, std::min(want, cap));
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Consecutive 32-block units per warp of the 3-D kernels, [encode][rate 16?];
// 0 = default.  The default was picked by timing on GB300 (the autotuner can
// override it); results never depend on it.
std::atomic<int> g_upw[2][2] = {{{0}, {0}}, {{0}, {0}}};
constexpr int kDefaultUpw = 2;

// One launch of a 3-D codec kernel (either alignment instantiation): one
// warp per upw consecutive units.
template <class In, class Out>
void launch3(void (*kernel)(In, Out, LaunchGeom, int), int warps, int encode, int rate, LaunchGeom g,
             cudaStream_t st, In in, Out out, int layout)
{
    g.upw = units_per_warp(encode, rate);
    const int64_t per_cta = (int64_t)g.upw * warps;
    const int64_t grid = (g.nunits + per_cta - 1) / per_cta;
    kernel<<<(unsigned)grid, 32 * warps, 0, st>>>(in, out, g, layout);
}

// vec: rows start on 16 bytes wherever a block starts (x0 multiple of 4).
bool vec_ok(const void *ptr, const int64_t s[3], const zfpx_plan_s *p, int which /*0 src,1 dst*/)
{
    if (!aligned16(ptr) || s[0] != 1 || (s[1] & 3) || (s[2] & 3)) return false;
    (void)which;
    for (const HostMsg &m : p->msgs)
        if (m.x0 & 3) return false;
    return true;
}

}  // namespace

bool codec_vec_ok(const void *ptr, const int64_t s[3], const zfpx_plan_s *p) { return vec_ok(ptr, s, p, 0); }

int launch_encode(int dims, int rate, const float *src, uint8_t *out, const LaunchGeom &g, int layout, int vec,
                  cudaStream_t st)
{
    if (g.nunits == 0) return ZFPX_OK;
    if (dims == 3) {
        if (rate == 8)
            launch3(vec ? encode3_kernel<8, true> : encode3_kernel<8, false>, kEnc3Warps<8>, 1, 8, g, st, src, out,
                    layout);
        else
            launch3(vec ? encode3_kernel<16, true> : encode3_kernel<16, false>, kEnc3Warps<16>, 1, 16, g, st, src, out,
                    layout);
    } else if (dims == 2) {
        if (rate == 8) encode2_kernel<8><<<grid_for(encode2_kernel<8>, g.nunits), kThreads, 0, st>>>(src, out, g, layout, vec);
        else encode2_kernel<16><<<grid_for(encode2_kernel<16>, g.nunits), kThreads, 0, st>>>(src, out, g, layout, vec);
    } else {
        if (rate == 8) encode1_kernel<8><<<grid_for(encode1_kernel<8>, g.nunits), kThreads, 0, st>>>(src, out, g, layout, vec);
        else encode1_kernel<16><<<grid_for(encode1_kernel<16>, g.nunits), kThreads, 0, st>>>(src, out, g, layout, vec);
    }
    count_launch();
    return check_launch();
}

int launch_decode(int dims, int rate, const uint8_t *in, float *dst, const LaunchGeom &g, int layout, int vec,
                  cudaStream_t st)
{
    if (g.nunits == 0) return ZFPX_OK;
    if (dims == 3) {
        if (rate == 8)
            launch3(vec ? decode3_kernel<8, true> : decode3_kernel<8, false>, kDec3Warps<8>, 0, 8, g, st, in, dst,
                    layout);
        else
            launch3(vec ? decode3_kernel<16, true> : decode3_kernel<16, false>, kDec3Warps<16>, 0, 16, g, st, in, dst,
                    layout);
    } else if (dims == 2) {
        if (rate == 8) decode2_kernel<8><<<grid_for(decode2_kernel<8>, g.nunits), kThreads, 0, st>>>(in, dst, g, layout, vec);
        else decode2_kernel<16><<<grid_for(decode2_kernel<16>, g.nunits), kThreads, 0, st>>>(in, dst, g, layout, vec);
    } else {
        if (rate == 8) decode1_kernel<8><<<grid_for(decode1_kernel<8>, g.nunits), kThreads, 0, st>>>(in, dst, g, layout, vec);
        else decode1_kernel<16><<<grid_for(decode1_kernel<16>, g.nunits), kThreads, 0, st>>>(in, dst, g, layout, vec);
    }
    count_launch();
    return check_launch();
}

int units_per_warp(int encode, int rate)
{
    const int v = g_upw[encode ? 1 : 0][rate == 16 ? 1 : 0].load(std::memory_order_relaxed);
    return v > 0 ? v : kDefaultUpw;
}
}  // namespace zfpx

using namespace zfpx;

extern "C" {

int zfpx_set_units_per_warp(int encode, int rate, int upw)
{
    if (!valid_codec_rate(rate) || upw < 0 || upw > 4096) return ZFPX_EINVAL;
    g_upw[encode ? 1 : 0][rate == 16 ? 1 : 0].store(upw, std::memory_order_relaxed);
    return ZFPX_OK;
}

int zfpx_get_units_per_warp(int encode, int rate)
{
    if (!valid_codec_rate(rate)) return ZFPX_EINVAL;
    return units_per_warp(encode, rate);
}

int zfpx_pack_compress(zfpx_plan p, int rate, const float *d_src, uint8_t *d_out, size_t cap, int layout,
                       void *stream)
{
    if (!p || !d_src || !d_out || !valid_codec_rate(rate)) return ZFPX_EINVAL;
    if (layout != ZFPX_LAYOUT_SEND && layout != ZFPX_LAYOUT_RECV) return ZFPX_EINVAL;
    if ((uintptr_t)d_out & 15u) return ZFPX_EINVAL;
    if ((int64_t)cap < buffer_bytes(p, rate)) return ZFPX_ESIZE;
    DevTable *t = nullptr;
    int rc = get_table(p, rate, UNIT_BLOCKS32, &t);
    if (rc) return rc;
    LaunchGeom g{};
    g.msgs = t->d_msgs; g.nmsg = (int)p->msgs.size(); g.nunits = t->nunits;
    for (int a = 0; a < 3; a++) { g.ss[a] = p->ss[a]; g.ds[a] = p->ds[a]; }
    const int vec = vec_ok(d_src, p->ss, p, 0) ? 1 : 0;
    return launch_encode(p->dims, rate, d_src, d_out, g, layout, vec, (cudaStream_t)stream);
}

int zfpx_decompress_unpack(zfpx_plan p, int rate, const uint8_t *d_in, size_t len, float *d_dst, int layout,
                           void *stream)
{
    if (!p || !d_in || !d_dst || !valid_codec_rate(rate)) return ZFPX_EINVAL;
    if (layout != ZFPX_LAYOUT_SEND && layout != ZFPX_LAYOUT_RECV) return ZFPX_EINVAL;
    if ((uintptr_t)d_in & 15u) return ZFPX_EINVAL;
    if ((int64_t)len < buffer_bytes(p, rate)) return ZFPX_ESIZE;
    DevTable *t = nullptr;
    int rc = get_table(p, rate, UNIT_BLOCKS32, &t);
    if (rc) return rc;
    LaunchGeom g{};
    g.msgs = t->d_msgs; g.nmsg = (int)p->msgs.size(); g.nunits = t->nunits;
    for (int a = 0; a < 3; a++) { g.ss[a] = p->ss[a]; g.ds[a] = p->ds[a]; }
    const int vec = vec_ok(d_dst, p->ds, p, 1) ? 1 : 0;
    return launch_decode(p->dims, rate, d_in, d_dst, g, layout, vec, (cudaStream_t)stream);
}

size_t zfpx_stream_bytes(int dims, int rate, const int64_t n[3])
{
    if (!n || dims < 1 || dims > 3 || !valid_codec_rate(rate)) return 0;
    for (int a = 0; a < 3; a++) if (n[a] < 1) return 0;
    const int64_t bx = (n[0] + 3) / 4;
    if (dims == 3) return (size_t)(bx * ((n[1] + 3) / 4) * ((n[2] + 3) / 4) * 8 * rate);
    if (dims == 2) return (size_t)(bx * ((n[1] + 3) / 4) * n[2] * 2 * rate);
    return (size_t)(bx * n[1] * n[2] * rate / 2);
}

}  // extern "C"

// The raw-array entry points run the same kernels on a one-message table
// that lives in a small per-device cache of plans keyed by shape.
#include <map>
#include <tuple>
namespace zfpx {
namespace {
std::mutex g_raw_mu;
std::map<std::tuple<int, int, int64_t, int64_t, int64_t, int64_t, int64_t, int64_t>, zfpx_plan> g_raw_plans;

int raw_plan(int dims, const int64_t n[3], const int64_t s[3], zfpx_plan *out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ZFPX_ECUDA;
    auto key = std::make_tuple(dev, dims, n[0], n[1], n[2], s[0], s[1], s[2]);
    std::lock_guard<std::mutex> g(g_raw_mu);
    auto it = g_raw_plans.find(key);
    if (it != g_raw_plans.end()) { *out = it->second; return ZFPX_OK; }
    if (g_raw_plans.size() > 256) {   // bounded cache
        for (auto &kv : g_raw_plans) zfpx_plan_destroy(kv.second);
        g_raw_plans.clear();
    }
    zfpx_view3 v;
    for (int a = 0; a < 3; a++) { v.n[a] = n[a]; v.stride[a] = s[a]; }
    int rc = zfpx_plan_create(out, &v, &v, 1, 1, 0, dims, ZFPX_SPLIT_BALANCED);
    if (rc) return rc;
    g_raw_plans[key] = *out;
    return ZFPX_OK;
}
}  // namespace
}  // namespace zfpx

extern "C" {

int zfpx_encode(int dims, int rate, const float *d_in, const int64_t n[3], const int64_t stride[3],
                uint8_t *d_out, size_t cap, void *stream)
{
    if (!d_in || !d_out || !n || !stride || dims < 1 || dims > 3 || !valid_codec_rate(rate)) return ZFPX_EINVAL;
    for (int a = 0; a < 3; a++) if (n[a] < 1 || stride[a] < 0) return ZFPX_EINVAL;
    if (cap < zfpx_stream_bytes(dims, rate, n)) return ZFPX_ESIZE;
    zfpx_plan p = nullptr;
    int rc = raw_plan(dims, n, stride, &p);
    if (rc) return rc;
    return zfpx_pack_compress(p, rate, d_in, d_out, cap + 256, ZFPX_LAYOUT_SEND, stream);
}

int zfpx_decode(int dims, int rate, const uint8_t *d_in, size_t len, const int64_t n[3], const int64_t stride[3],
                float *d_out, void *stream)
{
    if (!d_in || !d_out || !n || !stride || dims < 1 || dims > 3 || !valid_codec_rate(rate)) return ZFPX_EINVAL;
    for (int a = 0; a < 3; a++) if (n[a] < 1 || stride[a] < 0) return ZFPX_EINVAL;
    if (len < zfpx_stream_bytes(dims, rate, n)) return ZFPX_ESIZE;
    zfpx_plan p = nullptr;
    int rc = raw_plan(dims, n, stride, &p);
    if (rc) return rc;
    return zfpx_decompress_unpack(p, rate, d_in, len + 256, d_out, ZFPX_LAYOUT_SEND, stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// A transposition that allocates nothing.
//
// For callers that cannot allocate device memory at the point of the call --
// code running inside another framework's memory pool or allocator, real-time
// loops that must not pay for an allocation, programs with a fixed device
// memory map -- zfpx_transpose_noalloc keeps everything it needs beyond the
// caller's source and destination fields in one file-scope device array: the
// message table of the plan and the compressed messages (written straight
// into the receive layout, then decoded).  The array is ZFPX_NOALLOC_SCRATCH_BYTES
// long and stays reserved on every GPU that loads the library until the
// process exits.  Every call shares it and leaves its contents behind; nothing
// here depends on what an earlier call left (each call rewrites the table and
// every stream byte it later reads), but calls that overlap on the GPU -- on
// different streams, or from different host threads -- race on it.
#include <algorithm>
#include <mutex>
#include <vector>

static __device__ __align__(256) unsigned char g_noalloc_scratch[ZFPX_NOALLOC_SCRATCH_BYTES];

namespace zfpx {
namespace {
// device address of the scratch array, looked up once per device with that
// device current (a host-side name of the array is not a device address)
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64] = {nullptr};

int noalloc_scratch(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return ZFPX_ECUDA;
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ZFPX_ECUDA;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return ZFPX_OK;
}
}  // namespace
}  // namespace zfpx

extern "C" int zfpx_transpose_noalloc(zfpx_plan p, int rate, const float *d_src, float *d_dst, void *stream)
{
    if (!p || !d_src || !d_dst || !valid_codec_rate(rate)) return ZFPX_EINVAL;
    // message table (32-block work units, receive-layout offsets), built on the host
    const size_t M = p->msgs.size();
    std::vector<MsgDev> h(M);
    int64_t units = 0, so = 0, ro = 0;
    std::vector<int64_t> recv_off(M, 0);
    {
        std::vector<size_t> order(M);
        for (size_t i = 0; i < M; i++) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
            const HostMsg &x = p->msgs[a], &y = p->msgs[b];
            return x.dst != y.dst ? x.dst < y.dst : x.src_peer < y.src_peer;
        });
        for (size_t i : order) {
            recv_off[i] = ro;
            ro = (ro + message_bytes(p, p->msgs[i], rate) + 255) / 256 * 256;
        }
    }
    for (size_t i = 0; i < M; i++) {
        const HostMsg &m = p->msgs[i];
        MsgDev &d = h[i];
        const int64_t bx = (m.nx + 3) / 4;
        const int64_t by = p->dims >= 2 ? (m.ny + 3) / 4 : m.ny;
        const int64_t bz = p->dims == 3 ? (m.nz + 3) / 4 : m.nz;
        d.src_off = m.x0 * p->ss[0] + m.y0 * p->ss[1] + m.z0 * p->ss[2];
        d.dst_off = m.x0 * p->ds[0] + m.y0 * p->ds[1] + m.z0 * p->ds[2];
        d.off[0] = so;
        d.off[1] = recv_off[i];
        so = (so + message_bytes(p, m, rate) + 255) / 256 * 256;
        d.nx = (int32_t)m.nx; d.ny = (int32_t)m.ny; d.nz = (int32_t)m.nz;
        d.bx = (int32_t)bx; d.by = (int32_t)by; d.bz = (int32_t)bz;
        d.nblocks = bx * by * bz;
        set_block_divisors(d);
        d.unit0 = units;
        units += (d.nblocks + 31) / 32;
    }
    const size_t table_bytes = (M * sizeof(MsgDev) + 255) / 256 * 256;
    const size_t stream_bytes = (size_t)ro;
    // layout of the array: the message table, then the compressed messages
    if (table_bytes + stream_bytes > ZFPX_NOALLOC_SCRATCH_BYTES) return ZFPX_ESIZE;
    cudaStream_t st = (cudaStream_t)stream;
    // the table is copied from pageable host memory, which a stream capture
    // cannot record: refuse while the stream is capturing
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return ZFPX_ECUDA;
    if (cs != cudaStreamCaptureStatusNone) return ZFPX_EINVAL;
    void *scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    if (units == 0) return ZFPX_OK;
    // pageable source: the copy has read h before this call returns
    uint8_t *base = static_cast<uint8_t *>(scratch);
    if (cudaMemcpyAsync(base, h.data(), M * sizeof(MsgDev), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return ZFPX_ECUDA;
    uint8_t *buf = base + table_bytes;
    LaunchGeom g{};
    g.msgs = reinterpret_cast<const MsgDev *>(base);
    g.nmsg = (int)M;
    g.nunits = units;
    for (int a = 0; a < 3; a++) { g.ss[a] = p->ss[a]; g.ds[a] = p->ds[a]; }
    rc = launch_encode(p->dims, rate, d_src, buf, g, ZFPX_LAYOUT_RECV, vec_ok(d_src, p->ss, p, 0) ? 1 : 0, st);
    if (rc) return rc;
    return launch_decode(p->dims, rate, buf, d_dst, g, ZFPX_LAYOUT_RECV, vec_ok(d_dst, p->ds, p, 1) ? 1 : 0, st);
}
