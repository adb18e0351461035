// Comparator packs and the device-local all-to-all (sm_103a).
//
// zfpx_pack / zfpx_unpack: the plain float32 message buffer (paper Table 1,
// column "Float32").  zfpx_cast_fp16_pack / zfpx_fp16_unpack: the float16
// cast comparator (Sec. I; Sec. IV-D counts its cost as nil; Sec. IV-F
// measures its error by a round trip through float16).  zfpx_permute: the all-to-all of
// Sec. II-B on one device, recv[dst][src] <- send[src][dst].
// zfpx_count_nonfinite: the debug report of non-finite inputs, which the
// codec codes as zero blocks (the paper leaves such inputs unspecified).
//
// All three are pure data movement, bound by HBM bandwidth: every lane moves
// one 16-byte quad (4 values, or 16 stream bytes) per step, warps take
// contiguous unit ranges, and vector accesses are used wherever both sides
// are 16-byte (8 for halves) aligned.
#include <climits>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "zfpx_internal.h"

namespace zfpx {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;

struct LaneWalk {
    const MsgDev *msgs;
    int nmsg, mi;
    int64_t next0;
    __device__ __forceinline__ void start(const MsgDev *m, int n, int64_t u)
    {
        msgs = m; nmsg = n;
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (m[mid].unit0 <= u) lo = mid; else hi = mid - 1;
        }
        mi = lo;
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

// A lane's position among the quads (4 consecutive values along x) of one
// message: quad index in its row, row (y) and level (z).  Found by division
// when the lane enters a message, then stepped forward 32 quads at a time
// without dividing.
struct QuadPos {
    int quad, y, z;
    __device__ __forceinline__ void set(const MsgDev &m, int64_t rel)
    {
        const int qpr = (m.nx + 3) >> 2;
        const int row = (int)(rel / qpr);
        quad = (int)(rel - (int64_t)row * qpr);
        y = row % m.ny;
        z = row / m.ny;
    }
    __device__ __forceinline__ void step32(const MsgDev &m)
    {
        const int qpr = (m.nx + 3) >> 2;
        quad += 32;
        if (quad < qpr) return;
        int d = 1;
        if (qpr >= 32) quad -= qpr;
        else { d = quad / qpr; quad -= d * qpr; }
        y += d;
        while (y >= m.ny) { y -= m.ny; z++; }
    }
};

// MODE 0: f32 pack, 1: f32 unpack, 2: f16 pack RN, 3: f16 pack RZ, 4: f16 unpack
template <int MODE>
__global__ void __launch_bounds__(kThreads)
quad_kernel(const void *__restrict__ in, void *__restrict__ out, LaunchGeom g, int layout, int view_vec)
{
    constexpr bool pack = (MODE == 0 || MODE == 2 || MODE == 3);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t W = (int64_t)gridDim.x * kWarps;
    const int64_t gw = (int64_t)blockIdx.x * kWarps + wid;
    const int64_t u0 = gw * g.nunits / W, u1 = (gw + 1) * g.nunits / W;
    if (u0 + lane >= u1) return;
    LaneWalk walk;
    walk.start(g.msgs, g.nmsg, u0 + lane);
    int mi = -1;
    QuadPos qp;
    const int64_t *s = pack ? g.ss : g.ds;
    for (int64_t u = u0 + lane; u < u1; u += 32) {
        walk.advance(u);
        const MsgDev &m = g.msgs[walk.mi];
        if (walk.mi != mi) { mi = walk.mi; qp.set(m, u - m.unit0); }
        const int x = 4 * qp.quad;
        const int cnt = min(4, m.nx - x);
        const int64_t view_off = (pack ? m.src_off : m.dst_off) + (int64_t)x * s[0] + (int64_t)qp.y * s[1] +
                                 (int64_t)qp.z * s[2];
        const int64_t e = ((int64_t)qp.z * m.ny + qp.y) * m.nx + x;   // index inside the message
        const int64_t vs = s[0];
        const bool vview = view_vec && cnt == 4 && (view_off & 3) == 0;
        const bool vbuf = cnt == 4 && (e & 3) == 0;
        qp.step32(m);
        float v[4];
        if (pack) {
            const float *src = reinterpret_cast<const float *>(in) + view_off;
            if (vview) {
                const float4 f = __ldg(reinterpret_cast<const float4 *>(src));
                v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
            } else {
#pragma unroll
                for (int i = 0; i < 4; i++) v[i] = i < cnt ? __ldg(src + i * vs) : 0.0f;
            }
            if (MODE == 0) {
                float *dst = reinterpret_cast<float *>(reinterpret_cast<uint8_t *>(out) + m.off[layout]) + e;
                if (vbuf) *reinterpret_cast<float4 *>(dst) = make_float4(v[0], v[1], v[2], v[3]);
                else
                    for (int i = 0; i < cnt; i++) dst[i] = v[i];
            } else {
                __half h[4];
#pragma unroll
                for (int i = 0; i < 4; i++) h[i] = MODE == 2 ? __float2half_rn(v[i]) : __float2half_rz(v[i]);
                __half *dst = reinterpret_cast<__half *>(reinterpret_cast<uint8_t *>(out) + m.off[layout]) + e;
                if (vbuf) {
                    uint2 w;
                    w.x = (uint32_t)__half_as_ushort(h[0]) | ((uint32_t)__half_as_ushort(h[1]) << 16);
                    w.y = (uint32_t)__half_as_ushort(h[2]) | ((uint32_t)__half_as_ushort(h[3]) << 16);
                    *reinterpret_cast<uint2 *>(dst) = w;
                } else {
                    for (int i = 0; i < cnt; i++) dst[i] = h[i];
                }
            }
        } else {
            if (MODE == 1) {
                const float *src = reinterpret_cast<const float *>(reinterpret_cast<const uint8_t *>(in) + m.off[layout]) + e;
                if (vbuf) {
                    const float4 f = __ldg(reinterpret_cast<const float4 *>(src));
                    v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
                } else {
#pragma unroll
                    for (int i = 0; i < 4; i++) v[i] = i < cnt ? __ldg(src + i) : 0.0f;
                }
            } else {
                const __half *src = reinterpret_cast<const __half *>(reinterpret_cast<const uint8_t *>(in) + m.off[layout]) + e;
                if (vbuf) {
                    const uint2 w = __ldg(reinterpret_cast<const uint2 *>(src));
                    v[0] = __half2float(__ushort_as_half((unsigned short)(w.x & 0xffffu)));
                    v[1] = __half2float(__ushort_as_half((unsigned short)(w.x >> 16)));
                    v[2] = __half2float(__ushort_as_half((unsigned short)(w.y & 0xffffu)));
                    v[3] = __half2float(__ushort_as_half((unsigned short)(w.y >> 16)));
                } else {
#pragma unroll
                    for (int i = 0; i < 4; i++) v[i] = i < cnt ? __half2float(src[i]) : 0.0f;
                }
            }
            float *dst = reinterpret_cast<float *>(out) + view_off;
            if (vview) *reinterpret_cast<float4 *>(dst) = make_float4(v[0], v[1], v[2], v[3]);
            else
                for (int i = 0; i < cnt; i++) dst[i * vs] = v[i];
        }
    }
}

// Moves every message from its send slot to its receive slot, 16 bytes per lane.
__global__ void __launch_bounds__(kThreads)
permute_kernel(const uint8_t *__restrict__ send, uint8_t *__restrict__ recv, LaunchGeom g, int rate, int dims)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t W = (int64_t)gridDim.x * kWarps;
    const int64_t gw = (int64_t)blockIdx.x * kWarps + wid;
    const int64_t u0 = gw * g.nunits / W, u1 = (gw + 1) * g.nunits / W;
    if (u0 + lane >= u1) return;
    LaneWalk walk;
    walk.start(g.msgs, g.nmsg, u0 + lane);
    for (int64_t u = u0 + lane; u < u1; u += 32) {
        walk.advance(u);
        const MsgDev &m = g.msgs[walk.mi];
        const int64_t nv = (int64_t)m.nx * m.ny * m.nz;
        const int64_t bytes = rate == ZFPX_RATE_F32 ? 4 * nv
                            : rate == ZFPX_RATE_F16 ? 2 * nv
                            : (dims == 3 ? m.nblocks * 8 * rate : dims == 2 ? m.nblocks * 2 * rate : m.nblocks * rate / 2);
        const int64_t o = (u - m.unit0) * 16;
        const uint8_t *a = send + m.off[0] + o;
        uint8_t *b = recv + m.off[1] + o;
        if (o + 16 <= bytes) {
            *reinterpret_cast<uint4 *>(b) = __ldg(reinterpret_cast<const uint4 *>(a));
        } else {
            for (int64_t i = 0; o + i < bytes; i++) b[i] = a[i];
        }
    }
}

template <class K>
int grid_for(K kernel, int64_t nunits_per_warp_step)
{
    const int occ = occupancy((const void *)kernel, kThreads);
    const int64_t want = (nunits_per_warp_step + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)num_sms() * occ;
    return (int)std::max<int64_t>(1, std::min(want, cap));
}

bool view_vec(const void *ptr, const int64_t s[3])
{
    return (((uintptr_t)ptr & 15u) == 0) && s[0] == 1;
}

int run_quads(zfpx_plan p, int mode, int rate, const void *in, void *out, int layout, bool to_buf,
              size_t buf_len, cudaStream_t st)
{
    if (layout != ZFPX_LAYOUT_SEND && layout != ZFPX_LAYOUT_RECV) return ZFPX_EINVAL;
    if ((int64_t)buf_len < buffer_bytes(p, rate)) return ZFPX_ESIZE;
    const void *bufp = to_buf ? out : in;
    if ((uintptr_t)bufp & 15u) return ZFPX_EINVAL;
    DevTable *t = nullptr;
    int rc = get_table(p, rate, UNIT_QUADS, &t);
    if (rc) return rc;
    if (t->nunits == 0) return ZFPX_OK;
    LaunchGeom g{};
    g.msgs = t->d_msgs; g.nmsg = (int)p->msgs.size(); g.nunits = t->nunits;
    for (int a = 0; a < 3; a++) { g.ss[a] = p->ss[a]; g.ds[a] = p->ds[a]; }
    const int vv = view_vec(to_buf ? in : out, to_buf ? p->ss : p->ds) ? 1 : 0;
    switch (mode) {
    case 0: quad_kernel<0><<<grid_for(quad_kernel<0>, g.nunits), kThreads, 0, st>>>(in, out, g, layout, vv); break;
    case 1: quad_kernel<1><<<grid_for(quad_kernel<1>, g.nunits), kThreads, 0, st>>>(in, out, g, layout, vv); break;
    case 2: quad_kernel<2><<<grid_for(quad_kernel<2>, g.nunits), kThreads, 0, st>>>(in, out, g, layout, vv); break;
    case 3: quad_kernel<3><<<grid_for(quad_kernel<3>, g.nunits), kThreads, 0, st>>>(in, out, g, layout, vv); break;
    default: quad_kernel<4><<<grid_for(quad_kernel<4>, g.nunits), kThreads, 0, st>>>(in, out, g, layout, vv); break;
    }
    count_launch();
    return check_launch();
}

// Number of elements of a strided view whose exponent field is all ones (the
// infinities and NaNs; U = uint32_t for float32, uint64_t for float64): a
// grid-stride loop over the view's elements in raster order, a warp sum,
// one atomic add per warp into *out.
template <class U>
__global__ void __launch_bounds__(kThreads) count_nonfinite_kernel(const U *__restrict__ src, int64_t n0, int64_t n1,
                                                                   int64_t total, int64_t s0, int64_t s1, int64_t s2,
                                                                   U emask, unsigned long long *out)
{
    unsigned long long c = 0;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += step) {
        const int64_t t = i / n0, x = i - t * n0;
        const int64_t z = t / n1, y = t - z * n1;
        c += (__ldg(src + x * s0 + y * s1 + z * s2) & emask) == emask ? 1ull : 0ull;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

}  // namespace

int launch_permute(const uint8_t *send, uint8_t *recv, const LaunchGeom &g, int rate, int dims, cudaStream_t st)
{
    if (g.nunits == 0) return ZFPX_OK;
    permute_kernel<<<grid_for(permute_kernel, g.nunits), kThreads, 0, st>>>(send, recv, g, rate, dims);
    count_launch();
    return check_launch();
}
}  // namespace zfpx

using namespace zfpx;

extern "C" {

int zfpx_pack(zfpx_plan p, const float *d_src, float *d_out, size_t cap_bytes, int layout, void *stream)
{
    if (!p || !d_src || !d_out) return ZFPX_EINVAL;
    return run_quads(p, 0, ZFPX_RATE_F32, d_src, d_out, layout, true, cap_bytes, (cudaStream_t)stream);
}

int zfpx_unpack(zfpx_plan p, const float *d_in, size_t len_bytes, float *d_dst, int layout, void *stream)
{
    if (!p || !d_in || !d_dst) return ZFPX_EINVAL;
    return run_quads(p, 1, ZFPX_RATE_F32, d_in, d_dst, layout, false, len_bytes, (cudaStream_t)stream);
}

int zfpx_cast_fp16_pack(zfpx_plan p, int round_mode, const float *d_src, uint16_t *d_out, size_t cap_bytes,
                        int layout, void *stream)
{
    if (!p || !d_src || !d_out) return ZFPX_EINVAL;
    if (round_mode != ZFPX_ROUND_NEAREST && round_mode != ZFPX_ROUND_ZERO) return ZFPX_EINVAL;
    return run_quads(p, round_mode == ZFPX_ROUND_NEAREST ? 2 : 3, ZFPX_RATE_F16, d_src, d_out, layout, true,
                     cap_bytes, (cudaStream_t)stream);
}

int zfpx_fp16_unpack(zfpx_plan p, const uint16_t *d_in, size_t len_bytes, float *d_dst, int layout, void *stream)
{
    if (!p || !d_in || !d_dst) return ZFPX_EINVAL;
    return run_quads(p, 4, ZFPX_RATE_F16, d_in, d_dst, layout, false, len_bytes, (cudaStream_t)stream);
}

int zfpx_permute(zfpx_plan p, int rate, const void *d_send, void *d_recv, size_t len, void *stream)
{
    if (!p || !d_send || !d_recv) return ZFPX_EINVAL;
    if (rate != ZFPX_RATE_F32 && rate != ZFPX_RATE_F16 && !valid_codec_rate(rate)) return ZFPX_EINVAL;
    if (((uintptr_t)d_send & 15u) || ((uintptr_t)d_recv & 15u)) return ZFPX_EINVAL;
    const int64_t need = buffer_bytes(p, rate);
    if ((int64_t)len < need) return ZFPX_ESIZE;
    const uint8_t *a = (const uint8_t *)d_send;
    const uint8_t *b = (const uint8_t *)d_recv;
    if (a < b + need && b < a + need) return ZFPX_EINVAL;    // overlap
    DevTable *t = nullptr;
    int rc = get_table(p, rate, UNIT_CHUNK16, &t);
    if (rc) return rc;
    LaunchGeom g{};
    g.msgs = t->d_msgs; g.nmsg = (int)p->msgs.size(); g.nunits = t->nunits;
    return launch_permute(a, (uint8_t *)d_recv, g, rate, p->dims, (cudaStream_t)stream);
}

int zfpx_count_nonfinite(const void *d_src, int elem_bytes, const int64_t n[3], const int64_t stride[3],
                         unsigned long long *d_count, void *stream)
{
    if (!d_src || !n || !stride || !d_count) return ZFPX_EINVAL;
    if (elem_bytes != 4 && elem_bytes != 8) return ZFPX_EINVAL;
    if (((uintptr_t)d_src % (uintptr_t)elem_bytes) || ((uintptr_t)d_count & 7u)) return ZFPX_EINVAL;
    for (int a = 0; a < 3; a++)
        if (n[a] < 0 || stride[a] < 0) return ZFPX_EINVAL;
    if (n[0] == 0 || n[1] == 0 || n[2] == 0) return ZFPX_OK;
    if (n[0] > INT64_MAX / n[1] || n[0] * n[1] > INT64_MAX / n[2]) return ZFPX_EINVAL;
    const int64_t total = n[0] * n[1] * n[2];
    const cudaStream_t st = (cudaStream_t)stream;
    const int64_t want = (total + kThreads - 1) / kThreads;
    if (elem_bytes == 4) {
        const int occ = occupancy((const void *)count_nonfinite_kernel<uint32_t>, kThreads);
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms() * occ));
        count_nonfinite_kernel<uint32_t><<<grid, kThreads, 0, st>>>(
            (const uint32_t *)d_src, n[0], n[1], total, stride[0], stride[1], stride[2], 0x7f800000u, d_count);
    } else {
        const int occ = occupancy((const void *)count_nonfinite_kernel<uint64_t>, kThreads);
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms() * occ));
        count_nonfinite_kernel<uint64_t><<<grid, kThreads, 0, st>>>((const uint64_t *)d_src, n[0], n[1], total,
                                                                    stride[0], stride[1], stride[2],
                                                                    0x7ff0000000000000ull, d_count);
    }
    count_launch();
    return check_launch();
}

}  // extern "C"
