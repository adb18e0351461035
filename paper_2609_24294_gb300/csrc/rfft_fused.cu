// Decompression fused with the longitude FFT (Sec. II-A: the FFT in longitude
// follows the first transposition; Sec. VI: the spectral transform's
// neighbouring steps).  After the z -> lambda all-to-all every receiving rank
// holds lambda-pencils whose rows run over all longitudes; instead of
// decompressing them into a float32 field in HBM and reading that back for
// the FFT, this kernel takes the received ZFP streams straight to the
// wavenumber fields F_m, m < K (the same values, bit for bit, as
// zfpx_decompress_unpack followed by zfpx_rfft_lon on the same rows).
//
// A work unit is one block row of a receiving pencil: 4 latitudes x 4 levels
// across all longitudes, i.e. the blocks (bx, by, bz) of every message the
// pencil receives, one message per source longitude range.  A CTA decodes the
// unit's blocks, one lane per block, into a per-CTA row buffer in global
// memory (16 rows x N floats, small enough to stay in L2 across the
// decode and the FFT that reads it back), then each warp takes rows of the
// buffer through the self-sorting FFT in its shared memory and writes the
// wavenumbers.  The float32 lambda-pencil never travels to HBM and back.
#include <algorithm>
#include <cstring>
#include <cuda_runtime.h>

#include "zfpx_internal.h"
#include "zfpx_block.cuh"
#include "zfpx_smem.cuh"
#include "zfpx_fft.cuh"

namespace zfpx {
namespace {

using namespace blk;

struct FusedMsg {
    int64_t off;             // byte offset of the message's stream in the receive layout
    int32_t x0, nx, bxn, byn;
};
struct FusedUnit {
    int32_t m0, nm;          // the unit's messages (sorted by x0)
    int32_t by, bz;          // block row inside the messages' boxes
    int32_t y0, z0;          // global latitude and level of the block row's first row
    int32_t nyr, nzr;        // real latitudes and levels in the block row (<= 4)
};

constexpr int kWarps = 4;
constexpr int kRows = 16;                      // rows per unit

template <int RATE>
constexpr int dec_smem_bytes() { return (2 * RATE + kTileZeroRows<RATE>) * 32 * 4 + 32 * 32 * 8; }

template <int RATE>
__global__ void __launch_bounds__(32 * kWarps)
decode_rfft_kernel(const uint8_t *__restrict__ in, const FusedMsg *__restrict__ msgs, const FusedUnit *__restrict__ units,
                   int nunits, float *__restrict__ scratch, int N, int NP, fft::FftGeom fg, const float2 *__restrict__ tw,
                   float *__restrict__ re, float *__restrict__ im, int64_t os1, int64_t os2, int warp_bytes)
{
    extern __shared__ __align__(16) uint8_t fsmem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, tid = threadIdx.x;
    uint8_t *wsm = fsmem + (size_t)wid * warp_bytes;
    uint32_t *t32 = reinterpret_cast<uint32_t *>(wsm);
    uint64_t *wpl = reinterpret_cast<uint64_t *>(wsm + (2 * RATE + kTileZeroRows<RATE>) * 32 * 4);
    float *rows = scratch + (size_t)blockIdx.x * kRows * NP;     // row pitch NP: a multiple of 4 floats
    for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
        const FusedUnit U = units[u];
        // ---- decode the unit's blocks into the row buffer
#pragma unroll
        for (int r = 0; r < kTileZeroRows<RATE>; r++) t32[(2 * RATE + r) * 32 + lane] = 0u;
        int nblk = 0;
        for (int m = 0; m < U.nm; m++) nblk += msgs[U.m0 + m].bxn;
        for (int t0 = 0; t0 < nblk; t0 += 32 * kWarps) {
            const int t = t0 + tid;
            if (t < nblk) {
                int m = U.m0, bx = t;
                while (bx >= msgs[m].bxn) { bx -= msgs[m].bxn; m++; }
                const FusedMsg M = msgs[m];
                const int64_t b = bx + (int64_t)M.bxn * (U.by + (int64_t)M.byn * U.bz);
                const uint4 *src4 = reinterpret_cast<const uint4 *>(in + M.off) + b * (RATE / 2);
#pragma unroll
                for (int i = 0; i < RATE / 2; i++) {
                    const uint4 v = __ldcs(src4 + i);
                    t32[(4 * i) * 32 + lane] = v.x;
                    t32[(4 * i + 1) * 32 + lane] = v.y;
                    t32[(4 * i + 2) * 32 + lane] = v.z;
                    t32[(4 * i + 3) * 32 + lane] = v.w;
                }
                float x[64];
                const StreamTile tile{t32, lane};
                SmemPlanes pl{wpl, lane};
                decode_block3_tile<RATE>(tile, x, pl);
                const int xg = M.x0 + 4 * bx;
                const bool full = 4 * bx + 4 <= M.nx && (xg & 3) == 0;
#pragma unroll
                for (int k = 0; k < 4; k++) {
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        if (k < U.nzr && j < U.nyr) {
                            float *row = rows + (size_t)(4 * k + j) * NP;
                            if (full) {
                                *reinterpret_cast<float4 *>(row + xg) = make_float4(
                                    x[16 * k + 4 * j], x[16 * k + 4 * j + 1], x[16 * k + 4 * j + 2], x[16 * k + 4 * j + 3]);
                            } else {
#pragma unroll
                                for (int i = 0; i < 4; i++)
                                    if (4 * bx + i < M.nx) row[xg + i] = x[16 * k + 4 * j + i];
                            }
                        }
                    }
                }
            }
            __syncwarp();
        }
        __syncthreads();
        // ---- the FFT of every real row, one warp per row
        float2 *X = reinterpret_cast<float2 *>(wsm), *Y = X + fg.H;
        for (int r = wid; r < kRows; r += kWarps) {
            const int k = r >> 2, j = r & 3;
            if (k >= U.nzr || j >= U.nyr) continue;
            const float2 *src = reinterpret_cast<const float2 *>(rows + (size_t)r * NP);
            fft::load_row_async(X, src, fg.H, lane);
            fft::wait_rows();
            __syncwarp();
            const int64_t o = (int64_t)(U.z0 + k) * os2 + (int64_t)(U.y0 + j) * os1;
            fft::rfft_row(X, Y, tw, fg, lane, re + o, im + o);
        }
        __syncthreads();
    }
}

// The units of a z -> lambda plan: messages grouped by receiver, each group
// sharing its latitude and level range and tiling the longitudes; false if
// the plan is not of that form.
bool build_units(const zfpx_plan_s *p, int rate, std::vector<FusedMsg> &fm, std::vector<FusedUnit> &fu)
{
    const std::vector<int64_t> ro = layout_offsets(p, rate, ZFPX_LAYOUT_RECV, nullptr);
    std::vector<size_t> order(p->msgs.size());
    for (size_t i = 0; i < order.size(); i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        const HostMsg &x = p->msgs[a], &y = p->msgs[b];
        return x.dst != y.dst ? x.dst < y.dst : x.x0 < y.x0;
    });
    fm.clear();
    fu.clear();
    for (size_t s = 0; s < order.size();) {
        size_t e = s;
        while (e < order.size() && p->msgs[order[e]].dst == p->msgs[order[s]].dst) e++;
        size_t hq = s;                                        // the group's first message with values
        while (hq < e && p->msgs[order[hq]].nx * p->msgs[order[hq]].ny * p->msgs[order[hq]].nz == 0) hq++;
        if (hq == e) { s = e; continue; }
        const HostMsg &h = p->msgs[order[hq]];
        const int32_t m0 = (int32_t)fm.size();
        int64_t xn = 0;
        for (size_t q = s; q < e; q++) {
            const HostMsg &m = p->msgs[order[q]];
            if (m.nx * m.ny * m.nz == 0) continue;
            if (m.y0 != h.y0 || m.ny != h.ny || m.z0 != h.z0 || m.nz != h.nz || m.x0 != xn) return false;
            fm.push_back(FusedMsg{ro[order[q]], (int32_t)m.x0, (int32_t)m.nx, (int32_t)((m.nx + 3) / 4),
                                  (int32_t)((m.ny + 3) / 4)});
            xn += m.nx;
        }
        const int32_t nm = (int32_t)fm.size() - m0;
        if (nm > 0) {
            if (xn != p->n[0]) return false;
            const int byn = (int)((h.ny + 3) / 4), bzn = (int)((h.nz + 3) / 4);
            for (int bz = 0; bz < bzn; bz++)
                for (int by = 0; by < byn; by++)
                    fu.push_back(FusedUnit{m0, nm, by, bz, (int32_t)(h.y0 + 4 * by), (int32_t)(h.z0 + 4 * bz),
                                           (int32_t)std::min<int64_t>(4, h.ny - 4 * by),
                                           (int32_t)std::min<int64_t>(4, h.nz - 4 * bz)});
        }
        s = e;
    }
    return true;
}

constexpr int kMaxCtasPerSm = 4;

int warp_bytes(int rate, int H)
{
    const int dec = rate == 8 ? dec_smem_bytes<8>() : dec_smem_bytes<16>();
    return (std::max(dec, (int)(2 * sizeof(float2)) * H) + 15) / 16 * 16;
}

}  // namespace
}  // namespace zfpx

using namespace zfpx;

extern "C" {

size_t zfpx_decompress_rfft_workspace_bytes(zfpx_plan p)
{
    if (!p) return 0;
    return (size_t)num_sms() * kMaxCtasPerSm * kRows * (size_t)((p->n[0] + 3) / 4 * 4) * sizeof(float);
}

int zfpx_decompress_rfft(zfpx_plan p, int rate, const uint8_t *d_recv, size_t len, int K, float *d_re, float *d_im,
                         const int64_t ostride[3], void *d_work, size_t work_bytes, void *stream)
{
    if (!p || !d_recv || !d_re || !d_im || !ostride || !d_work || !valid_codec_rate(rate)) return ZFPX_EINVAL;
    if (p->dims != 3 || p->transposition != 0) return ZFPX_EINVAL;
    const int64_t N = p->n[0];
    if (N < 2 || N % 2 || N > 8192 || K < 1 || K > N / 2 + 1) return ZFPX_EINVAL;
    if (ostride[0] != 1 || ostride[1] < 0 || ostride[2] < 0) return ZFPX_EINVAL;
    if (((uintptr_t)d_recv & 15u) || ((uintptr_t)d_re & 3u) || ((uintptr_t)d_im & 3u) || ((uintptr_t)d_work & 15u))
        return ZFPX_EINVAL;
    if ((int64_t)len < buffer_bytes(p, rate)) return ZFPX_ESIZE;
    if (work_bytes < zfpx_decompress_rfft_workspace_bytes(p)) return ZFPX_ESIZE;
    fft::FftGeom fg{};
    fg.N = (int)N; fg.H = (int)(N / 2); fg.K = K;
    if (!fft_plan_half(fg.H, fg)) return ZFPX_EINVAL;
    std::vector<FusedMsg> fm;
    std::vector<FusedUnit> fu;
    if (!build_units(p, rate, fm, fu)) return ZFPX_EINVAL;
    if (fu.empty()) return ZFPX_OK;
    const float2 *tw = nullptr;
    int rc = fft_twiddles(fg.N, &tw);
    if (rc) return rc;
    // unit tables: one upload per (plan, rate), kept with the plan
    DevTable *t = nullptr;
    {
        std::lock_guard<std::mutex> g(p->mu);
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return ZFPX_ECUDA;
        const long long key = ((long long)dev << 32) | ((long long)(rate + 1024) << 4) | 15ll;
        auto it = p->tables.find(key);
        if (it == p->tables.end()) {
            DevTable nt;
            const size_t mb = fm.size() * sizeof(FusedMsg), ub = fu.size() * sizeof(FusedUnit);
            if (cudaMalloc((void **)&nt.d_msgs, mb + ub) != cudaSuccess) return ZFPX_ENOMEM;
            std::vector<uint8_t> h(mb + ub);
            std::memcpy(h.data(), fm.data(), mb);
            std::memcpy(h.data() + mb, fu.data(), ub);
            if (cudaMemcpy(nt.d_msgs, h.data(), mb + ub, cudaMemcpyHostToDevice) != cudaSuccess) {
                cudaFree(nt.d_msgs);
                return ZFPX_ECUDA;
            }
            nt.nunits = (int64_t)fm.size();
            it = p->tables.emplace(key, nt).first;
        }
        t = &it->second;
    }
    const FusedMsg *d_msgs = reinterpret_cast<const FusedMsg *>(t->d_msgs);
    const FusedUnit *d_units = reinterpret_cast<const FusedUnit *>(reinterpret_cast<const uint8_t *>(t->d_msgs) +
                                                                  (size_t)t->nunits * sizeof(FusedMsg));
    const int wb = warp_bytes(rate, fg.H);
    const size_t smem = (size_t)kWarps * wb;
    const void *fn = rate == 8 ? (const void *)decode_rfft_kernel<8> : (const void *)decode_rfft_kernel<16>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return ZFPX_ECUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * kWarps, smem) != cudaSuccess) return ZFPX_ECUDA;
    per_sm = std::max(1, std::min(per_sm, kMaxCtasPerSm));
    const int grid = (int)std::min<int64_t>((int64_t)fu.size(), (int64_t)num_sms() * per_sm);
    float *scratch = static_cast<float *>(d_work);
    cudaStream_t st = (cudaStream_t)stream;
    if (rate == 8)
        decode_rfft_kernel<8><<<grid, 32 * kWarps, smem, st>>>(d_recv, d_msgs, d_units, (int)fu.size(), scratch, (int)N,
                                                               (int)((N + 3) / 4 * 4), fg, tw, d_re, d_im, ostride[1], ostride[2], wb);
    else
        decode_rfft_kernel<16><<<grid, 32 * kWarps, smem, st>>>(d_recv, d_msgs, d_units, (int)fu.size(), scratch, (int)N,
                                                                (int)((N + 3) / 4 * 4), fg, tw, d_re, d_im, ostride[1], ostride[2], wb);
    count_launch();
    return check_launch();
}

}  // extern "C"
