// Internal declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cstddef>
#include <vector>
#include <mutex>
#include <map>

#include <cuda_runtime.h>

#include "../../include/zfpx.h"

namespace zfpx {

// One message as the kernels see it.  Element offsets are into the plan's
// src / dst views; byte offsets into the send / receive layouts.
struct MsgDev {
    int64_t src_off;    // element offset of the box origin in the source view
    int64_t dst_off;    // element offset of the box origin in the destination view
    int64_t off[2];     // byte offset in the send [0] and receive [1] layout
    int64_t unit0;      // first work unit (warp chunk or row quad) of this message
    int32_t nx, ny, nz; // box extents
    int32_t bx, by, bz; // block counts (dims 3: ceil(n/4) each; dims 1: ceil(nx/4), ny, nz)
    int64_t nblocks;    // bx * by * bz
    uint32_t bxm, bym;  // divisors of bx and by for divu (set_block_divisors)
    int32_t bxl, byl;
};

// Exact unsigned 32-bit division by an invariant d >= 1 as a high multiply,
// an add and shifts (Granlund and Montgomery, "Division by invariant integers
// using multiplication", 1994): l = ceil(log2 d), m = floor(2^32 (2^l - d) / d)
// + 1, then n / d = (t + ((n - t) >> 1)) >> (l - 1) with t = mulhi(n, m), and
// n itself when d = 1.
inline void block_divisor(uint32_t d, uint32_t &m, int32_t &l)
{
    l = 0;
    while (l < 32 && ((uint64_t)1 << l) < d) l++;
    m = (uint32_t)(((((uint64_t)1 << l) - d) << 32) / d + 1);
}
inline void set_block_divisors(MsgDev &d)
{
    block_divisor((uint32_t)d.bx, d.bxm, d.bxl);
    block_divisor((uint32_t)d.by, d.bym, d.byl);
}
#ifdef __CUDACC__
__device__ __forceinline__ uint32_t divu(uint32_t n, uint32_t m, int32_t l)
{
    const uint32_t t = __umulhi(n, m);
    return l ? (t + ((n - t) >> 1)) >> (l - 1) : n;
}
#endif

// Arguments common to every plan-driven launch.
struct LaunchGeom {
    const MsgDev *msgs; // device table (nmsg entries)
    int nmsg;
    int64_t nunits;     // total work units
    int64_t ss[3];      // source strides (elements)
    int64_t ds[3];      // destination strides (elements)
    int32_t upw;        // 3-D codec kernels: consecutive work units per warp (grid = units / (upw * warps))
};

struct HostMsg {
    int32_t src, dst, src_peer, dst_peer;
    int64_t x0, nx, y0, ny, z0, nz;
};

// Device tables of one (rate, unit kind, device) for a plan.
struct DevTable {
    MsgDev *d_msgs = nullptr;   // the message table
    int64_t nunits = 0;
};

}  // namespace zfpx

struct zfpx_plan_s {
    int64_t n[3];
    int64_t ss[3], ds[3];
    int pr, pc, P, transposition, dims, split_mode;
    std::vector<zfpx::HostMsg> msgs;              // send order
    std::mutex mu;
    std::map<long long, zfpx::DevTable> tables;   // key: (device, rate, unit kind)
};

namespace zfpx {

// Work-unit kinds: codec kernels take 32 blocks (one warp) per unit; packs
// take 4-value quads of one row per unit; the permutation 16 stream bytes.
enum UnitKind { UNIT_BLOCKS32 = 0, UNIT_QUADS = 1, UNIT_CHUNK16 = 2 };

int64_t message_bytes(const zfpx_plan_s *p, const HostMsg &m, int rate);
// Offsets of every message (send-order index) in the given layout; the total in *total.
std::vector<int64_t> layout_offsets(const zfpx_plan_s *p, int rate, int layout, int64_t *total);
int64_t buffer_bytes(const zfpx_plan_s *p, int rate);
// Fetches (building on first use) the device table; returns ZFPX_OK or an error.
int get_table(zfpx_plan_s *p, int rate, UnitKind kind, DevTable **out);
// Host copy of the table of the messages `subset` (send-order indices; empty
// = every message), work units numbered from 0 within it; returns the units.
// Offsets stay those of the whole plan's layouts.
int64_t host_table(const zfpx_plan_s *p, int rate, UnitKind kind, const std::vector<int> &subset,
                   std::vector<MsgDev> &h);
// Uploads a host table into a new device allocation (t->d_msgs, freed by the owner).
int upload_table(const std::vector<MsgDev> &h, int64_t units, DevTable *t);

// Kernel launchers over a table (geometry g: table, units, view strides).
// vec: every row the kernel touches starts on 16 bytes.
int launch_encode(int dims, int rate, const float *src, uint8_t *out, const LaunchGeom &g, int layout, int vec,
                  cudaStream_t st);
int launch_decode(int dims, int rate, const uint8_t *in, float *dst, const LaunchGeom &g, int layout, int vec,
                  cudaStream_t st);
int launch_permute(const uint8_t *send, uint8_t *recv, const LaunchGeom &g, int rate, int dims, cudaStream_t st);
// vec test of the codec kernels for a pointer and view strides over the plan's messages.
bool codec_vec_ok(const void *ptr, const int64_t s[3], const zfpx_plan_s *p);

int num_sms();
// Resident CTAs per SM of `fn` at `threads` threads (cached per kernel).
int occupancy(const void *fn, int threads);
void count_launch();
void uncount_launches(uint64_t n);   // launches recorded into a graph, not run
bool valid_codec_rate(int rate);
int check_launch();   // cudaGetLastError -> ZFPX_OK / ZFPX_ECUDA
// Work units per warp of the 3-D codec kernels for (direction, rate); 0 = the
// library's default.  Set through zfpx_set_units_per_warp (the autotuner).
int units_per_warp(int encode, int rate);

}  // namespace zfpx
