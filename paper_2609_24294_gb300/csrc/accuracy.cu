// Accuracy and precision modes: variable-rate coding of 3-D blocks to an
// absolute error tolerance, or to a fixed number of bit planes per block (the
// ZFP modes the paper names and leaves for future work, Sec. II-C), built on
// the fixed-rate kernels.  Precision p keeps planes 31 .. 32 - p; the rest of
// what follows holds for both.
//
// Readings (identical in the CPU oracle): minexp = floor(log2 tol); a block
// with exponent e_max keeps its bit planes 31 .. kmin, kmin = clamp(minexp -
// e_max + 22, 0, 32), cut at the rate-16 budget of 1024 bits; a zero block is
// its one 0 bit, a block with kmin = 32 its 9 header bits.  Because the plane
// coder is embedded, a block's accuracy-mode bits are the first L bits of its
// rate-16 stream, and the rate-16 decoder reads the same block from those L
// bits followed by zeros (zeros after the last coded plane are empty planes).
//
// Encode: the rate-16 encoder writes every block to a 128-byte slot; one
// thread per block walks its slot's planes down to kmin to find L; an
// exclusive scan of the L (per 1024-block tile, then over the tiles) gives
// every block's bit offset; one thread per block ORs its L bits into the
// zeroed payload at that offset (words shared by neighbouring blocks take
// atomic ORs).  Decode: the same scan, one thread per block copies its L bits
// back into a zeroed slot, then the rate-16 decoder.
#include <algorithm>
#include <cmath>
#include <vector>
#include <cuda_runtime.h>

#include "zfpx_internal.h"
#include "zfpx_block.cuh"

namespace zfpx {
namespace {

using namespace blk;

constexpr int kTile = 1024;                  // blocks per scan tile (one CTA)
constexpr int kSlotWords = 16;               // 1024 bits per block slot
constexpr int kCutBits = 64 * kSlotWords;

// Lowest plane kept: the accuracy rule, or 32 - prec in precision mode (prec > 0).
__device__ __forceinline__ int acc_kmin(int emax, int minexp, int prec)
{
    if (prec > 0) return 32 - prec;
    const int k = minexp - emax + 22;
    return k < 0 ? 0 : (k > 32 ? 32 : k);
}

// Reader over one block's slot in global memory; bits past the slot read as 0.
struct SlotReader {
    const uint64_t *w;
    int pos;
    __device__ __forceinline__ uint64_t peek() const
    {
        const int i = pos >> 6, sh = pos & 63;
        const uint64_t lo = i < kSlotWords ? __ldg(w + i) : 0ull;
        const uint64_t hi = i + 1 < kSlotWords ? __ldg(w + i + 1) : 0ull;
        return sh ? (lo >> sh) | (hi << (64 - sh)) : lo;
    }
    __device__ __forceinline__ void skip(int k) { pos += k; }
};

// L for every block: parse the slot's planes 31 .. kmin with the rate-16 budget.
__global__ void __launch_bounds__(256) acc_lengths_kernel(const uint64_t *__restrict__ slots, int64_t nblocks,
                                                          int minexp, int prec, uint16_t *__restrict__ lengths)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblocks) return;
    const uint64_t *w = slots + b * kSlotWords;
    const uint64_t head = __ldg(w);
    int L;
    if (!(head & 1ull)) {
        L = 1;
    } else {
        const int emax = (int)((head >> 1) & 0xffu) - 127;
        const int kmin = acc_kmin(emax, minexp, prec);
        SlotReader rd{w, 9};
        int n = 0, R = kCutBits - 9;
#pragma unroll 1
        for (int k = 31; k >= kmin && R > 0; k--) (void)decode_plane<64>(rd, n, R);
        L = kCutBits - R;
    }
    lengths[b] = (uint16_t)L;
}

// Exclusive scan of the lengths inside each tile of kTile blocks; the tile's
// total goes to totals[tile].
__global__ void __launch_bounds__(kTile) acc_scan_tiles_kernel(const uint16_t *__restrict__ lengths,
                                                               int64_t nblocks, uint32_t *__restrict__ local,
                                                               uint64_t *__restrict__ totals)
{
    __shared__ uint32_t warp_sum[kTile / 32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int64_t b = (int64_t)blockIdx.x * kTile + t;
    const uint32_t v = b < nblocks ? lengths[b] : 0u;
    uint32_t x = v;                                        // inclusive scan in the warp
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_sum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = warp_sum[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, s, d);
            if (lane >= d) s += y;
        }
        warp_sum[lane] = s;                                // inclusive over warps
    }
    __syncthreads();
    const uint32_t before = (wid ? warp_sum[wid - 1] : 0u) + x - v;
    if (b < nblocks) local[b] = before;
    if (t == kTile - 1) totals[blockIdx.x] = warp_sum[kTile / 32 - 1];
}

// Exclusive scan of the tile totals (one CTA, sequential over chunks of
// kTile tiles); the grand total goes to *total_bits.
__global__ void __launch_bounds__(kTile) acc_scan_totals_kernel(const uint64_t *__restrict__ totals, int64_t ntiles,
                                                                uint64_t *__restrict__ tile_off,
                                                                uint64_t *__restrict__ total_bits)
{
    __shared__ uint64_t warp_sum[kTile / 32];
    __shared__ uint64_t carry;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    if (t == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < ntiles; base += kTile) {
        const int64_t i = base + t;
        const uint64_t v = i < ntiles ? totals[i] : 0ull;
        uint64_t x = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) warp_sum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            uint64_t s = warp_sum[lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint64_t y = __shfl_up_sync(0xffffffffu, s, d);
                if (lane >= d) s += y;
            }
            warp_sum[lane] = s;
        }
        __syncthreads();
        const uint64_t c = carry;
        if (i < ntiles) tile_off[i] = c + (wid ? warp_sum[wid - 1] : 0ull) + x - v;
        __syncthreads();
        if (t == 0) carry = c + warp_sum[kTile / 32 - 1];
        __syncthreads();
    }
    if (t == 0) *total_bits = carry;
}

// Every block ORs its L bits into the zeroed payload at its bit offset.
__global__ void __launch_bounds__(256) acc_pack_kernel(const uint64_t *__restrict__ slots, int64_t nblocks,
                                                       const uint16_t *__restrict__ lengths,
                                                       const uint32_t *__restrict__ local,
                                                       const uint64_t *__restrict__ tile_off,
                                                       unsigned long long *__restrict__ payload)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblocks) return;
    const uint64_t off = tile_off[b / kTile] + local[b];
    const int L = lengths[b];
    const uint64_t *w = slots + b * kSlotWords;
    const int sh = (int)(off & 63);
    unsigned long long *d = payload + (off >> 6);
#pragma unroll 1
    for (int i = 0; 64 * i < L; i++) {
        uint64_t v = __ldg(w + i);
        const int rem = L - 64 * i;
        if (rem < 64) v &= (1ull << rem) - 1ull;
        if (!v) continue;
        atomicOr(d + i, (unsigned long long)(v << sh));
        if (sh && (v >> (64 - sh))) atomicOr(d + i + 1, (unsigned long long)(v >> (64 - sh)));
    }
}

// Every block copies its L bits back into a zeroed 1024-bit slot.
__global__ void __launch_bounds__(256) acc_unpack_kernel(const uint64_t *__restrict__ payload, int64_t pwords,
                                                         int64_t nblocks, const uint16_t *__restrict__ lengths,
                                                         const uint32_t *__restrict__ local,
                                                         const uint64_t *__restrict__ tile_off,
                                                         uint64_t *__restrict__ slots)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblocks) return;
    const uint64_t off = tile_off[b / kTile] + local[b];
    const int L = min((int)lengths[b], kCutBits);
    const int sh = (int)(off & 63);
    const int64_t j0 = (int64_t)(off >> 6);
    uint64_t *s = slots + b * kSlotWords;
#pragma unroll
    for (int i = 0; i < kSlotWords; i++) {
        uint64_t v = 0;
        const int rem = L - 64 * i;
        if (rem > 0) {
            const int64_t j = j0 + i;
            const uint64_t lo = j < pwords ? __ldg(payload + j) : 0ull;
            const uint64_t hi = (sh && j + 1 < pwords) ? __ldg(payload + j + 1) : 0ull;
            v = sh ? (lo >> sh) | (hi << (64 - sh)) : lo;
            if (rem < 64) v &= (1ull << rem) - 1ull;
        }
        s[i] = v;
    }
}

struct AccWork {
    uint64_t *slots;
    uint32_t *local;
    uint64_t *totals, *tile_off, *total;
    int64_t nblocks, ntiles;
};

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

int64_t acc_blocks(const int64_t n[3]) { return ((n[0] + 3) / 4) * ((n[1] + 3) / 4) * ((n[2] + 3) / 4); }

size_t acc_work_bytes(int64_t nb)
{
    const int64_t nt = (nb + kTile - 1) / kTile;
    return align256((size_t)nb * 128) + align256((size_t)nb * 4) + 2 * align256((size_t)nt * 8) + 256;
}

AccWork acc_carve(void *work, int64_t nb)
{
    AccWork a;
    a.nblocks = nb;
    a.ntiles = (nb + kTile - 1) / kTile;
    char *p = static_cast<char *>(work);
    a.slots = reinterpret_cast<uint64_t *>(p); p += align256((size_t)nb * 128);
    a.local = reinterpret_cast<uint32_t *>(p); p += align256((size_t)nb * 4);
    a.totals = reinterpret_cast<uint64_t *>(p); p += align256((size_t)a.ntiles * 8);
    a.tile_off = reinterpret_cast<uint64_t *>(p); p += align256((size_t)a.ntiles * 8);
    a.total = reinterpret_cast<uint64_t *>(p);
    return a;
}

int acc_scan(const AccWork &a, const uint16_t *lengths, uint64_t *total_bits, cudaStream_t st)
{
    acc_scan_tiles_kernel<<<(unsigned)a.ntiles, kTile, 0, st>>>(lengths, a.nblocks, a.local, a.totals);
    count_launch();
    acc_scan_totals_kernel<<<1, kTile, 0, st>>>(a.totals, a.ntiles, a.tile_off, total_bits);
    count_launch();
    return check_launch();
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

}  // namespace
}  // namespace zfpx

using namespace zfpx;

extern "C" {

size_t zfpx_accuracy_workspace_bytes(const int64_t n[3])
{
    if (!n || n[0] < 1 || n[1] < 1 || n[2] < 1) return 0;
    return acc_work_bytes(acc_blocks(n));
}

size_t zfpx_accuracy_max_payload_bytes(const int64_t n[3])
{
    if (!n || n[0] < 1 || n[1] < 1 || n[2] < 1) return 0;
    return (size_t)acc_blocks(n) * 128;
}

static int encode_variable(const float *d_in, const int64_t n[3], const int64_t stride[3], int minexp, int prec,
                           uint16_t *d_lengths, uint8_t *d_payload, size_t cap, uint64_t *d_total_bits,
                           void *d_work, size_t work_bytes, void *stream)
{
    if (!d_in || !n || !stride || !d_lengths || !d_payload || !d_total_bits || !d_work) return ZFPX_EINVAL;
    for (int a = 0; a < 3; a++) if (n[a] < 1 || stride[a] < 0) return ZFPX_EINVAL;
    if (!aligned(d_payload, 8) || !aligned(d_work, 256) || !aligned(d_lengths, 2) || !aligned(d_total_bits, 8))
        return ZFPX_EINVAL;
    const int64_t nb = acc_blocks(n);
    if (cap < (size_t)nb * 128 || work_bytes < acc_work_bytes(nb)) return ZFPX_ESIZE;
    cudaStream_t st = (cudaStream_t)stream;
    const AccWork a = acc_carve(d_work, nb);
    int rc = zfpx_encode(3, 16, d_in, n, stride, reinterpret_cast<uint8_t *>(a.slots), (size_t)nb * 128, stream);
    if (rc) return rc;
    const unsigned grid = (unsigned)((nb + 255) / 256);
    acc_lengths_kernel<<<grid, 256, 0, st>>>(a.slots, nb, minexp, prec, d_lengths);
    count_launch();
    if ((rc = check_launch())) return rc;
    if ((rc = acc_scan(a, d_lengths, d_total_bits, st))) return rc;
    if (cudaMemsetAsync(d_payload, 0, (size_t)nb * 128, st) != cudaSuccess) return ZFPX_ECUDA;
    acc_pack_kernel<<<grid, 256, 0, st>>>(a.slots, nb, d_lengths, a.local, a.tile_off,
                                          reinterpret_cast<unsigned long long *>(d_payload));
    count_launch();
    return check_launch();
}

int zfpx_encode_accuracy(const float *d_in, const int64_t n[3], const int64_t stride[3], double tolerance,
                         uint16_t *d_lengths, uint8_t *d_payload, size_t cap, uint64_t *d_total_bits,
                         void *d_work, size_t work_bytes, void *stream)
{
    if (!(tolerance > 0.0) || !(tolerance < HUGE_VAL)) return ZFPX_EINVAL;
    int e = 0;
    (void)frexp(tolerance, &e);                         // floor(log2 tolerance) = e - 1
    return encode_variable(d_in, n, stride, e - 1, 0, d_lengths, d_payload, cap, d_total_bits, d_work,
                           work_bytes, stream);
}

int zfpx_encode_precision(const float *d_in, const int64_t n[3], const int64_t stride[3], int precision,
                          uint16_t *d_lengths, uint8_t *d_payload, size_t cap, uint64_t *d_total_bits,
                          void *d_work, size_t work_bytes, void *stream)
{
    if (precision < 1 || precision > 32) return ZFPX_EINVAL;
    return encode_variable(d_in, n, stride, 0, precision, d_lengths, d_payload, cap, d_total_bits, d_work,
                           work_bytes, stream);
}

int zfpx_decode_accuracy(const uint16_t *d_lengths, const uint8_t *d_payload, size_t len, const int64_t n[3],
                         const int64_t stride[3], float *d_out, void *d_work, size_t work_bytes, void *stream)
{
    if (!d_lengths || !d_payload || !n || !stride || !d_out || !d_work) return ZFPX_EINVAL;
    for (int a = 0; a < 3; a++) if (n[a] < 1 || stride[a] < 0) return ZFPX_EINVAL;
    if (!aligned(d_payload, 8) || !aligned(d_work, 256) || !aligned(d_lengths, 2)) return ZFPX_EINVAL;
    const int64_t nb = acc_blocks(n);
    if (work_bytes < acc_work_bytes(nb)) return ZFPX_ESIZE;
    cudaStream_t st = (cudaStream_t)stream;
    const AccWork a = acc_carve(d_work, nb);
    int rc = acc_scan(a, d_lengths, a.total, st);
    if (rc) return rc;
    acc_unpack_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(
        reinterpret_cast<const uint64_t *>(d_payload), (int64_t)(len / 8), nb, d_lengths, a.local, a.tile_off, a.slots);
    count_launch();
    if ((rc = check_launch())) return rc;
    return zfpx_decode(3, 16, reinterpret_cast<const uint8_t *>(a.slots), (size_t)nb * 128, n, stride, d_out, stream);
}

}  // extern "C"

// ============================================================================
// The accuracy mode on a transposition plan: every message is coded as in the
// raw accuracy mode (its box's 3-D blocks, edge-replicated inside the box);
// messages become variable in size, so the exchange is an all-to-all-v: the
// per-message word counts go first, then the payloads.  On one GPU both are
// device-local copies.  A message's payload starts on a 64-bit word.
namespace zfpx {
std::vector<int64_t> layout_offsets(const zfpx_plan_s *p, int rate, int layout, int64_t *total);
namespace {

// One message as the accuracy kernels see it (send-order index m).
struct AccMsg {
    int64_t gb0;        // first block in the send-order block list (and lengths array)
    int64_t gr0;        // first block in the receive-order block list
    int64_t nb;         // blocks
    int64_t slot_send;  // byte offset of its rate-16 slots in the send layout
    int64_t slot_recv;  // byte offset of its rate-16 slots in the receive layout
};

struct PlanAcc {
    const AccMsg *msgs;       // M, send order
    const int32_t *rorder;    // M: send index of the message at receive position r
    const int64_t *rgb0;      // M: gr0 of the message at receive position r (ascending)
    int64_t *pay_send;        // M: payload word offset in the send buffer
    int64_t *pay_recv;        // M: payload word offset in the receive buffer
    int M;
    int64_t G;                // blocks in all messages
};

__device__ __forceinline__ int last_le(const int64_t *a, const AccMsg *m, int M, int64_t g, bool by_msgs)
{
    int lo = 0, hi = M - 1;                  // last index whose start <= g (starts ascending)
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int64_t s = by_msgs ? m[mid].gb0 : a[mid];
        if (s <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ uint64_t goff(const uint32_t *local, const uint64_t *tile_off, int64_t G,
                                         const uint64_t *total, int64_t g)
{
    return g < G ? tile_off[g / kTile] + local[g] : *total;
}

__global__ void __launch_bounds__(256) pacc_lengths_kernel(PlanAcc P, const uint8_t *__restrict__ slots, int minexp,
                                                           int prec, uint16_t *__restrict__ lengths)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= P.G) return;
    const int m = last_le(nullptr, P.msgs, P.M, g, true);
    const AccMsg &a = P.msgs[m];
    const uint64_t *w = reinterpret_cast<const uint64_t *>(slots + a.slot_send) + (g - a.gb0) * kSlotWords;
    const uint64_t head = __ldg(w);
    int L = 1;
    if (head & 1ull) {
        const int kmin = acc_kmin((int)((head >> 1) & 0xffu) - 127, minexp, prec);
        SlotReader rd{w, 9};
        int n = 0, R = kCutBits - 9;
#pragma unroll 1
        for (int k = 31; k >= kmin && R > 0; k--) (void)decode_plane<64>(rd, n, R);
        L = kCutBits - R;
    }
    lengths[g] = (uint16_t)L;
}

// Word counts and payload offsets of the messages (one thread: M is a few
// thousand at most).  With `send` the counts come from the block scan of the
// send-order lengths and are written to words[]; otherwise words[] is input.
__global__ void pacc_messages_kernel(PlanAcc P, const uint32_t *__restrict__ local,
                                     const uint64_t *__restrict__ tile_off, const uint64_t *__restrict__ total,
                                     uint64_t *__restrict__ words, int send)
{
    if (threadIdx.x || blockIdx.x) return;
    int64_t o = 0;
    for (int m = 0; m < P.M; m++) {
        if (send) {
            const AccMsg &a = P.msgs[m];
            const uint64_t bits = goff(local, tile_off, P.G, total, a.gb0 + a.nb) - goff(local, tile_off, P.G, total, a.gb0);
            words[m] = (bits + 63) / 64;
        }
        P.pay_send[m] = o;
        o += (int64_t)words[m];
    }
    o = 0;
    for (int r = 0; r < P.M; r++) {
        const int m = P.rorder[r];
        P.pay_recv[m] = o;
        o += (int64_t)words[m];
    }
}

__global__ void __launch_bounds__(256) pacc_pack_kernel(PlanAcc P, const uint8_t *__restrict__ slots,
                                                        const uint16_t *__restrict__ lengths,
                                                        const uint32_t *__restrict__ local,
                                                        const uint64_t *__restrict__ tile_off,
                                                        const uint64_t *__restrict__ total,
                                                        unsigned long long *__restrict__ payload)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= P.G) return;
    const int m = last_le(nullptr, P.msgs, P.M, g, true);
    const AccMsg &a = P.msgs[m];
    const uint64_t off = (uint64_t)P.pay_send[m] * 64 +
                         (goff(local, tile_off, P.G, total, g) - goff(local, tile_off, P.G, total, a.gb0));
    const int L = lengths[g];
    const uint64_t *w = reinterpret_cast<const uint64_t *>(slots + a.slot_send) + (g - a.gb0) * kSlotWords;
    const int sh = (int)(off & 63);
    unsigned long long *d = payload + (off >> 6);
#pragma unroll 1
    for (int i = 0; 64 * i < L; i++) {
        uint64_t v = __ldg(w + i);
        const int rem = L - 64 * i;
        if (rem < 64) v &= (1ull << rem) - 1ull;
        if (!v) continue;
        atomicOr(d + i, (unsigned long long)(v << sh));
        if (sh && (v >> (64 - sh))) atomicOr(d + i + 1, (unsigned long long)(v >> (64 - sh)));
    }
}

// The all-to-all-v on one GPU: CTA m moves message m's payload words and its
// block bit counts from the send to the receive buffers.
__global__ void __launch_bounds__(256) pacc_exchange_kernel(PlanAcc P, const uint64_t *__restrict__ words,
                                                            const uint64_t *__restrict__ pay_in,
                                                            uint64_t *__restrict__ pay_out,
                                                            const uint16_t *__restrict__ len_in,
                                                            uint16_t *__restrict__ len_out, int64_t cap_words)
{
    const int m = blockIdx.x;
    const AccMsg a = P.msgs[m];
    // counts that would run past either buffer are cut there
    const int64_t nw = min((int64_t)min(words[m], (uint64_t)cap_words),
                           cap_words - max(P.pay_send[m], P.pay_recv[m]));
    const uint64_t *s = pay_in + P.pay_send[m];
    uint64_t *d = pay_out + P.pay_recv[m];
    for (int64_t i = threadIdx.x; i < nw; i += blockDim.x) d[i] = __ldg(s + i);
    for (int64_t i = threadIdx.x; i < a.nb; i += blockDim.x) len_out[a.gr0 + i] = len_in[a.gb0 + i];
}

__global__ void __launch_bounds__(256) pacc_unpack_kernel(PlanAcc P, const uint64_t *__restrict__ payload, int64_t pwords,
                                                          const uint16_t *__restrict__ lengths,
                                                          const uint32_t *__restrict__ local,
                                                          const uint64_t *__restrict__ tile_off,
                                                          const uint64_t *__restrict__ total, uint8_t *__restrict__ slots)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;     // receive-order block
    if (g >= P.G) return;
    const int r = last_le(P.rgb0, nullptr, P.M, g, false);
    const int m = P.rorder[r];
    const AccMsg &a = P.msgs[m];
    const uint64_t off = (uint64_t)P.pay_recv[m] * 64 +
                         (goff(local, tile_off, P.G, total, g) - goff(local, tile_off, P.G, total, a.gr0));
    const int L = min((int)lengths[g], kCutBits);
    const int sh = (int)(off & 63);
    const int64_t j0 = (int64_t)(off >> 6);
    uint64_t *s = reinterpret_cast<uint64_t *>(slots + a.slot_recv) + (g - a.gr0) * kSlotWords;
#pragma unroll
    for (int i = 0; i < kSlotWords; i++) {
        uint64_t v = 0;
        const int rem = L - 64 * i;
        if (rem > 0) {
            const int64_t j = j0 + i;
            const uint64_t lo = j < pwords ? __ldg(payload + j) : 0ull;
            const uint64_t hi = (sh && j + 1 < pwords) ? __ldg(payload + j + 1) : 0ull;
            v = sh ? (lo >> sh) | (hi << (64 - sh)) : lo;
            if (rem < 64) v &= (1ull << rem) - 1ull;
        }
        s[i] = v;
    }
}

struct PlanAccWork {
    PlanAcc P;
    uint8_t *slots;
    AccWork scan;             // local / totals / tile_off / total for G blocks
    size_t bytes;
};

int64_t plan_blocks(const zfpx_plan_s *p, std::vector<AccMsg> *msgs, std::vector<int32_t> *rorder,
                    std::vector<int64_t> *rgb0)
{
    const size_t M = p->msgs.size();
    auto c4 = [](int64_t v) { return (v + 3) / 4; };
    std::vector<int64_t> nb(M);
    int64_t G = 0;
    for (size_t i = 0; i < M; i++) {
        const HostMsg &m = p->msgs[i];
        nb[i] = c4(m.nx) * c4(m.ny) * c4(m.nz);
        G += nb[i];
    }
    if (!msgs) return G;
    const std::vector<int64_t> so = layout_offsets(p, 16, ZFPX_LAYOUT_SEND, nullptr);
    const std::vector<int64_t> ro = layout_offsets(p, 16, ZFPX_LAYOUT_RECV, nullptr);
    std::vector<int32_t> ord(M);
    for (size_t i = 0; i < M; i++) ord[i] = (int32_t)i;
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) {
        const HostMsg &x = p->msgs[a], &y = p->msgs[b];
        return x.dst != y.dst ? x.dst < y.dst : x.src_peer < y.src_peer;
    });
    msgs->assign(M, AccMsg{});
    rorder->assign(ord.begin(), ord.end());
    rgb0->assign(M, 0);
    int64_t g = 0;
    for (size_t i = 0; i < M; i++) {
        (*msgs)[i].gb0 = g; (*msgs)[i].nb = nb[i];
        (*msgs)[i].slot_send = so[i]; (*msgs)[i].slot_recv = ro[i];
        g += nb[i];
    }
    g = 0;
    for (size_t r = 0; r < M; r++) {
        (*msgs)[ord[r]].gr0 = g;
        (*rgb0)[r] = g;
        g += nb[ord[r]];
    }
    return G;
}

size_t plan_acc_bytes(const zfpx_plan_s *p, int64_t G)
{
    const size_t M = p->msgs.size();
    return align256((size_t)buffer_bytes(p, 16)) + acc_work_bytes(G) - align256((size_t)G * 128) +
           align256(M * sizeof(AccMsg)) + align256(M * 4) + 3 * align256(M * 8);
}

// Carves the scratch and uploads the message tables (pageable copies: the
// host vectors have been read when the call returns).
int plan_acc_setup(const zfpx_plan_s *p, void *work, size_t work_bytes, cudaStream_t st, PlanAccWork *w)
{
    std::vector<AccMsg> msgs;
    std::vector<int32_t> rorder;
    std::vector<int64_t> rgb0;
    const int64_t G = plan_blocks(p, &msgs, &rorder, &rgb0);
    const size_t M = msgs.size();
    if (work_bytes < plan_acc_bytes(p, G)) return ZFPX_ESIZE;
    char *c = static_cast<char *>(work);
    w->slots = reinterpret_cast<uint8_t *>(c); c += align256((size_t)buffer_bytes(p, 16));
    w->scan.nblocks = G;
    w->scan.ntiles = (G + kTile - 1) / kTile;
    w->scan.slots = nullptr;
    w->scan.local = reinterpret_cast<uint32_t *>(c); c += align256((size_t)G * 4);
    w->scan.totals = reinterpret_cast<uint64_t *>(c); c += align256((size_t)w->scan.ntiles * 8);
    w->scan.tile_off = reinterpret_cast<uint64_t *>(c); c += align256((size_t)w->scan.ntiles * 8);
    w->scan.total = reinterpret_cast<uint64_t *>(c); c += 256;
    AccMsg *dm = reinterpret_cast<AccMsg *>(c); c += align256(M * sizeof(AccMsg));
    int32_t *dr = reinterpret_cast<int32_t *>(c); c += align256(M * 4);
    int64_t *dg = reinterpret_cast<int64_t *>(c); c += align256(M * 8);
    w->P.pay_send = reinterpret_cast<int64_t *>(c); c += align256(M * 8);
    w->P.pay_recv = reinterpret_cast<int64_t *>(c); c += align256(M * 8);
    w->P.msgs = dm; w->P.rorder = dr; w->P.rgb0 = dg; w->P.M = (int)M; w->P.G = G;
    if (M && (cudaMemcpyAsync(dm, msgs.data(), M * sizeof(AccMsg), cudaMemcpyHostToDevice, st) != cudaSuccess ||
              cudaMemcpyAsync(dr, rorder.data(), M * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
              cudaMemcpyAsync(dg, rgb0.data(), M * 8, cudaMemcpyHostToDevice, st) != cudaSuccess))
        return ZFPX_ECUDA;
    return ZFPX_OK;
}

unsigned grid256(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + 255) / 256); }

}  // namespace
}  // namespace zfpx

extern "C" {

size_t zfpx_plan_accuracy_blocks(zfpx_plan p)
{
    return p ? (size_t)plan_blocks(p, nullptr, nullptr, nullptr) : 0;
}

size_t zfpx_plan_accuracy_workspace_bytes(zfpx_plan p)
{
    if (!p || p->dims != 3) return 0;
    return plan_acc_bytes(p, plan_blocks(p, nullptr, nullptr, nullptr));
}

static int pack_compress_variable(zfpx_plan p, int minexp, int prec, const float *d_src, uint16_t *d_lengths,
                                  uint8_t *d_payload, size_t cap, uint64_t *d_msg_words, void *d_work,
                                  size_t work_bytes, void *stream)
{
    if (!p || !d_src || !d_lengths || !d_payload || !d_msg_words || !d_work || p->dims != 3) return ZFPX_EINVAL;
    if (!aligned(d_payload, 8) || !aligned(d_work, 256) || !aligned(d_lengths, 2) || !aligned(d_msg_words, 8))
        return ZFPX_EINVAL;
    const int64_t G = plan_blocks(p, nullptr, nullptr, nullptr);
    if (cap < (size_t)G * 128) return ZFPX_ESIZE;
    cudaStream_t st = (cudaStream_t)stream;
    PlanAccWork w;
    int rc = plan_acc_setup(p, d_work, work_bytes, st, &w);
    if (rc) return rc;
    if (G == 0)                                    // every message empty
        return cudaMemsetAsync(d_msg_words, 0, p->msgs.size() * 8, st) == cudaSuccess ? ZFPX_OK : ZFPX_ECUDA;
    if ((rc = zfpx_pack_compress(p, 16, d_src, w.slots, (size_t)buffer_bytes(p, 16), ZFPX_LAYOUT_SEND, stream)))
        return rc;
    pacc_lengths_kernel<<<grid256(G), 256, 0, st>>>(w.P, w.slots, minexp, prec, d_lengths);
    count_launch();
    if ((rc = check_launch()) || (rc = acc_scan(w.scan, d_lengths, w.scan.total, st))) return rc;
    pacc_messages_kernel<<<1, 32, 0, st>>>(w.P, w.scan.local, w.scan.tile_off, w.scan.total, d_msg_words, 1);
    count_launch();
    if (cudaMemsetAsync(d_payload, 0, (size_t)G * 128, st) != cudaSuccess) return ZFPX_ECUDA;
    pacc_pack_kernel<<<grid256(G), 256, 0, st>>>(w.P, w.slots, d_lengths, w.scan.local, w.scan.tile_off,
                                                 w.scan.total, reinterpret_cast<unsigned long long *>(d_payload));
    count_launch();
    return check_launch();
}

int zfpx_pack_compress_accuracy(zfpx_plan p, double tolerance, const float *d_src, uint16_t *d_lengths,
                                uint8_t *d_payload, size_t cap, uint64_t *d_msg_words, void *d_work,
                                size_t work_bytes, void *stream)
{
    if (!(tolerance > 0.0) || !(tolerance < HUGE_VAL)) return ZFPX_EINVAL;
    int e = 0;
    (void)frexp(tolerance, &e);
    return pack_compress_variable(p, e - 1, 0, d_src, d_lengths, d_payload, cap, d_msg_words, d_work, work_bytes,
                                  stream);
}

int zfpx_pack_compress_precision(zfpx_plan p, int precision, const float *d_src, uint16_t *d_lengths,
                                 uint8_t *d_payload, size_t cap, uint64_t *d_msg_words, void *d_work,
                                 size_t work_bytes, void *stream)
{
    if (precision < 1 || precision > 32) return ZFPX_EINVAL;
    return pack_compress_variable(p, 0, precision, d_src, d_lengths, d_payload, cap, d_msg_words, d_work,
                                  work_bytes, stream);
}

int zfpx_exchange_accuracy(zfpx_plan p, const uint64_t *d_msg_words, const uint16_t *d_len_send,
                           const uint8_t *d_pay_send, uint16_t *d_len_recv, uint8_t *d_pay_recv, size_t cap,
                           void *d_work, size_t work_bytes, void *stream)
{
    if (!p || !d_msg_words || !d_len_send || !d_pay_send || !d_len_recv || !d_pay_recv || !d_work || p->dims != 3)
        return ZFPX_EINVAL;
    if (!aligned(d_pay_send, 8) || !aligned(d_pay_recv, 8) || !aligned(d_work, 256)) return ZFPX_EINVAL;
    const int64_t G = plan_blocks(p, nullptr, nullptr, nullptr);
    if (cap < (size_t)G * 128) return ZFPX_ESIZE;
    cudaStream_t st = (cudaStream_t)stream;
    PlanAccWork w;
    int rc = plan_acc_setup(p, d_work, work_bytes, st, &w);
    if (rc || w.P.M == 0) return rc;
    pacc_messages_kernel<<<1, 32, 0, st>>>(w.P, nullptr, nullptr, nullptr, const_cast<uint64_t *>(d_msg_words), 0);
    count_launch();
    pacc_exchange_kernel<<<(unsigned)w.P.M, 256, 0, st>>>(w.P, d_msg_words,
                                                           reinterpret_cast<const uint64_t *>(d_pay_send),
                                                           reinterpret_cast<uint64_t *>(d_pay_recv), d_len_send,
                                                           d_len_recv, (int64_t)(cap / 8));
    count_launch();
    return check_launch();
}

int zfpx_decompress_unpack_accuracy(zfpx_plan p, const uint64_t *d_msg_words, const uint16_t *d_len_recv,
                                    const uint8_t *d_pay_recv, size_t len, float *d_dst, void *d_work,
                                    size_t work_bytes, void *stream)
{
    if (!p || !d_msg_words || !d_len_recv || !d_pay_recv || !d_dst || !d_work || p->dims != 3) return ZFPX_EINVAL;
    if (!aligned(d_pay_recv, 8) || !aligned(d_work, 256) || !aligned(d_len_recv, 2)) return ZFPX_EINVAL;
    const int64_t G = plan_blocks(p, nullptr, nullptr, nullptr);
    cudaStream_t st = (cudaStream_t)stream;
    PlanAccWork w;
    int rc = plan_acc_setup(p, d_work, work_bytes, st, &w);
    if (rc || G == 0) return rc;
    pacc_messages_kernel<<<1, 32, 0, st>>>(w.P, nullptr, nullptr, nullptr, const_cast<uint64_t *>(d_msg_words), 0);
    count_launch();
    if ((rc = acc_scan(w.scan, d_len_recv, w.scan.total, st))) return rc;
    pacc_unpack_kernel<<<grid256(G), 256, 0, st>>>(w.P, reinterpret_cast<const uint64_t *>(d_pay_recv),
                                                   (int64_t)(len / 8), d_len_recv, w.scan.local, w.scan.tile_off,
                                                   w.scan.total, w.slots);
    count_launch();
    if ((rc = check_launch())) return rc;
    return zfpx_decompress_unpack(p, 16, w.slots, (size_t)buffer_bytes(p, 16), d_dst, ZFPX_LAYOUT_RECV, stream);
}

}  // extern "C"
