// The 3-D block encoder of the codec kernels (paper Sec. II-C; Sec. IV-B),
// one lane per block, written so that the lanes of a warp never take
// different paths: every loop runs while any lane still has work, and a lane
// without work runs the same instructions on values that change nothing.
// The readings are those of encode_block3 in zfpx_block.cuh, which this
// produces bit for bit; all stream arithmetic is on 32-bit words.
//
// Layout per warp (shared memory, each lane in its own column, so the lanes'
// accesses never share a bank):
//   tile   [RATE * 2 + 4][32] 32-bit words, word w of lane l at w * 32 + l:
//          the lane's stream (2 RATE words, then four slack words that catch
//          the bits of a plane running past the budget).  Zero on entry;
//          store_stream() copies the stream out and zeroes the tile again.
//   planes [32][32] 64-bit: bit plane k of lane l at k * 32 + l; pass 1
//          reuses the slots of planes already read for its list of planes
//          with newly significant coefficients (entry f at slot 31 - f).
//   spos   [32][32] uint16: for list entry f, the stream position of the
//          plane's first group bit plus one.
//
// The stream of a block is its header (a 1 bit and e_max + 127 in 8 bits),
// then the bit planes from the top.  Plane k, with n coefficients already
// significant, holds n verbatim bits, then (n < 64) a group bit, which is 1
// if bits n .. 63 of the plane hold ones, c of them with the highest at h;
// then, coefficient by coefficient from n, a value bit for each coefficient
// up to h, each one followed by a group bit (1 while more ones follow), the
// one at coefficient 63 implied (neither bit).  So the plane takes n + 1 bits
// without new ones and n + 1 + (h - n + 1) + c bits with them (two fewer when
// h = 63); the stream is cut at exactly 64 RATE bits.
//
// Phase A walks the planes while n < 64: it writes the verbatim bits and the
// first group bit, leaves the group-tested part as zeros and lists the plane
// if it has new ones.  Phase B: once n = 64 every later plane is its 64 bits
// verbatim, so the rest of the stream is the remaining planes back to back,
// one funnel shift per 32-bit word.  Pass 2 walks the list one new
// coefficient per step: the t-th one of a listed plane, at coefficient p,
// has its value bit at (listed position) + p + t, its group bit right after;
// positions only grow, so the first one past the budget ends a lane's pass.
#pragma once
#include <cstdint>

#include "zfpx_block.cuh"

namespace zfpx {
namespace enc3 {

using namespace blk;

// 32-bit tile words per lane at `rate`
template <int RATE>
constexpr int kWords = 2 * RATE + 4;

// One warp's shared memory: tile (kWords<RATE> * 32 words, or more), planes
// (32 * 32), spos (32 * 32).
struct View {
    uint32_t *tile;
    uint64_t *planes;
    uint16_t *spos;
};

// Storage of one warp at `rate`.
template <int RATE>
struct Shared {
    uint32_t tile[kWords<RATE> * 32];
    uint64_t planes[32 * 32];
    uint16_t spos[32 * 32];
    __device__ __forceinline__ View view() { return View{tile, planes, spos}; }
};

__device__ __forceinline__ uint32_t shl(uint32_t a, uint32_t s)
{
    uint32_t r;
    asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(s));   // s >= 32 gives 0
    return r;
}
__device__ __forceinline__ uint32_t shr(uint32_t a, uint32_t s)
{
    uint32_t r;
    asm("shr.b32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(s));   // s >= 32 gives 0
    return r;
}
// high word of (hi:lo) << s, 0 <= s < 32
__device__ __forceinline__ uint32_t funnel(uint32_t lo, uint32_t hi, uint32_t s) { return __funnelshift_l(lo, hi, s); }
__device__ __forceinline__ void red_or(uint32_t *p, uint32_t v) { atomicOr(p, v); }

template <int RATE>
__device__ __forceinline__ void encode(const float (&x)[64], bool valid, const View &sh, int lane)
{
    constexpr int kSeq[64] = ZFPX_SEQ3;
    constexpr int END = 64 * RATE;
    constexpr unsigned FULL = 0xffffffffu;
    uint32_t *tile = sh.tile + lane;                   // word w at tile[32 w]
    uint64_t *planes = sh.planes + lane;               // plane k at planes[32 k]
    uint16_t *spos = sh.spos + lane;
    uint32_t amax = 0;
#pragma unroll
    for (int i = 0; i < 64; i++) {
        const uint32_t a = f2u(x[i]) & 0x7fffffffu;
        amax = a > amax ? a : amax;
    }
    // E = e_max + 126; a block whose maximum is zero, below 2^-127 or not
    // finite is a single 0 bit (the tile is already zero)
    const int E = (int)(amax >> 23);
    bool act = valid && amax >= 0x00400000u && E != 255;
    const QuantScale qs(act ? E : 127);
    int32_t q[64];
#pragma unroll
    for (int i = 0; i < 64; i++) q[i] = qs(x[i]);
    xform3_fwd(q);
    uint32_t lo[32], hi[32];
#pragma unroll
    for (int t = 0; t < 32; t++) {
        lo[t] = to_negabinary(q[kSeq[t]]);
        hi[t] = to_negabinary(q[kSeq[32 + t]]);
    }
    // planes kLow .. 31 finished now, 0 .. kLow - 1 half-transposed until a
    // lane needs them (the budget rarely reaches below plane 16 at rate 8,
    // plane 8 at rate 16)
    constexpr int kLow = RATE == 8 ? 16 : 8;
    uint32_t *p32 = reinterpret_cast<uint32_t *>(planes);   // half h of plane k at p32[64 k + h]
#pragma unroll 1
    for (int half = 0; half < 2; half++) {
        if (half) {
#pragma unroll
            for (int t = 0; t < 32; t++) lo[t] = hi[t];
        }
        transpose32_part1<kLow>(lo);
#pragma unroll
        for (int k = 0; k < 32; k++) p32[64 * k + half] = lo[k];
    }
    bool low_done = false;
    auto finish_low = [&]() {
        uint32_t a[32], b[32];
#pragma unroll
        for (int i = 0; i < kLow; i++) {
            a[i] = p32[64 * i];
            b[i] = p32[64 * i + 1];
        }
        transpose32_part2<kLow>(a);
        transpose32_part2<kLow>(b);
#pragma unroll
        for (int i = 0; i < kLow; i++) planes[32 * i] = ((uint64_t)b[i] << 32) | a[i];
        low_done = true;
    };
    tile[0] = act ? 1u | ((uint32_t)(E + 1) << 1) : 0u;

    // ---- phase A: planes while n < 64
    int n = 0, pos = 9, nf = 0, kB = -1;
    uint32_t lml = 0, lmh = 0;                         // low n bits
    uint32_t gml = 1, gmh = 0;                         // bit n
    bool pa = act;                                      // in phase A
#pragma unroll 1
    for (int k = 31; k >= 0; k--) {
        if (!__any_sync(FULL, pa)) break;
        if (k == kLow - 1) finish_low();
        const uint64_t X = planes[32 * k];
        const uint32_t xl = (uint32_t)X, xh = (uint32_t)(X >> 32);
        const uint32_t yl = xl & ~lml, yh = xh & ~lmh;
        const bool has = pa && (yl | yh) != 0;
        const uint32_t hm = has ? 0xffffffffu : 0u, am = pa ? 0xffffffffu : 0u;
        const uint32_t vl = ((xl & lml) | (gml & hm)) & am, vh = ((xh & lmh) | (gmh & hm)) & am;
        const uint32_t w = (uint32_t)(pa ? pos : 0) >> 5, s = (uint32_t)pos & 31u;
        red_or(tile + 32 * w, vl << s);
        red_or(tile + 32 * (w + 1), funnel(vl, vh, s));
        red_or(tile + 32 * (w + 2), funnel(vh, 0u, s));
        const int h = yh ? 32 + highest_set32(yh) : highest_set32(yl | 1u);
        const int c = popc32(yl) + popc32(yh);
        if (has) {
            planes[32 * (31 - nf)] = ((uint64_t)yh << 32) | yl;
            spos[32 * nf] = (uint16_t)(pos + 1);
            nf++;
            // n = h + 1: low mask (2 << h) - 1 and bit n, as 32-bit halves
            lml = shl(2u, (uint32_t)h) - 1u;                             // all ones from h = 31
            lmh = h >= 32 ? shl(2u, (uint32_t)(h - 32)) - 1u : 0u;
            gml = h < 31 ? 2u << h : 0u;
            gmh = h >= 31 && h < 63 ? 1u << (h - 31) : 0u;
            n = h + 1;
        }
        pos += pa ? (has ? h + c + (h < 63 ? 2 : 0) : n + 1) : 0;
        const bool full = pa && n == 64 && pos < END;
        kB = full ? k - 1 : kB;
        pa = pa && n < 64 && pos < END;
    }

    // ---- phase B: planes kB, kB - 1, ... verbatim from bit pB = pos
    bool pb = act && n == 64 && pos < END;
    {
        const uint32_t s = (uint32_t)pos & 31u;
        const int w0 = pos >> 5;
        // the lowest plane a lane reads here: planes kB - m for the m with
        // w0 + 2 m < 2 RATE
        const int need = kB - ((2 * RATE - w0 + 1) / 2 - 1);
        if (!low_done && __any_sync(FULL, pb && need < kLow)) finish_low();
        uint32_t prev = 0;
#pragma unroll 1
        for (int m = 0;; m++) {
            const int wa = w0 + 2 * m;                 // words wa (from the previous plane's high half) and wa + 1
            const bool live = pb && wa < 2 * RATE;
            if (!__any_sync(FULL, live)) break;
            const int kp = kB - m;
            const uint64_t X = live && kp >= 0 ? planes[32 * kp] : 0ull;
            const uint32_t xl = (uint32_t)X, xh = (uint32_t)(X >> 32);
            if (live) {
                if (m == 0) red_or(tile + 32 * wa, xl << s);
                else tile[32 * wa] = funnel(prev, xl, s);
                tile[32 * (wa + 1)] = funnel(xl, xh, s);
            }
            prev = xh;
        }
    }

    // ---- pass 2: the listed planes' new coefficients
    int f = 0, ap = 0, t = 0;
    uint32_t rl = 0, rh = 0;
#pragma unroll 1
    for (;;) {
        const bool need = (rl | rh) == 0 && f < nf;
        if (!__any_sync(FULL, need || (rl | rh) != 0)) break;
        if (need) {
            const uint64_t Y = planes[32 * (31 - f)];
            rl = (uint32_t)Y;
            rh = (uint32_t)(Y >> 32);
            ap = spos[32 * f];
            t = 0;
            f++;
        }
        const bool live = (rl | rh) != 0;
        const bool inlo = rl != 0;
        const int p = inlo ? lowest_set32(rl) : 32 + lowest_set32(rh | 0x80000000u);
        if (inlo) rl &= rl - 1u;
        else rh &= rh - 1u;
        const int A = ap + p + t;
        t++;
        const bool ok = live && A < END;
        if (live && A >= END) {                        // this one and every later one past the budget
            rl = rh = 0;
            f = nf;
        }
        // value bit (coefficient 63's is implied) and the group bit after it,
        // which may land in the next word or a slack word
        const uint32_t b = ok ? (uint32_t)(p != 63) | ((rl | rh) != 0 ? 2u : 0u) : 0u;
        const uint32_t w = (uint32_t)(ok ? A : 0) >> 5, s = (uint32_t)A & 31u;
        red_or(tile + 32 * w, b << s);
        red_or(tile + 32 * (w + 1), shr(b, 32u - s));
    }
}

// Copies this lane's 2 RATE stream words to dst (16-byte aligned, the
// block's slot) with 16-byte stores when `valid`, and zeroes the lane's tile
// column for the next block.  Every lane of the warp calls it.
template <int RATE>
__device__ __forceinline__ void store_stream(const View &sh, int lane, bool valid, uint8_t *dst)
{
    uint32_t *tile = sh.tile + lane;
#pragma unroll
    for (int i = 0; i < RATE / 2; i++) {
        const uint4 v = make_uint4(tile[32 * (4 * i)], tile[32 * (4 * i + 1)], tile[32 * (4 * i + 2)],
                                   tile[32 * (4 * i + 3)]);
        if (valid) reinterpret_cast<uint4 *>(dst)[i] = v;
    }
#pragma unroll
    for (int w = 0; w < kWords<RATE>; w++) tile[32 * w] = 0u;
}

// Zeroes this lane's column of the first `words` tile words.
__device__ __forceinline__ void clear(const View &sh, int lane, int words)
{
    for (int w = 0; w < words; w++) sh.tile[32 * w + lane] = 0u;
}

}  // namespace enc3
}  // namespace zfpx
