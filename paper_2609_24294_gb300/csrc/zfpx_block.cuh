// One ZFP fixed-rate block: encode and decode (paper Sec. II-C; Sec. IV-B).
//
// Readings (identical to the CPU oracle, stated in include/zfpx.h):
//   e_max = frexp exponent of max|x|; a block whose e_max + 127 <= 0 (max|x|
//   below 2^-127, zero included) or whose max is non-finite is a single 0 bit
//   and zero fill, decoding to +0.0;
//   header = 1 bit, then e_max + 127 in 8 bits, LSB first;
//   q = trunc(x 2^(30 - e_max)); five-step integer lifting with floor halving
//   along x, then y, then z; 3-D coefficients in total-sequency order;
//   negabinary; bit planes 31..0 with group testing, cut at exactly 4^d r
//   bits; truncated bits decode as 0; x = (float)(q 2^(e_max - 30)) with one
//   rounding to nearest even.
//
// The functions are __host__ __device__ so the same block code serves the
// kernels and can be compiled for a CPU.  On the GPU the 64 coefficients of a
// 3-D block sit in registers, their 32 bit planes are built with two 32x32
// bit-matrix transposes, and group testing is one find-first-set per newly
// significant coefficient.
#pragma once

#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define ZFPX_HD __host__ __device__ __forceinline__
#else
#define ZFPX_HD inline
#endif

namespace zfpx {
namespace blk {

// ----------------------------------------------------------------- primitives
ZFPX_HD uint32_t f2u(float x)
{
#ifdef __CUDA_ARCH__
    return __float_as_uint(x);
#else
    uint32_t u; std::memcpy(&u, &x, 4); return u;
#endif
}
ZFPX_HD float u2f(uint32_t u)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float x; std::memcpy(&x, &u, 4); return x;
#endif
}
ZFPX_HD uint32_t byte_perm(uint32_t a, uint32_t b, uint32_t sel)
{
#ifdef __CUDA_ARCH__
    return __byte_perm(a, b, sel);
#else
    const uint64_t v = ((uint64_t)b << 32) | a;
    uint32_t r = 0;
    for (int i = 0; i < 4; i++) r |= (uint32_t)((v >> (8 * ((sel >> (4 * i)) & 7))) & 0xff) << (8 * i);
    return r;
#endif
}
// index of the lowest set bit (x != 0)
ZFPX_HD int lowest_set(uint64_t x)
{
#ifdef __CUDA_ARCH__
    return __ffsll((long long)x) - 1;
#else
    return __builtin_ctzll(x);
#endif
}
ZFPX_HD int lowest_set32(uint32_t x)
{
#ifdef __CUDA_ARCH__
    return __ffs((int)x) - 1;
#else
    return __builtin_ctz(x);
#endif
}
ZFPX_HD int popc32(uint32_t x)
{
#ifdef __CUDA_ARCH__
    return __popc(x);
#else
    return __builtin_popcount(x);
#endif
}
ZFPX_HD int popc64(uint64_t x)
{
#ifdef __CUDA_ARCH__
    return __popcll(x);
#else
    return __builtin_popcountll(x);
#endif
}
// index of the highest set bit (x != 0)
ZFPX_HD int highest_set64(uint64_t x)
{
#ifdef __CUDA_ARCH__
    return 63 - __clzll((long long)x);
#else
    return 63 - __builtin_clzll(x);
#endif
}
ZFPX_HD int highest_set32(uint32_t x)
{
#ifdef __CUDA_ARCH__
    return 31 - __clz((int)x);
#else
    return 31 - __builtin_clz(x);
#endif
}
ZFPX_HD uint64_t low_mask(int n) { return n >= 64 ? ~0ull : ((1ull << n) - 1); }
ZFPX_HD int imin(int a, int b) { return a < b ? a : b; }

// int32 ring arithmetic: wraps like the hardware, without signed overflow.
ZFPX_HD int32_t wadd(int32_t a, int32_t b) { return (int32_t)((uint32_t)a + (uint32_t)b); }
ZFPX_HD int32_t wsub(int32_t a, int32_t b) { return (int32_t)((uint32_t)a - (uint32_t)b); }

// ----------------------------------------------------------------- block float
ZFPX_HD int32_t f2i_rz(float y)
{
#ifdef __CUDA_ARCH__
    return __float2int_rz(y);
#else
    return (int32_t)y;
#endif
}
ZFPX_HD float i2f_rn(int32_t q)
{
#ifdef __CUDA_ARCH__
    return __int2float_rn(q);
#else
    return (float)q;
#endif
}

// q = trunc(x 2^(30 - e_max)), e_max = E - 126 (E: biased exponent of the
// block maximum, 0..254).  The scale 2^(156 - E) is applied as two exact
// power-of-two products, (x * s1) * s2 with s1 = 1 for E >= 29 and 2^64
// below, so every factor is a normal float and no product rounds wherever
// the integer part is non-zero.  No branch, no double precision.
struct QuantScale {
    float s1, s2;
    ZFPX_HD explicit QuantScale(int E)
    {
        const bool small = E < 29;
        s1 = small ? 18446744073709551616.0f : 1.0f;                 // 2^64
        s2 = u2f((uint32_t)((small ? 92 - E : 156 - E) + 127) << 23);
    }
    ZFPX_HD int32_t operator()(float x) const { return f2i_rz((x * s1) * s2); }
};

ZFPX_HD float u2f_rn(uint32_t a)
{
#ifdef __CUDA_ARCH__
    return __uint2float_rn(a);
#else
    return (float)a;
#endif
}

// x = (float)(q 2^(e - 157)) rounded once to nearest even (e = e_max + 127).
// For e >= 31 the scale is a normal float and converting q then scaling is
// exact after the conversion's single rounding.
ZFPX_HD float dequantize_fast(int32_t q, float scale) { return i2f_rn(q) * scale; }
ZFPX_HD float dequant_scale(int e) { return u2f((uint32_t)(e - 30) << 23); }

// The rare headers e < 31, where the result may be subnormal: integer
// rounding at the subnormal quantum 2^-149, no double precision.
ZFPX_HD float dequantize_small(int32_t q, int e)
{
    if (q == 0) return 0.0f;
    const uint32_t sign = q < 0 ? 0x80000000u : 0u;
    const uint32_t a = q < 0 ? 0u - (uint32_t)q : (uint32_t)q;        // |q| <= 2^31
    uint32_t bits;
    if ((uint64_t)a >= (1ull << (31 - e))) {
        // normal result (>= 2^-126): the conversion rounds once, the two
        // power-of-two scalings (2^-64, then 2^(e-93)) are exact
        bits = f2u((u2f_rn(a) * 5.42101086242752217e-20f) * u2f((uint32_t)(e + 34) << 23));
    } else if (e >= 8) {
        bits = a << (e - 8);                                             // exact subnormal
    } else {
        const int d = 8 - e;                                             // a / 2^d to nearest even
        const uint32_t m = a >> d, rem = a & ((1u << d) - 1u), half = 1u << (d - 1);
        bits = m + ((rem > half || (rem == half && (m & 1u))) ? 1u : 0u);
    }
    return u2f(bits | sign);
}

// ----------------------------------------------------------------- transform
// Five lifting steps of the 4-point decorrelating transform (floor halving).
ZFPX_HD void lift_fwd(int32_t &a, int32_t &b, int32_t &c, int32_t &d)
{
    a = wadd(a, d) >> 1; d = wsub(d, a);
    c = wadd(c, b) >> 1; b = wsub(b, c);
    a = wadd(a, c) >> 1; c = wsub(c, a);
    d = wadd(d, b) >> 1; b = wsub(b, d);
    d = wadd(d, b >> 1); b = wsub(b, d >> 1);
}
// The same steps undone in reverse order.
ZFPX_HD void lift_inv(int32_t &a, int32_t &b, int32_t &c, int32_t &d)
{
    b = wadd(b, d >> 1); d = wsub(d, b >> 1);
    b = wadd(b, d); d = wsub(wadd(d, d), b);
    c = wadd(c, a); a = wsub(wadd(a, a), c);
    b = wadd(b, c); c = wsub(wadd(c, c), b);
    d = wadd(d, a); a = wsub(wadd(a, a), d);
}

ZFPX_HD void xform3_fwd(int32_t (&q)[64])
{
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
        for (int j = 0; j < 4; j++)
            lift_fwd(q[16 * k + 4 * j], q[16 * k + 4 * j + 1], q[16 * k + 4 * j + 2], q[16 * k + 4 * j + 3]);
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
        for (int i = 0; i < 4; i++)
            lift_fwd(q[16 * k + i], q[16 * k + i + 4], q[16 * k + i + 8], q[16 * k + i + 12]);
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
        for (int i = 0; i < 4; i++)
            lift_fwd(q[4 * j + i], q[4 * j + i + 16], q[4 * j + i + 32], q[4 * j + i + 48]);
}

ZFPX_HD void xform3_inv(int32_t (&q)[64])
{
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
        for (int i = 0; i < 4; i++)
            lift_inv(q[4 * j + i], q[4 * j + i + 16], q[4 * j + i + 32], q[4 * j + i + 48]);
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
        for (int i = 0; i < 4; i++)
            lift_inv(q[16 * k + i], q[16 * k + i + 4], q[16 * k + i + 8], q[16 * k + i + 12]);
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
        for (int j = 0; j < 4; j++)
            lift_inv(q[16 * k + 4 * j], q[16 * k + 4 * j + 1], q[16 * k + 4 * j + 2], q[16 * k + 4 * j + 3]);
}

ZFPX_HD uint32_t to_negabinary(int32_t q) { return ((uint32_t)q + 0xAAAAAAAAu) ^ 0xAAAAAAAAu; }
ZFPX_HD int32_t from_negabinary(uint32_t u) { return (int32_t)((u ^ 0xAAAAAAAAu) - 0xAAAAAAAAu); }

// Coefficient (i + 4j + 16k) coded at position t: total sequency i+j+k
// ascending, ties by i^2+j^2+k^2, then by the index.
#define ZFPX_SEQ3 {0, 1, 4, 16, 5, 17, 20, 2, 8, 32, 21, 6, 9, 18, 24, 33, 36, 3, 12, 48, 22, 25,   \
                   37, 10, 34, 40, 7, 13, 19, 28, 49, 52, 26, 38, 41, 23, 29, 53, 11, 14, 35, 44, \
                   50, 56, 42, 27, 30, 39, 45, 54, 57, 15, 51, 60, 43, 46, 58, 31, 55, 61, 47,    \
                   59, 62, 63}

// In-place transpose of a 32x32 bit matrix: afterwards bit i of w[k] is
// what bit k of w[i] was.  Off-diagonal blocks are swapped at sizes 16, 8,
// 4, 2, 1; the 16- and 8-bit swaps are single byte permutes.
//
// The five stages swap one bit of the row index with the same bit of the
// column index each, so they commute and may run in any order; a stage of
// size S < L keeps each L-aligned group of words to itself.
// tstage<S, B, E>: the stage of size S on the pairs (i, i + S), B <= i < E.
template <int S, int B, int E>
ZFPX_HD void tstage(uint32_t (&w)[32])
{
#pragma unroll
    for (int i = B; i < E; i++) {
        if (i & S) continue;
        const uint32_t a = w[i], b = w[i + S];
        if (S == 16) {
            w[i] = byte_perm(a, b, 0x5410);
            w[i + S] = byte_perm(a, b, 0x7632);
        } else if (S == 8) {
            w[i] = byte_perm(a, b, 0x6240);
            w[i + S] = byte_perm(a, b, 0x7351);
        } else {
            constexpr uint32_t m = S == 4 ? 0x0F0F0F0Fu : S == 2 ? 0x33333333u : 0x55555555u;
            const uint32_t t = ((a >> S) ^ b) & m;
            w[i + S] = b ^ t;
            w[i] = a ^ (t << S);
        }
    }
}

ZFPX_HD void transpose32(uint32_t (&w)[32])
{
    tstage<16, 0, 32>(w);
    tstage<8, 0, 32>(w);
    tstage<4, 0, 32>(w);
    tstage<2, 0, 32>(w);
    tstage<1, 0, 32>(w);
}

// The transpose in two parts, for coding planes from the top: part 1
// finishes output words L..31 (L = 8 or 16) and leaves words 0..L-1 halfway;
// part 2 finishes those.
template <int L>
ZFPX_HD void transpose32_part1(uint32_t (&w)[32])
{
    tstage<16, 0, 32>(w);
    if (L == 8) tstage<8, 0, 32>(w);
    else tstage<8, 16, 32>(w);
    tstage<4, L, 32>(w);
    tstage<2, L, 32>(w);
    tstage<1, L, 32>(w);
}
template <int L>
ZFPX_HD void transpose32_part2(uint32_t (&w)[32])
{
    if (L == 16) tstage<8, 0, 16>(w);
    tstage<4, 0, L>(w);
    tstage<2, 0, L>(w);
    tstage<1, 0, L>(w);
}

// The transpose of a matrix whose words 0..L-1 are zero (L = 8 or 16): the
// stages smaller than L only touch words L..31.
template <int L>
ZFPX_HD void transpose32_zero_low(uint32_t (&w)[32])
{
#pragma unroll
    for (int i = 0; i < L; i++) w[i] = 0u;
    if (L == 16) tstage<8, 16, 32>(w);
    tstage<4, L, 32>(w);
    tstage<2, L, 32>(w);
    tstage<1, L, 32>(w);
    if (L == 8) tstage<8, 0, 32>(w);
    tstage<16, 0, 32>(w);
}

// ----------------------------------------------------------------- coder
// Group-tested coding of one bit plane X of S coefficients, n of which are
// already significant, spending at most R bits.  Writer: put(bits, len),
// 1 <= len <= 64, bits < 2^len.
template <int S, class Writer>
ZFPX_HD void code_plane(Writer &wr, uint64_t X, int &n, int &R)
{
    const int m = imin(n, R);
    if (m > 0) { wr.put(X & low_mask(m), m); R -= m; }
    while (R > 0 && n < S) {
        const uint64_t rest = X >> n;
        if (rest == 0) { wr.put(0ull, 1); R -= 1; break; }
        const int p = lowest_set(rest);              // zeros before the next one
        int len;
        uint64_t pat;
        if (n + p == S - 1) { len = p + 1; pat = 1ull; }                  // last one implied
        else { len = p + 2; pat = 1ull | (1ull << (p + 1)); }
        if (len > R) { wr.put(pat & low_mask(R), R); R = 0; break; }
        wr.put(pat, len);
        R -= len;
        n += p + 1;
    }
}

// Mirror of code_plane.  Reader: peek() = next 64 stream bits, skip(k).
// Bits past the budget are never consumed, so whatever follows the stream
// in the window cannot change the result.
template <int S, class Reader>
ZFPX_HD uint64_t decode_plane(Reader &rd, int &n, int &R)
{
    uint64_t X = 0;
    const int m = imin(n, R);
    if (m > 0) { X = rd.peek() & low_mask(m); rd.skip(m); R -= m; }
    while (R > 0 && n < S) {
        const uint64_t w = rd.peek();
        if (!(w & 1ull)) { rd.skip(1); R -= 1; break; }          // group empty
        const uint64_t after = w >> 1;                           // 63 bits after the group bit
        const int tz = after ? lowest_set(after) : 63;
        const int lim = S - 1 - n;                               // readable before the implied one
        if (tz < lim) {
            if (R < tz + 2) { R = 0; break; }                    // budget ends inside the zeros
            rd.skip(tz + 2); R -= tz + 2;
            X |= 1ull << (n + tz);
            n += tz + 1;
        } else {
            if (R < lim + 1) { R = 0; break; }
            rd.skip(lim + 1); R -= lim + 1;
            X |= 1ull << (S - 1);                                // implied
            n = S;
        }
    }
    return X;
}

// ----------------------------------------------------------------- 3-D block
// Encodes 64 values (x[i + 4j + 16k]) into exactly 64 RATE bits.
//
// Two passes over the bit planes, so that lanes coding different blocks do
// not diverge per plane.  Pass 1 walks the planes with closed forms: plane k
// with n significant coefficients costs n verbatim bits, a group bit and, if
// its bits n..63 hold c ones with the highest at h, (h - n + 1) value bits
// and c group bits after them (one value bit and one group bit less when
// h = 63, whose one is implied).  It writes the verbatim bits and the first
// group bit and leaves zeros for the rest.  Pass 2 visits each newly
// significant coefficient once: the t-th one (t = 0, 1, ...) of a plane, at
// coefficient p, sits at (plane start + n + 1) + (p - n) + t, that is plane
// start + 1 + p + t, with its group bit right after; pass 2 ORs those bits
// into the stream.
//
// Writer: RATE + 2 64-bit words, the last two slack that the caller drops;
// put(bits, len) for 1 <= len <= 64, zeros(len), finish() (flush and
// zero-fill to RATE words), orw(i, v) (OR v into word i after finish).
// Planes: store(k, X) / load(k), store_half(k, h, w), 32 slots.
template <int RATE, class Writer, class Planes>
ZFPX_HD void encode_block3(const float (&x)[64], Writer &wr, Planes &pl)
{
    constexpr int kSeq[64] = ZFPX_SEQ3;
    constexpr int END = 64 * RATE;
    uint32_t amax = 0;
#pragma unroll
    for (int i = 0; i < 64; i++) {
        const uint32_t a = f2u(x[i]) & 0x7fffffffu;
        amax = a > amax ? a : amax;
    }
    // E = e_max + 126; a subnormal max in [2^-127, 2^-126) has e_max = -126 too
    const int E = (int)(amax >> 23);
    if (amax < 0x00400000u || E == 255) { wr.finish(); return; }
    const QuantScale qs(E);
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
    // One transpose body for both halves keeps the kernel's code compact.
    // The budget rarely reaches below plane 16 at rate 8 (plane 8 at rate
    // 16): the planes above are finished here, and the words below wait
    // half-transposed in their slots until the coder first needs them.
    constexpr int kLow = RATE == 8 ? 16 : 8;
#pragma unroll 1
    for (int half = 0; half < 2; half++) {
        if (half) {
#pragma unroll
            for (int t = 0; t < 32; t++) lo[t] = hi[t];
        }
        transpose32_part1<kLow>(lo);
#pragma unroll
        for (int k = 0; k < 32; k++) pl.store_half(k, half, lo[k]);
    }
    wr.put(1ull | ((uint64_t)(E + 1) << 1), 9);
    // pass 1: plane costs, verbatim bits, first group bits.  The last plane
    // may run past the budget: its excess lands in the writer's two slack
    // words, so no bit count is clipped here.  A plane with new ones keeps
    // them in its own slot (already read) and is flagged in evm.
    int n = 0, pos = 9;
    uint32_t evm = 0;
    uint64_t lm = 0;                                             // low_mask(n)
#pragma unroll 1
    for (int k = 31; k >= 0 && pos < END; k--) {
        if (k == kLow - 1) {                                     // finish planes 0..kLow-1
            uint32_t a[32], b[32];
#pragma unroll
            for (int i = 0; i < kLow; i++) {
                a[i] = pl.load_half(i, 0);
                b[i] = pl.load_half(i, 1);
            }
            transpose32_part2<kLow>(a);
            transpose32_part2<kLow>(b);
#pragma unroll
            for (int i = 0; i < kLow; i++) pl.store(i, ((uint64_t)b[i] << 32) | a[i]);
        }
        const uint64_t X = pl.load(k);
        if (n >= 64) {                                           // every coefficient significant
            wr.put(X, 64);
            pos += 64;
            continue;
        }
        const uint64_t Y = X & ~lm;                              // candidates for significance
        wr.put((X & lm) | (Y ? lm + 1ull : 0ull), n + 1);        // verbatim bits, group bit
        int L = n + 1;
        if (Y) {
            const int h = highest_set64(Y);
            L = h < 63 ? h + 2 + popc64(Y) : h + popc64(Y);
            wr.zeros(L - n - 1);
            pl.store(k, Y);
            evm |= 1u << k;
            n = h + 1;
            lm = low_mask(n);
        }
        pos += L;
    }
    wr.finish();
    // pass 2: the bits of each newly significant coefficient, in stream
    // order.  A flagged plane's start follows from the previous one's: that
    // plane's cost, then one bit more than the significant count for each
    // plane without new ones in between.
    uint64_t rest = 0, cacc = 0;
    int ap = 0, t = 0, cw = 0, kp = 32, endp = 9, np = 0;
#pragma unroll 1
    for (;;) {
        if (!rest) {
            if (!evm) break;
            const int k = highest_set32(evm);
            evm &= ~(1u << k);
            rest = pl.load(k);
            const int start = endp + (kp - 1 - k) * (np + 1);
            ap = start + 1;
            const int h = highest_set64(rest), c = popc64(rest);
            endp = start + (h < 63 ? h + 2 + c : h + c);
            np = h + 1;
            kp = k;
            t = 0;
        }
        const int p = lowest_set(rest);
        rest &= rest - 1;
        const int A = ap + p + t;
        t++;
        if (A >= END) break;                                     // positions only grow
        // coefficient 63's one is implied; the group bit (more ones follow)
        // may fall at END, in a slack word
        const uint64_t b = (p != 63 ? 1ull : 0ull) | (rest ? 2ull : 0ull);
        const int w = A >> 6, s = A & 63;
        if (w != cw) {
            if (cacc) wr.orw(cw, cacc);
            cw = w;
            cacc = 0;
        }
        cacc |= b << s;
        if (s == 63 && (b & 2ull)) {
            wr.orw(cw, cacc);
            cw = w + 1;
            cacc = 1ull;
        }
    }
    if (cacc) wr.orw(cw, cacc);
}

// ----------------------------------------------------------------- 3-D decoder over a stream tile
// Reads are 64-bit windows funnel-shifted out of three tile words.  The tile
// holds the 2 RATE stream words and kTileZeroRows<RATE> zero words after
// them: three let the decoder read a window at the stream's end without a
// test; at rate 16 the decoder tests instead and two suffice, which is what
// lets six 3-warp CTAs share an SM.
template <int RATE>
constexpr int kTileZeroRows = RATE == 16 ? 2 : 3;
template <class Tile>
ZFPX_HD uint64_t tile_peek(const Tile &t, int pos)
{
    const int i = pos >> 5, sh = pos & 31;
    const uint32_t a = t.get(i), b = t.get(i + 1), c = t.get(i + 2);
#ifdef __CUDA_ARCH__
    const uint32_t lo = __funnelshift_r(a, b, sh), hi = __funnelshift_r(b, c, sh);
#else
    const uint32_t lo = (uint32_t)((((uint64_t)b << 32) | a) >> sh);
    const uint32_t hi = (uint32_t)((((uint64_t)c << 32) | b) >> sh);
#endif
    return ((uint64_t)hi << 32) | lo;
}

// The group-tested part of a plane, read from the window W that starts
// right after its first (set) group bit.  The part is a run of tokens: "0"
// (a coefficient that stays insignificant) or "1g" (a newly significant one
// and the group bit after it); it ends at the first g = 0, or without a
// closing bit where coefficient 63 is reached, whose one is implied.  Inside
// the part every run of ones starts on a value bit and alternates value,
// group, value, ...; a run of odd length ends on a value bit, and the 0
// after it closes the part.  Returns the value ones of W read that way
// (exact below the part's end) and in `term` the closing-0 candidates.
ZFPX_HD uint64_t group_values(uint64_t W, uint64_t &term)
{
    constexpr uint64_t kEven = 0x5555555555555555ull;
    const uint64_t starts = W & ~(W << 1);
    const uint64_t even_runs = W & ~(W + (starts & kEven));     // the carry clears runs that start even
    const uint64_t val = (even_runs & kEven) | (W & ~even_runs & ~kEven);
    const uint64_t ends = W & ~(W >> 1) & ~(1ull << 63);         // a run at bit 63 may go on
    term = (ends & val) << 1;
    return val;
}

// The bit planes of a 64-coefficient block, planes ktop, ktop - 1, ... from
// stream bit pos on, with the budget ending at bit END: plane by plane, each
// plane's group-tested part in one step when it closes inside a 64-bit
// window, below coefficient 63 and inside the budget; otherwise (rare) one
// newly significant coefficient per step.  SAFE: the tile holds at least
// three zero words after the budget, so a window may be read at any position
// before END + 32 without a test.  Stores every plane it reaches (pl.store)
// and returns the lowest; the planes below stay for the caller to clear.
template <bool SAFE, class Tile, class Planes>
ZFPX_HD int parse_planes64(const Tile &tile, int pos, const int END, const int ktop, Planes &pl)
{
    int n = 0, kmin = ktop + 1;
    uint64_t lm = 0;                                             // low_mask(n)
#pragma unroll 1
    for (int k = ktop; k >= 0 && pos < END; k--) {
        kmin = k;                                                // every pass stores plane k
        const int rem = END - pos;
        const uint64_t w = tile_peek(tile, pos);
        if (n >= 64) {                                           // verbatim plane
            pl.store(k, rem < 64 ? w & low_mask(rem) : w);
            pos += 64;
            continue;
        }
        uint64_t X = w & lm;
        if (rem <= n) { pl.store(k, w & low_mask(rem)); break; }     // budget ends in the verbatim bits
        pos += n + 1;
        if (!(w & (lm + 1ull))) { pl.store(k, X); continue; }       // group empty (lm + 1 = bit n)
        {
            // The whole part from one window.  The tile is zero past the
            // budget, so no one and no closing 0 can be read there: a part
            // cut by the budget shows as one that runs on, and only the
            // implied one needs the check that its zeros fit (B bits left).
            uint64_t term;
            uint64_t V = group_values(SAFE || pos < END ? tile_peek(tile, pos) : 0ull, term);
            const uint64_t below = term ? (term & (0ull - term)) - 1ull : ~0ull;   // bits before the closing 0
            const int T = popc64(below);                         // offset of the closing 0 (64: none)
            const int lim = 62 - n;                              // offset - rank of coefficient 62
            const int B = END - pos;
            // the t-th one, at offset p, is coefficient n + p - t: take the
            // ones lowest first, shifting the rest down by one after each
            int t = 0;
            uint64_t nw = 0;
            V &= below;
            while (V) {
                const uint64_t b = V & (0ull - V);
                nw |= b;
                V = (V ^ b) >> 1;
                t++;
            }
            // ones past coefficient 62 lie beyond a part that ends at the
            // implied one; the ones below stay, in the order they came
            const uint64_t keep = (~0ull >> n) >> 1;             // low_mask(lim + 1)
            const bool over = (nw & ~keep) != 0ull;             // a one past coefficient 62
            if (over) {
                nw &= keep;
                t = popc64(nw);
            }
            X |= nw << n;
            const int E = 63 - n + t;                            // end of the part if it ends at the implied one
            if (!over && term) {                                 // closed by a 0 below coefficient 63
                pl.store(k, X);
                n += T - t + 1;
                lm = low_mask(n);
                pos += T + 1;
                continue;
            }
            if (E <= 64) {                                       // ends at the implied one
                if (E > B) { pl.store(k, X); break; }
                X |= 1ull << 63;
                pl.store(k, X);
                pos += E;
                n = 64;
                lm = ~0ull;
                continue;
            }
            // else: the part runs past the window; X's low bits are reread below
            X = w & lm;
        }
        // one coefficient per step, with the budget and the implied last one
        bool cut = false;
#pragma unroll 1
        for (;;) {
            const int r = END - pos;
            const uint64_t v = SAFE || pos < END ? tile_peek(tile, pos) : 0ull;
            const int lim = 63 - n;
            const int tz = v ? lowest_set(v) : 64;
            if (tz >= lim) {                                     // only the implied one is left
                if (r < lim) { cut = true; break; }
                pos += lim;
                X |= 1ull << 63;
                n = 64;
                break;
            }
            if (r < tz + 1) { cut = true; break; }
            X |= 1ull << (n + tz);
            n += tz + 1;
            if (r == tz + 1) { cut = true; break; }              // budget ends before the group bit
            pos += tz + 2;
            if (!((v >> (tz + 1)) & 1ull)) break;                // group empty: plane done
        }
        pl.store(k, X);
        if (cut) break;
        lm = low_mask(n);
    }
    return kmin;
}

// Decodes one block from this lane's stream tile: its planes by
// parse_planes64, then the transposes, the inverse transform and the
// dequantisation.
template <int RATE, class Tile, class Planes>
ZFPX_HD void decode_block3_tile(const Tile &tile, float (&x)[64], Planes &pl)
{
    constexpr int kSeq[64] = ZFPX_SEQ3;
    constexpr int END = 64 * RATE;
    const uint64_t head = tile_peek(tile, 0);
    if (!(head & 1ull)) {
#pragma unroll
        for (int i = 0; i < 64; i++) x[i] = 0.0f;
        return;
    }
    const int e = (int)((head >> 1) & 0xffu);
    // planes below kmin stay zero
    const int kmin = parse_planes64<kTileZeroRows<RATE> >= 3>(tile, 9, END, 31, pl);
    uint32_t lo[32], hi[32];
    // Planes below kmin are zero; when that holds for planes 0..kLow-1 in
    // every lane of the warp, the stages smaller than kLow skip them.
    constexpr int kLow = RATE == 8 ? 16 : 8;
#ifdef __CUDA_ARCH__
    const bool low_zero = __all_sync(__activemask(), kmin >= kLow);
#else
    const bool low_zero = kmin >= kLow;
#endif
    if (low_zero) {
#pragma unroll
        for (int kk = kLow; kk < 32; kk++) {
            lo[kk] = kk >= kmin ? pl.load_half(kk, 0) : 0u;
            hi[kk] = kk >= kmin ? pl.load_half(kk, 1) : 0u;
        }
        transpose32_zero_low<kLow>(lo);
        transpose32_zero_low<kLow>(hi);
    } else {
#pragma unroll
        for (int kk = 0; kk < 32; kk++) {
            lo[kk] = kk >= kmin ? pl.load_half(kk, 0) : 0u;
            hi[kk] = kk >= kmin ? pl.load_half(kk, 1) : 0u;
        }
        transpose32(lo);
        transpose32(hi);
    }
    int32_t q[64];
#pragma unroll
    for (int t = 0; t < 32; t++) {
        q[kSeq[t]] = from_negabinary(lo[t]);
        q[kSeq[32 + t]] = from_negabinary(hi[t]);
    }
    xform3_inv(q);
    if (e >= 31) {
        const float sc = dequant_scale(e);
#pragma unroll
        for (int i = 0; i < 64; i++) x[i] = dequantize_fast(q[i], sc);
    } else {
        // tiny exponents (rare): a rolled loop over a local copy
        int32_t t[64];
#pragma unroll
        for (int i = 0; i < 64; i++) t[i] = q[i];
#pragma unroll 1
        for (int i = 0; i < 64; i++) t[i] = (int32_t)f2u(dequantize_small(t[i], e));
#pragma unroll
        for (int i = 0; i < 64; i++) x[i] = u2f((uint32_t)t[i]);
    }
}

// ----------------------------------------------------------------- 2-D block
// A 2-D block is 4 x 4 values x[i + 4j] (i along axis 0, j along axis 1) of
// one level, coded into exactly 16 RATE bits (128 at rate 8, 256 at rate 16).
// Transform: the lifting along i for every j, then along j for every i.
// Coefficient (i + 4j) coded at position t: total sequency i + j ascending,
// ties by i^2 + j^2, then by the index (the 3-D rule with k = 0).
#define ZFPX_SEQ2 {0, 1, 4, 5, 2, 8, 6, 9, 3, 12, 10, 7, 13, 11, 14, 15}

ZFPX_HD void xform2_fwd(int32_t (&q)[16])
{
#pragma unroll
    for (int j = 0; j < 4; j++) lift_fwd(q[4 * j], q[4 * j + 1], q[4 * j + 2], q[4 * j + 3]);
#pragma unroll
    for (int i = 0; i < 4; i++) lift_fwd(q[i], q[i + 4], q[i + 8], q[i + 12]);
}

ZFPX_HD void xform2_inv(int32_t (&q)[16])
{
#pragma unroll
    for (int i = 0; i < 4; i++) lift_inv(q[i], q[i + 4], q[i + 8], q[i + 12]);
#pragma unroll
    for (int j = 0; j < 4; j++) lift_inv(q[4 * j], q[4 * j + 1], q[4 * j + 2], q[4 * j + 3]);
}

// Encodes x[i + 4j] into 16 RATE bits.  The 16 coefficients' bit planes come
// from one 32x32 transpose whose lower 16 rows are zero (the coefficients sit
// in rows 16..31, so plane k is the high 16 bits of word k and the stages
// below 16 only touch the upper rows), parked in the lane's plane slots;
// the planes are coded in the two passes of encode_block3.  Writer: as for
// encode_block3 (put, zeros, finish, orw; two slack words past 16 RATE
// bits).  Planes: store_half(k, 0, w) / load_half(k, 0), 32 slots of 32 bits.
template <int RATE, class Writer, class Planes>
ZFPX_HD void encode_block2(const float (&x)[16], Writer &wr, Planes &pl)
{
    constexpr int kSeq[16] = ZFPX_SEQ2;
    uint32_t amax = 0;
#pragma unroll
    for (int i = 0; i < 16; i++) {
        const uint32_t a = f2u(x[i]) & 0x7fffffffu;
        amax = a > amax ? a : amax;
    }
    const int E = (int)(amax >> 23);
    if (amax < 0x00400000u || E == 255) { wr.finish(); return; }
    const QuantScale qs(E);
    int32_t q[16];
#pragma unroll
    for (int i = 0; i < 16; i++) q[i] = qs(x[i]);
    xform2_fwd(q);
    uint32_t w[32];
#pragma unroll
    for (int t = 0; t < 16; t++) w[16 + t] = to_negabinary(q[kSeq[t]]);
    transpose32_zero_low<16>(w);
#pragma unroll
    for (int k = 0; k < 32; k++) pl.store_half(k, 0, w[k] >> 16);
    wr.put(1ull | ((uint64_t)(E + 1) << 1), 9);
    // The two passes of encode_block3 with 16 coefficients: pass 1 writes each
    // plane's verbatim bits and first group bit and leaves zeros for its
    // group-tested part (the last plane may run into the writer's slack
    // words); planes with new ones keep them in their slot, flagged in evm.
    constexpr int END = 16 * RATE;
    int n = 0, pos = 9;
    uint32_t evm = 0, lm = 0;                                    // lm = low_mask(n)
#pragma unroll 1
    for (int k = 31; k >= 0 && pos < END; k--) {
        const uint32_t X = pl.load_half(k, 0);
        if (n >= 16) {                                           // every coefficient significant
            wr.put(X, 16);
            pos += 16;
            continue;
        }
        const uint32_t Y = X & ~lm;
        wr.put((X & lm) | (Y ? lm + 1u : 0u), n + 1);
        int L = n + 1;
        if (Y) {
            const int h = highest_set32(Y), c = popc32(Y);
            L = h < 15 ? h + 2 + c : h + c;
            wr.zeros(L - n - 1);
            pl.store_half(k, 0, Y);
            evm |= 1u << k;
            n = h + 1;
            lm = (2u << h) - 1u;
        }
        pos += L;
    }
    wr.finish();
    // pass 2: the bits of each newly significant coefficient (the t-th one of
    // a plane, at coefficient p, sits at plane start + 1 + p + t, its group
    // bit right after; coefficient 15's one is implied)
    uint32_t rest = 0;
    uint64_t cacc = 0;
    int ap = 0, t = 0, cw = 0, kp = 32, endp = 9, np = 0;
#pragma unroll 1
    for (;;) {
        if (!rest) {
            if (!evm) break;
            const int k = highest_set32(evm);
            evm &= ~(1u << k);
            rest = pl.load_half(k, 0);
            const int start = endp + (kp - 1 - k) * (np + 1);
            ap = start + 1;
            const int h = highest_set32(rest), c = popc32(rest);
            endp = start + (h < 15 ? h + 2 + c : h + c);
            np = h + 1;
            kp = k;
            t = 0;
        }
        const int p = lowest_set32(rest);
        rest &= rest - 1u;
        const int A = ap + p + t;
        t++;
        if (A >= END) break;                                     // positions only grow
        const uint64_t b = (p != 15 ? 1ull : 0ull) | (rest ? 2ull : 0ull);
        const int w = A >> 6, sh = A & 63;
        if (w != cw) {
            if (cacc) wr.orw(cw, cacc);
            cw = w;
            cacc = 0;
        }
        cacc |= b << sh;
        if (sh == 63 && (b & 2ull)) {
            wr.orw(cw, cacc);
            cw = w + 1;
            cacc = 1ull;
        }
    }
    if (cacc) wr.orw(cw, cacc);
}

// Reader over a stream tile: peek() = the 64 bits from the current position.
template <class Tile>
struct TileReader {
    const Tile &t;
    int pos;
    ZFPX_HD uint64_t peek() const { return tile_peek(t, pos); }
    ZFPX_HD void skip(int k) { pos += k; }
};

// Decodes one 2-D block from this lane's stream tile (2 RATE / 4 words of 32
// bits, then at least two zero words).  Planes below the last one the budget
// reached stay zero.
template <int RATE, class Tile, class Planes>
ZFPX_HD void decode_block2_tile(const Tile &tile, float (&x)[16], Planes &pl)
{
    constexpr int kSeq[16] = ZFPX_SEQ2;
    const uint64_t head = tile_peek(tile, 0);
    if (!(head & 1ull)) {
#pragma unroll
        for (int i = 0; i < 16; i++) x[i] = 0.0f;
        return;
    }
    const int e = (int)((head >> 1) & 0xffu);
    // Plane by plane from one 64-bit window: n verbatim bits, the first group
    // bit, and a group-tested part of at most 16 - n value bits and 15 group
    // bits, 48 bits in all.  The tile is zero past the budget, so a part the
    // budget cuts reads on as zeros: no one and no closing 0 appear there,
    // and only the implied one of coefficient 15 needs the check that its
    // bits fit (the 3-D decoder's reading, with 16 coefficients).
    constexpr int END = 16 * RATE;
    int pos = 9, n = 0, kmin = 32;
    uint32_t lm = 0;                                             // low n bits
#pragma unroll 1
    for (int k = 31; k >= 0 && pos < END; k--) {
        kmin = k;
        const int rem = END - pos;
        const uint64_t w = tile_peek(tile, pos);
        if (n >= 16) {                                           // verbatim plane
            pl.store_half(k, 0, (uint32_t)w & (rem < 16 ? (1u << rem) - 1u : 0xffffu));
            pos += 16;
            continue;
        }
        uint32_t X = (uint32_t)w & lm;
        if (rem <= n) { pl.store_half(k, 0, (uint32_t)w & ((1u << rem) - 1u)); break; }   // cut in the verbatim bits
        pos += n + 1;
        if (!(w & (uint64_t)(lm + 1u))) { pl.store_half(k, 0, X); continue; }           // group empty
        uint64_t term;
        uint64_t V = group_values(w >> (n + 1), term);
        const uint64_t below = term ? (term & (0ull - term)) - 1ull : ~0ull;   // bits before the closing 0
        const int T = popc64(below);
        // the t-th one, at offset p, is coefficient n + p - t: take the ones
        // lowest first, shifting the rest down by one after each
        int t = 0;
        uint64_t nw = 0;
        V &= below;
        while (V) {
            const uint64_t b = V & (0ull - V);
            nw |= b;
            V = (V ^ b) >> 1;
            t++;
        }
        // ones past coefficient 14 lie beyond a part that ends at the implied one
        const uint64_t keep = (1ull << (15 - n)) - 1ull;
        const bool over = (nw & ~keep) != 0ull;
        if (over) {
            nw &= keep;
            t = popc64(nw);
        }
        X |= (uint32_t)nw << n;
        if (!over && term) {                                     // closed by a 0 below coefficient 15
            pl.store_half(k, 0, X);
            n += T - t + 1;
            lm = (1u << n) - 1u;
            pos += T + 1;
            continue;
        }
        const int E = 15 - n + t;                                // the part ends at the implied one
        if (E > END - pos) { pl.store_half(k, 0, X); break; }
        pl.store_half(k, 0, X | 0x8000u);
        pos += E;
        n = 16;
        lm = 0xffffu;
    }
    // Planes below kmin are zero; when planes 0..15 are zero in every lane of
    // the warp, the transpose stages below 16 skip them.
    uint32_t w[32];
#ifdef __CUDA_ARCH__
    const bool low_zero = __all_sync(__activemask(), kmin >= 16);
#else
    const bool low_zero = kmin >= 16;
#endif
    if (low_zero) {
#pragma unroll
        for (int k = 16; k < 32; k++) w[k] = k >= kmin ? pl.load_half(k, 0) : 0u;
        transpose32_zero_low<16>(w);
    } else {
#pragma unroll
        for (int k = 0; k < 32; k++) w[k] = k >= kmin ? pl.load_half(k, 0) : 0u;
        transpose32(w);
    }
    int32_t q[16];
#pragma unroll
    for (int t = 0; t < 16; t++) q[kSeq[t]] = from_negabinary(w[t]);
    xform2_inv(q);
    if (e >= 31) {
        const float sc = dequant_scale(e);
#pragma unroll
        for (int i = 0; i < 16; i++) x[i] = dequantize_fast(q[i], sc);
    } else {
        // tiny exponents (rare): a rolled loop over a local copy
        int32_t t[16];
#pragma unroll
        for (int i = 0; i < 16; i++) t[i] = q[i];
#pragma unroll 1
        for (int i = 0; i < 16; i++) t[i] = (int32_t)f2u(dequantize_small(t[i], e));
#pragma unroll
        for (int i = 0; i < 16; i++) x[i] = u2f((uint32_t)t[i]);
    }
}

// ----------------------------------------------------------------- 1-D block
// A 1-D block is 4 RATE <= 64 bits, returned in one word (LSB = first bit).
struct RegWriter {
    uint64_t acc;
    int nb;
    ZFPX_HD void put(uint64_t bits, int len) { acc |= bits << nb; nb += len; }
};
struct WordReader {
    uint64_t w;
    int off;
    ZFPX_HD uint64_t peek() const { return off < 64 ? (w >> off) : 0ull; }
    ZFPX_HD void skip(int k) { off += k; }
};

// With four coefficients a plane's code depends only on n (significant
// coefficients, 0..4) and its four bits X (encoding) or the next seven stream
// bits (decoding; no plane of four takes more).  The coders look planes up in
// a table built from code_plane / decode_plane at launch: encoder entry
// (n, X) = code bits 0..6, length bits 7..9, new n bits 10..12; decoder entry
// (n, w7) = X bits 0..3, length bits 4..6, new n bits 7..9.
// The encoder's output is the first 4 RATE bits of the unbounded code
// (code_plane only ever cuts a plane short), so its loop just stops at the
// budget.  For a plane the budget cuts after r bits the decoder looks up the
// window with the bits from r on cleared: zeros past the budget add no one
// except, when n < 4, the implied one of coefficient 3, which needs the whole
// plane and so is dropped; what is left is what reading stops at the budget
// gives.  Both run K blocks of a lane in lockstep so that their table
// lookups, which each plane's successor waits for, overlap.
struct Plane4Enc {
    uint16_t e[5 * 16];
};
struct Plane4Dec {
    uint16_t d[5 * 128];
};

ZFPX_HD uint16_t plane4_enc_entry(int n, uint32_t X)
{
    RegWriter wr{0ull, 0};
    int nn = n, R = 64;
    code_plane<4>(wr, X, nn, R);
    return (uint16_t)((uint32_t)wr.acc | ((uint32_t)wr.nb << 7) | ((uint32_t)nn << 10));
}

ZFPX_HD uint16_t plane4_dec_entry(int n, uint32_t w7)
{
    WordReader rd{w7, 0};
    int nn = n, R = 64;
    const uint32_t X = (uint32_t)decode_plane<4>(rd, nn, R);
    return (uint16_t)(X | ((uint32_t)rd.off << 4) | ((uint32_t)nn << 7));
}

// Fills a table with `nthreads` threads, thread `t` taking every nthreads-th
// entry (the caller synchronises).
ZFPX_HD void plane4_fill(Plane4Enc &tab, int t, int nthreads)
{
    for (int i = t; i < 5 * 16; i += nthreads) tab.e[i] = plane4_enc_entry(i >> 4, (uint32_t)i & 15u);
}
ZFPX_HD void plane4_fill(Plane4Dec &tab, int t, int nthreads)
{
    for (int i = t; i < 5 * 128; i += nthreads) tab.d[i] = plane4_dec_entry(i >> 7, (uint32_t)i & 127u);
}

// Encodes K blocks x[b][0..3]; w[b] = the block's 4 RATE bits.
template <int RATE, int K>
ZFPX_HD void encode_blocks1(const float (&x)[K][4], const Plane4Enc &tab, uint64_t (&w)[K])
{
    constexpr int END = 4 * RATE;
    uint32_t u[K][4];
    int pos[K], n[K];
#pragma unroll
    for (int b = 0; b < K; b++) {
        uint32_t amax = 0;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const uint32_t a = f2u(x[b][i]) & 0x7fffffffu;
            amax = a > amax ? a : amax;
        }
        const int E = (int)(amax >> 23);
        const bool zero = amax < 0x00400000u || E == 255;          // a single 0 bit
        const QuantScale qs(zero ? 127 : E);
        int32_t q0 = qs(x[b][0]), q1 = qs(x[b][1]), q2 = qs(x[b][2]), q3 = qs(x[b][3]);
        lift_fwd(q0, q1, q2, q3);
        u[b][0] = to_negabinary(q0); u[b][1] = to_negabinary(q1);
        u[b][2] = to_negabinary(q2); u[b][3] = to_negabinary(q3);
        w[b] = zero ? 0ull : 1ull | ((uint64_t)(E + 1) << 1);      // header, 9 bits
        pos[b] = zero ? END : 9;
        n[b] = 0;
    }
#pragma unroll 1
    for (int k = 31; k >= 0; k--) {
        bool more = false;
#pragma unroll
        for (int b = 0; b < K; b++) {
            if (pos[b] >= END) continue;
            const uint32_t X = ((u[b][0] >> k) & 1u) | (((u[b][1] >> k) & 1u) << 1) | (((u[b][2] >> k) & 1u) << 2) |
                               (((u[b][3] >> k) & 1u) << 3);
            const uint32_t e = tab.e[n[b] * 16 + (int)X];
            w[b] |= (uint64_t)(e & 127u) << pos[b];                // pos < END <= 64
            pos[b] += (int)((e >> 7) & 7u);
            n[b] = (int)(e >> 10);
            more |= pos[b] < END;
        }
        if (!more) break;
    }
#pragma unroll
    for (int b = 0; b < K; b++) w[b] &= low_mask(END);
}

// Decodes K blocks from their 4 RATE-bit words.
template <int RATE, int K>
ZFPX_HD void decode_blocks1(const uint64_t (&win)[K], const Plane4Dec &tab, float (&x)[K][4])
{
    constexpr int END = 4 * RATE;
    uint64_t w[K];
    uint32_t u[K][4];
    int pos[K], n[K];
#pragma unroll
    for (int b = 0; b < K; b++) {
        w[b] = win[b] & low_mask(END);
        pos[b] = (w[b] & 1ull) ? 9 : END;
        n[b] = 0;
        u[b][0] = u[b][1] = u[b][2] = u[b][3] = 0u;
    }
#pragma unroll 1
    for (int k = 31; k >= 0; k--) {
        bool more = false;
#pragma unroll
        for (int b = 0; b < K; b++) {
            if (pos[b] >= END) continue;
            const int r = END - pos[b];
            uint32_t w7 = (uint32_t)(w[b] >> pos[b]) & 127u;       // pos < END <= 64
            if (r < 7) w7 &= (1u << r) - 1u;
            const uint32_t d = tab.d[n[b] * 128 + (int)w7];
            uint32_t X = d & 15u;
            const int len = (int)((d >> 4) & 7u);
            if (len > r) {                                         // the budget cuts this plane
                if (n[b] < 4) X &= 7u;
                pos[b] = END;
            } else {
                pos[b] += len;
                n[b] = (int)(d >> 7);
            }
            u[b][0] |= (X & 1u) << k;
            u[b][1] |= ((X >> 1) & 1u) << k;
            u[b][2] |= ((X >> 2) & 1u) << k;
            u[b][3] |= ((X >> 3) & 1u) << k;
            more |= pos[b] < END;
        }
        if (!more) break;
    }
#pragma unroll
    for (int b = 0; b < K; b++) {
        if (!(w[b] & 1ull)) {
            x[b][0] = x[b][1] = x[b][2] = x[b][3] = 0.0f;
            continue;
        }
        const int e = (int)((w[b] >> 1) & 0xffu);
        int32_t q0 = from_negabinary(u[b][0]), q1 = from_negabinary(u[b][1]);
        int32_t q2 = from_negabinary(u[b][2]), q3 = from_negabinary(u[b][3]);
        lift_inv(q0, q1, q2, q3);
        if (e >= 31) {
            const float sc = dequant_scale(e);
            x[b][0] = dequantize_fast(q0, sc); x[b][1] = dequantize_fast(q1, sc);
            x[b][2] = dequantize_fast(q2, sc); x[b][3] = dequantize_fast(q3, sc);
        } else {
            x[b][0] = dequantize_small(q0, e); x[b][1] = dequantize_small(q1, e);
            x[b][2] = dequantize_small(q2, e); x[b][3] = dequantize_small(q3, e);
        }
    }
}

template <int RATE>
ZFPX_HD uint64_t encode_block1(const float (&x)[4], const Plane4Enc &tab)
{
    const float (&xx)[1][4] = reinterpret_cast<const float (&)[1][4]>(x);
    uint64_t w[1];
    encode_blocks1<RATE, 1>(xx, tab, w);
    return w[0];
}

template <int RATE>
ZFPX_HD void decode_block1(uint64_t w, float (&x)[4], const Plane4Dec &tab)
{
    const uint64_t win[1] = {w};
    float (&xx)[1][4] = reinterpret_cast<float (&)[1][4]>(x);
    decode_blocks1<RATE, 1>(win, tab, xx);
}

}  // namespace blk
}  // namespace zfpx
