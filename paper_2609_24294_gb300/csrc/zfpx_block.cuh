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
ZFPX_HD double ll2d(long long v)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double(v);
#else
    double d; std::memcpy(&d, &v, 8); return d;
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
ZFPX_HD uint64_t low_mask(int n) { return n >= 64 ? ~0ull : ((1ull << n) - 1); }
ZFPX_HD int imin(int a, int b) { return a < b ? a : b; }

// int32 ring arithmetic: wraps like the hardware, without signed overflow.
ZFPX_HD int32_t wadd(int32_t a, int32_t b) { return (int32_t)((uint32_t)a + (uint32_t)b); }
ZFPX_HD int32_t wsub(int32_t a, int32_t b) { return (int32_t)((uint32_t)a - (uint32_t)b); }

// ----------------------------------------------------------------- block float
// q = trunc(x 2^(30 - e_max)), e_max = E - 126 with E the biased exponent of
// a normal max.  For E >= 29 the scale is a normal float and the product is
// exact wherever its integer part is non-zero; smaller E go through double.
ZFPX_HD int32_t quantize(float x, int E)
{
    if (E >= 29) {
        const float y = x * u2f((uint32_t)(283 - E) << 23);
#ifdef __CUDA_ARCH__
        return __float2int_rz(y);
#else
        return (int32_t)y;
#endif
    }
    const double y = (double)x * ll2d((long long)(1023 + 156 - E) << 52);
#ifdef __CUDA_ARCH__
    return __double2int_rz(y);
#else
    return (int32_t)y;
#endif
}
// x = (float)(q 2^(e_max - 30)), e = e_max + 127: for e >= 31 the scale is a
// normal float and rounding q once to float then scaling is exact.
ZFPX_HD float dequantize(int32_t q, int e)
{
    if (e >= 31) {
#ifdef __CUDA_ARCH__
        return __int2float_rn(q) * u2f((uint32_t)(e - 30) << 23);
#else
        return (float)q * u2f((uint32_t)(e - 30) << 23);
#endif
    }
    const double y = (double)q * ll2d((long long)(1023 + e - 157) << 52);
#ifdef __CUDA_ARCH__
    return __double2float_rn(y);
#else
    return (float)y;
#endif
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
ZFPX_HD void transpose32(uint32_t (&w)[32])
{
#pragma unroll
    for (int i = 0; i < 16; i++) {
        const uint32_t a = w[i], b = w[i + 16];
        w[i] = byte_perm(a, b, 0x5410);
        w[i + 16] = byte_perm(a, b, 0x7632);
    }
#pragma unroll
    for (int i = 0; i < 32; i++) {
        if (i & 8) continue;
        const uint32_t a = w[i], b = w[i + 8];
        w[i] = byte_perm(a, b, 0x6240);
        w[i + 8] = byte_perm(a, b, 0x7351);
    }
#pragma unroll
    for (int i = 0; i < 32; i++) {
        if (i & 4) continue;
        const uint32_t t = ((w[i] >> 4) ^ w[i + 4]) & 0x0F0F0F0Fu;
        w[i + 4] ^= t; w[i] ^= t << 4;
    }
#pragma unroll
    for (int i = 0; i < 32; i++) {
        if (i & 2) continue;
        const uint32_t t = ((w[i] >> 2) ^ w[i + 2]) & 0x33333333u;
        w[i + 2] ^= t; w[i] ^= t << 2;
    }
#pragma unroll
    for (int i = 0; i < 32; i++) {
        if (i & 1) continue;
        const uint32_t t = ((w[i] >> 1) ^ w[i + 1]) & 0x55555555u;
        w[i + 1] ^= t; w[i] ^= t << 1;
    }
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
// Encodes 64 values (x[i + 4j + 16k]) into exactly 64 RATE bits through wr;
// wr.finish() is called once at the end to flush and zero-fill.
template <int RATE, class Writer>
ZFPX_HD void encode_block3(const float (&x)[64], Writer &wr)
{
    constexpr int kSeq[64] = ZFPX_SEQ3;
    uint32_t amax = 0;
#pragma unroll
    for (int i = 0; i < 64; i++) {
        const uint32_t a = f2u(x[i]) & 0x7fffffffu;
        amax = a > amax ? a : amax;
    }
    // E = e_max + 126; a subnormal max in [2^-127, 2^-126) has e_max = -126 too
    const int E = (int)(amax >> 23);
    if (amax < 0x00400000u || E == 255) { wr.finish(); return; }
    int32_t q[64];
#pragma unroll
    for (int i = 0; i < 64; i++) q[i] = quantize(x[i], E);
    xform3_fwd(q);
    uint32_t lo[32], hi[32];
#pragma unroll
    for (int t = 0; t < 32; t++) {
        lo[t] = to_negabinary(q[kSeq[t]]);
        hi[t] = to_negabinary(q[kSeq[32 + t]]);
    }
    transpose32(lo);
    transpose32(hi);
    wr.put(1ull | ((uint64_t)(E + 1) << 1), 9);
    int n = 0, R = 64 * RATE - 9;
#pragma unroll
    for (int k = 31; k >= 0; k--) {
        if (R > 0) code_plane<64>(wr, ((uint64_t)hi[k] << 32) | lo[k], n, R);
    }
    wr.finish();
}

template <int RATE, class Reader>
ZFPX_HD void decode_block3(Reader &rd, float (&x)[64])
{
    constexpr int kSeq[64] = ZFPX_SEQ3;
    const uint64_t head = rd.peek();
    if (!(head & 1ull)) {
#pragma unroll
        for (int i = 0; i < 64; i++) x[i] = 0.0f;
        return;
    }
    const int e = (int)((head >> 1) & 0xffu);
    rd.skip(9);
    uint32_t lo[32], hi[32];
    int n = 0, R = 64 * RATE - 9;
#pragma unroll
    for (int k = 31; k >= 0; k--) {
        uint64_t X = 0;
        if (R > 0) X = decode_plane<64>(rd, n, R);
        lo[k] = (uint32_t)X;
        hi[k] = (uint32_t)(X >> 32);
    }
    transpose32(lo);
    transpose32(hi);
    int32_t q[64];
#pragma unroll
    for (int t = 0; t < 32; t++) {
        q[kSeq[t]] = from_negabinary(lo[t]);
        q[kSeq[32 + t]] = from_negabinary(hi[t]);
    }
    xform3_inv(q);
#pragma unroll
    for (int i = 0; i < 64; i++) x[i] = dequantize(q[i], e);
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

template <int RATE>
ZFPX_HD uint64_t encode_block1(const float (&x)[4])
{
    uint32_t amax = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const uint32_t a = f2u(x[i]) & 0x7fffffffu;
        amax = a > amax ? a : amax;
    }
    const int E = (int)(amax >> 23);
    RegWriter wr{0ull, 0};
    if (amax < 0x00400000u || E == 255) return 0ull;
    int32_t q0 = quantize(x[0], E), q1 = quantize(x[1], E), q2 = quantize(x[2], E), q3 = quantize(x[3], E);
    lift_fwd(q0, q1, q2, q3);
    const uint32_t u0 = to_negabinary(q0), u1 = to_negabinary(q1);
    const uint32_t u2 = to_negabinary(q2), u3 = to_negabinary(q3);
    wr.put(1ull | ((uint64_t)(E + 1) << 1), 9);
    int n = 0, R = 4 * RATE - 9;
#pragma unroll
    for (int k = 31; k >= 0; k--) {
        if (R > 0) {
            const uint64_t X = ((u0 >> k) & 1u) | (((u1 >> k) & 1u) << 1) | (((u2 >> k) & 1u) << 2) |
                               (((u3 >> k) & 1u) << 3);
            code_plane<4>(wr, X, n, R);
        }
    }
    return wr.acc;
}

template <int RATE>
ZFPX_HD void decode_block1(uint64_t w, float (&x)[4])
{
    x[0] = x[1] = x[2] = x[3] = 0.0f;
    if (!(w & 1ull)) return;
    const int e = (int)((w >> 1) & 0xffu);
    WordReader rd{w, 9};
    uint32_t u[4] = {0u, 0u, 0u, 0u};
    int n = 0, R = 4 * RATE - 9;
#pragma unroll
    for (int k = 31; k >= 0; k--) {
        if (R > 0) {
            const uint64_t X = decode_plane<4>(rd, n, R);
#pragma unroll
            for (int i = 0; i < 4; i++) u[i] |= (uint32_t)((X >> i) & 1ull) << k;
        }
    }
    int32_t q0 = from_negabinary(u[0]), q1 = from_negabinary(u[1]);
    int32_t q2 = from_negabinary(u[2]), q3 = from_negabinary(u[3]);
    lift_inv(q0, q1, q2, q3);
    x[0] = dequantize(q0, e); x[1] = dequantize(q1, e);
    x[2] = dequantize(q2, e); x[3] = dequantize(q3, e);
}

}  // namespace blk
}  // namespace zfpx
