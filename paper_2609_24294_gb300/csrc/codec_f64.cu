// float64 fields, 3-D blocks, fixed rate (raw arrays).  The float32 method
// with the double format's sizes (readings identical in the CPU oracle):
// e_max = frexp exponent of max|x|; zero block (one 0 bit) if max|x| is 0,
// below 2^-1023 or non-finite; header = a 1 bit and e_max + 1023 in 11 bits;
// q = trunc(x 2^(62 - e_max)) in int64; the five-step lifting in int64 along
// x, y, z; the 3-D coefficient order; 64-bit negabinary; group-tested bit
// planes 63 .. 0 cut at exactly 64 r bits; decode x = q 2^(e_max - 62)
// rounded once to nearest even.
//
// One lane per block, 32 consecutive blocks per warp, one warp per CTA.  A
// block's 64 int64 values live in the lane's registers (128 of them) through
// the gather, quantisation, transform and negabinary map; the 64 bit planes
// come from four 32x32 register transposes (low / high 32 coefficients x low
// / high 32 bits) and wait in shared memory ([plane][lane]) for the coder,
// which writes the lane's column of a [word][lane] stream tile.  Rates 1 .. 32
// bits per value.
#include <algorithm>
#include <climits>
#include <cuda_runtime.h>

#include "zfpx_internal.h"
#include "zfpx_block.cuh"
#include "zfpx_smem.cuh"

namespace zfpx {
namespace {

using namespace blk;

constexpr int kMaxRate = 32;
constexpr int kF64MinCtas = 10;         // one-warp CTAs per SM the registers are budgeted for
constexpr uint64_t kNega64 = 0xAAAAAAAAAAAAAAAAull;

__device__ __forceinline__ int64_t add64(int64_t a, int64_t b) { return (int64_t)((uint64_t)a + (uint64_t)b); }
__device__ __forceinline__ int64_t sub64(int64_t a, int64_t b) { return (int64_t)((uint64_t)a - (uint64_t)b); }

// Writer into this lane's column of a [word][lane] tile of nwords + 2 words.
struct VarWriter {
    uint64_t *sm;
    uint64_t acc;
    int nb, w, lane, nwords;
    __device__ __forceinline__ uint64_t &word(int i) const { return sm[i * 32 + lane]; }
    __device__ __forceinline__ void put(uint64_t bits, int len)
    {
        acc |= bits << nb;
        int t = nb + len;
        if (t >= 64) {
            word(w) = acc;
            w++;
            acc = nb ? (bits >> (64 - nb)) : 0ull;
            t -= 64;
        }
        nb = t;
    }
    __device__ __forceinline__ void finish()
    {
        if (nb > 0) { word(w) = acc; w++; }
        for (; w < nwords; w++) word(w) = 0ull;
    }
};

// One lane's stream in a [64-bit word][lane] tile; peek(pos) = the 64 stream
// bits from bit pos on (reads words pos / 64 and pos / 64 + 1).
struct Tile64 {
    const uint64_t *sm;
    int lane;
    __device__ __forceinline__ uint64_t peek(int pos) const
    {
        const int w = pos >> 6, sh = pos & 63;
        const uint64_t a = sm[w * 32 + lane];
        return sh ? (a >> sh) | (sm[(w + 1) * 32 + lane] << (64 - sh)) : a;
    }
};

// The same stream as 32-bit words (word i is the low half of 64-bit word
// i / 2 for even i, the high half for odd i), for the float32 path's plane
// parser.
struct Tile64As32 {
    const uint32_t *sm;
    int lane;
    __device__ __forceinline__ uint32_t get(int i) const { return sm[2 * ((i >> 1) * 32 + lane) + (i & 1)]; }
};

struct Geom64 {
    int64_t n[3], s[3];
    int64_t bx, by, nblocks, nunits;
    int rate;
    int vec;        // unit x stride, even y and z strides, 16-byte aligned base: rows of a block are
                    // two 16-byte moves each
};

__device__ __forceinline__ void block_origin(const Geom64 &g, int64_t b, int64_t &x0, int64_t &y0, int64_t &z0)
{
    const int64_t t = b / g.bx;
    x0 = 4 * (b - t * g.bx);
    y0 = 4 * (t % g.by);
    z0 = 4 * (t / g.by);
}

// exponent: 0 for a zero block, else e_max + 1023 (1 .. 2046)
__device__ __forceinline__ int block_exponent(uint64_t amax)
{
    const int E = (int)(amax >> 52);
    if (E == 2047 || amax < 0x0008000000000000ull) return 0;     // non-finite, or below 2^-1023
    return E == 0 ? 1 : E + 1;                                   // frexp exponent + 1023
}

// The quantisation and the dequantisation of the common case in integer
// operations on the bits: on this GPU the float64 pipe runs at a small
// fraction of the integer one, and these are the path's only float64
// arithmetic.  Both give the bits of the float64 formulas exactly (the
// products by powers of two there are exact, so only the truncation and the
// one rounding of q to 53 bits remain).
//
// q = trunc(x 2^(62 - e_max)), e = e_max + 1023 the block's exponent: x =
// +-M 2^(E - 1075) with E the biased exponent (taken as 1 for subnormals) and
// M the significand (with the implicit bit for normals), so |q| is M shifted
// left by E + 10 - e (at most 10 within the block whose maximum set e) or
// right by its negative.
__device__ __forceinline__ int64_t quantize64(uint64_t bits, int e)
{
    const int E = (int)((bits >> 52) & 0x7ffu);
    const uint64_t M = (bits & 0x000fffffffffffffull) | (E ? 0x0010000000000000ull : 0ull);
    const int t = (E ? E : 1) + 10 - e;
    const uint64_t a = t >= 0 ? (M << t) : (t > -64 ? (M >> -t) : 0ull);
    return (bits >> 63) ? (int64_t)(0ull - a) : (int64_t)a;
}

// x = q 2^(e - 1085) rounded once to nearest even, for e >= 63, where every
// non-zero result is normal (or, past the largest double, infinite): the one
// rounding is the conversion of q, and the power-of-two scaling an integer
// add to the exponent field (infinity where it passes the largest exponent).
__device__ __forceinline__ double dequantize64_normal(int64_t q, int e)
{
    const uint64_t b = (uint64_t)__double_as_longlong(__ll2double_rn(q));
    const int E = (int)((b >> 52) & 0x7ffu);                     // 0 only for q = 0
    const int ne = E + e - 1085;                                 // >= 1 for q != 0
    const uint64_t r = ne >= 2047 ? (b & 0x8000000000000000ull) | 0x7ff0000000000000ull
                                  : b + ((uint64_t)(int64_t)(e - 1085) << 52);
    return __longlong_as_double((long long)(E ? r : b));
}

// The 3-D transform on a block held in registers (int64 v[i + 4j + 16k]).
__device__ __forceinline__ void lift_fwd64r(int64_t &a, int64_t &b, int64_t &c, int64_t &d)
{
    a = add64(a, d) >> 1; d = sub64(d, a);
    c = add64(c, b) >> 1; b = sub64(b, c);
    a = add64(a, c) >> 1; c = sub64(c, a);
    d = add64(d, b) >> 1; b = sub64(b, d);
    d = add64(d, b >> 1); b = sub64(b, d >> 1);
}
__device__ __forceinline__ void lift_inv64r(int64_t &a, int64_t &b, int64_t &c, int64_t &d)
{
    b = add64(b, d >> 1); d = sub64(d, b >> 1);
    b = add64(b, d); d = sub64(add64(d, d), b);
    c = add64(c, a); a = sub64(add64(a, a), c);
    b = add64(b, c); c = sub64(add64(c, c), b);
    d = add64(d, a); a = sub64(add64(a, a), d);
}
__device__ __forceinline__ void xform3_fwd64(int64_t (&v)[64])
{
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
        for (int j = 0; j < 4; j++)
            lift_fwd64r(v[16 * k + 4 * j], v[16 * k + 4 * j + 1], v[16 * k + 4 * j + 2], v[16 * k + 4 * j + 3]);
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
        for (int i = 0; i < 4; i++)
            lift_fwd64r(v[16 * k + i], v[16 * k + i + 4], v[16 * k + i + 8], v[16 * k + i + 12]);
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
        for (int i = 0; i < 4; i++)
            lift_fwd64r(v[4 * j + i], v[4 * j + i + 16], v[4 * j + i + 32], v[4 * j + i + 48]);
}
__device__ __forceinline__ void xform3_inv64(int64_t (&v)[64])
{
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
        for (int i = 0; i < 4; i++)
            lift_inv64r(v[4 * j + i], v[4 * j + i + 16], v[4 * j + i + 32], v[4 * j + i + 48]);
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
        for (int i = 0; i < 4; i++)
            lift_inv64r(v[16 * k + i], v[16 * k + i + 4], v[16 * k + i + 8], v[16 * k + i + 12]);
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
        for (int j = 0; j < 4; j++)
            lift_inv64r(v[16 * k + 4 * j], v[16 * k + 4 * j + 1], v[16 * k + 4 * j + 2], v[16 * k + 4 * j + 3]);
}

// Shared memory of one warp: the 64 bit planes ([plane][lane]) and the stream
// tile ([64-bit word][lane], rate words and two zero words).
__host__ __device__ constexpr size_t f64_smem_bytes(int rate) { return (size_t)(64 + rate + 2) * 32 * 8; }

__global__ void __launch_bounds__(32, kF64MinCtas) encode_f64_kernel(const double *__restrict__ src,
                                                                     uint8_t *__restrict__ out, Geom64 g)
{
    extern __shared__ uint64_t sm64[];
    uint64_t *stile = sm64 + 64 * 32;
    const int lane = threadIdx.x;
    SmemPlanes pl{sm64, lane};
    constexpr int kSeq[64] = ZFPX_SEQ3;
    for (int64_t u = blockIdx.x; u < g.nunits; u += gridDim.x) {
        const int64_t b0 = u * 32;
        const int nact = (int)min((int64_t)32, g.nblocks - b0);
        if (lane < nact) {
            int64_t x0, y0, z0;
            block_origin(g, b0 + lane, x0, y0, z0);
            int64_t v[64];
            if (g.vec && x0 + 4 <= g.n[0] && y0 + 4 <= g.n[1] && z0 + 4 <= g.n[2]) {
                // an interior block: two 16-byte loads per row
#pragma unroll
                for (int k = 0; k < 4; k++)
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        const double2 *row = reinterpret_cast<const double2 *>(src + (z0 + k) * g.s[2] +
                                                                               (y0 + j) * g.s[1] + x0);
                        const double2 a = __ldg(row), b = __ldg(row + 1);
                        v[16 * k + 4 * j] = __double_as_longlong(a.x);
                        v[16 * k + 4 * j + 1] = __double_as_longlong(a.y);
                        v[16 * k + 4 * j + 2] = __double_as_longlong(b.x);
                        v[16 * k + 4 * j + 3] = __double_as_longlong(b.y);
                    }
            } else {
                // edge blocks and other layouts: element loads, the last row, level
                // and point repeated past the array's end, through a local array
                // kept rolled so the hot path's code stays compact
                int64_t t[64];
#pragma unroll 1
                for (int r = 0; r < 64; r++) {
                    const int i = r & 3, j = (r >> 2) & 3, k = r >> 4;
                    t[r] = __double_as_longlong(__ldg(src + min(z0 + k, g.n[2] - 1) * g.s[2] +
                                                      min(y0 + j, g.n[1] - 1) * g.s[1] +
                                                      min(x0 + i, g.n[0] - 1) * g.s[0]));
                }
#pragma unroll
                for (int r = 0; r < 64; r++) v[r] = t[r];
            }
            uint64_t amax = 0;
#pragma unroll
            for (int r = 0; r < 64; r++) {
                const uint64_t a = (uint64_t)v[r] & 0x7fffffffffffffffull;
                amax = a > amax ? a : amax;
            }
            const int e = block_exponent(amax);
            VarWriter wr{stile, 0ull, 0, 0, lane, g.rate};
            if (!e) {
                wr.finish();
            } else {
#pragma unroll
                for (int r = 0; r < 64; r++) v[r] = quantize64((uint64_t)v[r], e);
                xform3_fwd64(v);
#pragma unroll
                for (int r = 0; r < 64; r++) v[r] = (int64_t)(((uint64_t)v[r] + kNega64) ^ kNega64);
                // the 64 planes by quadrant: bits 32 hb .. 32 hb + 31 of the
                // coefficients 32 ch .. 32 ch + 31 in coding order.  The loop over
                // ch stays rolled (a select picks the coefficient): half the code
                // of four unrolled quadrants, which the instruction cache holds
                // better beside the unrolled lifting
#pragma unroll
                for (int hb = 0; hb < 2; hb++)
#pragma unroll 1
                    for (int ch = 0; ch < 2; ch++) {
                        uint32_t w[32];
#pragma unroll
                        for (int t = 0; t < 32; t++)
                            w[t] = (uint32_t)((uint64_t)(ch ? v[kSeq[32 + t]] : v[kSeq[t]]) >> (32 * hb));
                        transpose32(w);
#pragma unroll
                        for (int k = 0; k < 32; k++) pl.store_half(32 * hb + k, ch, w[k]);
                    }
                wr.put(1ull | ((uint64_t)e << 1), 12);
                int n = 0, R = 64 * g.rate - 12;
#pragma unroll 1
                for (int k = 63; k >= 0 && R > 0; k--) code_plane<64>(wr, pl.load(k), n, R);
                wr.finish();
            }
        }
        __syncwarp();
        uint64_t *dst = reinterpret_cast<uint64_t *>(out) + b0 * g.rate;
        for (int idx = lane; idx < nact * g.rate; idx += 32) dst[idx] = stile[(idx % g.rate) * 32 + idx / g.rate];
        __syncwarp();
    }
}

// x = q 2^(e_max - 62) rounded once to nearest even, e_max = e - 1023 (every
// exponent; the kernels take dequantize64_normal where it applies).
__device__ __forceinline__ double dequantize64(int64_t q, int e)
{
    const int s = e - 1023 - 62;                                 // x = q 2^s
    if (s >= -1022 || q == 0) {
        // (double)q rounds once; the scaling by 2^s is exact while the result
        // is normal, which holds for every q != 0 once s >= -1022
        const int s1 = s < -600 ? -600 : s;
        return (__ll2double_rn(q) * __longlong_as_double((long long)(s1 + 1023) << 52)) *
               __longlong_as_double((long long)(s - s1 + 1023) << 52);
    }
    const uint64_t a = q < 0 ? 0ull - (uint64_t)q : (uint64_t)q;
    const uint64_t sign = q < 0 ? 0x8000000000000000ull : 0ull;
    // normal result: a 2^s >= 2^-1022, i.e. a >= 2^(-1022 - s)
    const int t = -1022 - s;                                     // >= 1 here
    if (t < 64 && a >= (1ull << t)) {
        const int s1 = s < -600 ? -600 : s;
        const double r = (__ull2double_rn(a) * __longlong_as_double((long long)(s1 + 1023) << 52)) *
                         __longlong_as_double((long long)(s - s1 + 1023) << 52);
        return sign ? -r : r;
    }
    // subnormal: a 2^(s + 1074) units of 2^-1074, rounded to nearest even
    const int u = s + 1074;
    uint64_t m;
    if (u >= 0) {
        m = a << u;                                              // a < 2^(t) so this stays below 2^52
    } else {
        const int d = -u;
        if (d >= 64) {
            m = 0;                                               // below half the smallest subnormal
        } else {
            const uint64_t lo = a & ((1ull << d) - 1ull), half = 1ull << (d - 1);
            m = a >> d;
            m += (lo > half || (lo == half && (m & 1ull))) ? 1ull : 0ull;
        }
    }
    return __longlong_as_double((long long)(m | sign));
}

__global__ void __launch_bounds__(32, kF64MinCtas) decode_f64_kernel(const uint8_t *__restrict__ in,
                                                                     double *__restrict__ dst, Geom64 g)
{
    extern __shared__ uint64_t sm64[];
    uint64_t *tile = sm64 + 64 * 32;
    const int lane = threadIdx.x;
    const Tile64 st{tile, lane};
    SmemPlanes pl{sm64, lane};
    constexpr int kSeq[64] = ZFPX_SEQ3;
    for (int64_t u = blockIdx.x; u < g.nunits; u += gridDim.x) {
        const int64_t b0 = u * 32;
        const int nact = (int)min((int64_t)32, g.nblocks - b0);
        if (lane >= nact) continue;
        const int64_t b = b0 + lane;
        const uint64_t *s64 = reinterpret_cast<const uint64_t *>(in) + b * g.rate;
#pragma unroll 4
        for (int i = 0; i < g.rate; i++) tile[i * 32 + lane] = __ldg(s64 + i);
        tile[g.rate * 32 + lane] = 0ull;
        tile[(g.rate + 1) * 32 + lane] = 0ull;
        int64_t x0, y0, z0;
        block_origin(g, b, x0, y0, z0);
        const uint64_t head = st.peek(0);
        double x[64];
        if (!(head & 1ull)) {
#pragma unroll
            for (int r = 0; r < 64; r++) x[r] = 0.0;
        } else {
            const int e = (int)((head >> 1) & 0x7ffu);
            // the planes from bit 12 on; the tile's two zero 64-bit words let the
            // parser read past the budget without a test
            const Tile64As32 t32{reinterpret_cast<const uint32_t *>(tile), lane};
            const int kmin = parse_planes64<true>(t32, 12, 64 * g.rate, 63, pl);
#pragma unroll 1
            for (int k = 0; k < kmin; k++) pl.store(k, 0ull);
            int64_t v[64];
#pragma unroll
            for (int hb = 0; hb < 2; hb++)
#pragma unroll
                for (int ch = 0; ch < 2; ch++) {
                    uint32_t w[32];
#pragma unroll
                    for (int k = 0; k < 32; k++) w[k] = pl.load_half(32 * hb + k, ch);
                    transpose32(w);
                    // w[t] = bits 32 hb .. 32 hb + 31 of coefficient 32 ch + t
#pragma unroll
                    for (int t = 0; t < 32; t++) {
                        int64_t &c = v[kSeq[32 * ch + t]];
                        c = hb ? (int64_t)(((uint64_t)c & 0xffffffffull) | ((uint64_t)w[t] << 32)) : (int64_t)w[t];
                    }
                }
#pragma unroll
            for (int r = 0; r < 64; r++) v[r] = sub64((int64_t)((uint64_t)v[r] ^ kNega64), (int64_t)kNega64);
            xform3_inv64(v);
            if (e >= 63) {
#pragma unroll
                for (int r = 0; r < 64; r++) x[r] = dequantize64_normal(v[r], e);
            } else {
                // tiny exponents (rare): a rolled loop over a local copy
                int64_t t[64];
#pragma unroll
                for (int r = 0; r < 64; r++) t[r] = v[r];
#pragma unroll 1
                for (int r = 0; r < 64; r++) t[r] = __double_as_longlong(dequantize64(t[r], e));
#pragma unroll
                for (int r = 0; r < 64; r++) x[r] = __longlong_as_double(t[r]);
            }
        }
        if (g.vec && x0 + 4 <= g.n[0] && y0 + 4 <= g.n[1] && z0 + 4 <= g.n[2]) {
            // an interior block: two 16-byte stores per row
#pragma unroll
            for (int k = 0; k < 4; k++)
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    double2 *row = reinterpret_cast<double2 *>(dst + (z0 + k) * g.s[2] + (y0 + j) * g.s[1] + x0);
                    row[0] = make_double2(x[16 * k + 4 * j], x[16 * k + 4 * j + 1]);
                    row[1] = make_double2(x[16 * k + 4 * j + 2], x[16 * k + 4 * j + 3]);
                }
        } else {
            // edge blocks and other layouts: element stores inside the array,
            // through a local array kept rolled
            double t[64];
#pragma unroll
            for (int r = 0; r < 64; r++) t[r] = x[r];
#pragma unroll 1
            for (int r = 0; r < 64; r++) {
                const int i = r & 3, j = (r >> 2) & 3, k = r >> 4;
                if (x0 + i < g.n[0] && y0 + j < g.n[1] && z0 + k < g.n[2])
                    dst[(z0 + k) * g.s[2] + (y0 + j) * g.s[1] + (x0 + i) * g.s[0]] = t[r];
            }
        }
    }
}

Geom64 make_geom(const int64_t n[3], const int64_t s[3], int rate, const void *base)
{
    Geom64 g;
    g.vec = s[0] == 1 && s[1] % 2 == 0 && s[2] % 2 == 0 && !((uintptr_t)base & 15u);
    for (int a = 0; a < 3; a++) { g.n[a] = n[a]; g.s[a] = s[a]; }
    g.bx = (n[0] + 3) / 4; g.by = (n[1] + 3) / 4;
    g.nblocks = g.bx * g.by * ((n[2] + 3) / 4);
    g.nunits = (g.nblocks + 31) / 32;
    g.rate = rate;
    return g;
}

unsigned grid_f64(const void *fn, int64_t nunits, size_t smem)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32, smem) != cudaSuccess || per_sm < 1) per_sm = 1;
    const int64_t cap = (int64_t)num_sms() * per_sm;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(nunits, cap));
}

// Dynamic shared memory above 48 KB is opted into per kernel.
int f64_prepare(const void *fn, size_t smem)
{
    if (smem <= 48 * 1024) return ZFPX_OK;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess
               ? ZFPX_OK : ZFPX_ECUDA;
}

bool valid_f64_args(int rate, const int64_t n[3], const int64_t stride[3])
{
    if (rate < 1 || rate > kMaxRate || !n || !stride) return false;
    for (int a = 0; a < 3; a++) if (n[a] < 1 || stride[a] < 0) return false;
    return true;
}

}  // namespace
}  // namespace zfpx

using namespace zfpx;

extern "C" {

size_t zfpx_stream_bytes_f64(int rate, const int64_t n[3])
{
    if (!n || rate < 1 || rate > kMaxRate) return 0;
    for (int a = 0; a < 3; a++) if (n[a] < 1) return 0;
    return (size_t)(((n[0] + 3) / 4) * ((n[1] + 3) / 4) * ((n[2] + 3) / 4) * 8 * rate);
}

int zfpx_encode_f64(int rate, const double *d_in, const int64_t n[3], const int64_t stride[3], uint8_t *d_out,
                    size_t cap, void *stream)
{
    if (!d_in || !d_out || !valid_f64_args(rate, n, stride)) return ZFPX_EINVAL;
    if (((uintptr_t)d_out & 7u) || ((uintptr_t)d_in & 7u)) return ZFPX_EINVAL;
    if (cap < zfpx_stream_bytes_f64(rate, n)) return ZFPX_ESIZE;
    const Geom64 g = make_geom(n, stride, rate, d_in);
    const size_t smem = f64_smem_bytes(rate);
    const int rc = f64_prepare((const void *)encode_f64_kernel, smem);
    if (rc) return rc;
    encode_f64_kernel<<<grid_f64((const void *)encode_f64_kernel, g.nunits, smem), 32, smem, (cudaStream_t)stream>>>(
        d_in, d_out, g);
    count_launch();
    return check_launch();
}

int zfpx_decode_f64(int rate, const uint8_t *d_in, size_t len, const int64_t n[3], const int64_t stride[3],
                    double *d_out, void *stream)
{
    if (!d_in || !d_out || !valid_f64_args(rate, n, stride)) return ZFPX_EINVAL;
    if (((uintptr_t)d_out & 7u) || ((uintptr_t)d_in & 7u)) return ZFPX_EINVAL;
    if (len < zfpx_stream_bytes_f64(rate, n)) return ZFPX_ESIZE;
    const Geom64 g = make_geom(n, stride, rate, d_out);
    const size_t smem = f64_smem_bytes(rate);
    const int rc = f64_prepare((const void *)decode_f64_kernel, smem);
    if (rc) return rc;
    decode_f64_kernel<<<grid_f64((const void *)decode_f64_kernel, g.nunits, smem), 32, smem, (cudaStream_t)stream>>>(
        d_in, d_out, g);
    count_launch();
    return check_launch();
}

}  // extern "C"
