/*
 * zfp_oracle.c -- TEST INFRASTRUCTURE, not part of the product path.
 *
 * A plain, slow, scalar CPU statement of ZFP fixed-rate coding of float32
 * blocks, written step by step from the method the paper uses (Sec. II-C:
 * the array is cut into disjoint 4^d blocks, each decorrelated by a lifting
 * transform and then reduced in precision; fixed-rate mode spends exactly r
 * bits per value, Sec. II-C and Sec. IV-B, ZFP 1.0.1) and from the cited published method
 * (Lindstrom 2014, the paper's reference for ZFP).  Where both are silent the
 * reading used is stated at the step below.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference
 * leg may load this library.  It shares no code, header, table or constant
 * with the CUDA library; neither includes the other.
 *
 * Every function is deliberately unoptimised: one bit at a time, one block at
 * a time, exact integer arithmetic in int64 with an explicit wrap to int32
 * (the method's integer type) and an overflow counter, so that a reader can
 * check each step against the method by eye.
 *
 * Parity status: every function here is pinned by tests/test_oracle_*.py
 * (closed forms, the published transform matrix, hand-derived golden
 * streams, brute force and invariants).  Byte compatibility with the zfp
 * 1.0.1 library itself is NOT pinned (no zfp build is available); the
 * readings at the steps below decide where the method leaves a choice.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------------ */
/* Overflow accounting: every lifting result that would not fit int32.       */
/* ------------------------------------------------------------------------ */
static long long g_overflow = 0;
long long zfpo_overflow_count(void) { return g_overflow; }
void zfpo_overflow_reset(void) { g_overflow = 0; }

/* Wrap an exact integer to int32 (two's complement), counting any change. */
static int64_t wrap32(int64_t v)
{
    int64_t w = (int64_t)(int32_t)(uint32_t)(uint64_t)v;
    if (w != v) g_overflow++;
    return w;
}

/* floor(v / 2) for any sign: (v - (v mod 2)) / 2 with v mod 2 in {0, 1}. */
static int64_t floor_half(int64_t v) { return (v - (v & 1)) / 2; }

/* ------------------------------------------------------------------------ */
/* Bit stream.  Bit p of a stream is bit (p % 8) of byte (p / 8): the same   */
/* thing as writing LSB-first into little-endian 64-bit words.               */
/* ------------------------------------------------------------------------ */
typedef struct { uint8_t *buf; uint64_t pos; } bitw;   /* writer; buf zeroed */
typedef struct { const uint8_t *buf; uint64_t pos; } bitr;

static void put_bit(bitw *w, unsigned b)
{
    if (w->buf && b) w->buf[w->pos >> 3] |= (uint8_t)(1u << (w->pos & 7));
    w->pos++;
}
static unsigned get_bit(bitr *r)
{
    unsigned b = (r->buf[r->pos >> 3] >> (r->pos & 7)) & 1u;
    r->pos++;
    return b;
}

/* ------------------------------------------------------------------------ */
/* Step 4: decorrelating transform.                                          */
/* The published real-valued 4-point transform (Lindstrom 2014) is           */
/*     (1/16) [[ 4, 4, 4, 4], [ 5, 1,-1,-5], [-4, 4, 4,-4], [-2, 6,-6, 2]].  */
/* It is applied as five lifting steps.  Written with exact halving they     */
/* give that matrix exactly (derivation, for input (a,b,c,d)):               */
/*   L1: a' = (a+d)/2,            d' = (d-a)/2                               */
/*   L2: c' = (c+b)/2,            b' = (b-c)/2                               */
/*   L3: a''= (a+b+c+d)/4,        c''= (-a+b+c-d)/4                          */
/*   L4: d''= (-a+b-c+d)/4,       b''= (a+b-c-d)/4                           */
/*   L5: d  = d''+b''/2 = (-a+3b-3c+d)/8,  b = b''-d/2 = (5a+b-c-5d)/16      */
/* giving (a'', b, c'', d) = rows 1..4 of the matrix.  In integers every      */
/* halving is a floor, which is why the transform is only nearly reversible. */
/* The same five steps are instantiated twice: on exact doubles (used only   */
/* by the test that checks the matrix) and on integers (the codec).          */
/* ------------------------------------------------------------------------ */
#define LIFT_FORWARD(a, b, c, d, HALF)                                        \
    do {                                                                      \
        a = HALF(a + d); d = d - a;                 /* L1 */                  \
        c = HALF(c + b); b = b - c;                 /* L2 */                  \
        a = HALF(a + c); c = c - a;                 /* L3 */                  \
        d = HALF(d + b); b = b - d;                 /* L4 */                  \
        d = d + HALF(b); b = b - HALF(d);           /* L5 */                  \
    } while (0)

/* Undo L5, L4, L3, L2, L1 in that order.  L5 is undone exactly; L1..L4 lose
 * the floor's discarded bit (a = 2a' - d restores a only up to that bit). */
#define LIFT_INVERSE(a, b, c, d, HALF)                                        \
    do {                                                                      \
        b = b + HALF(d); d = d - HALF(b);           /* undo L5 */             \
        b = b + d; d = 2 * d - b;                   /* undo L4 */             \
        c = c + a; a = 2 * a - c;                   /* undo L3 */             \
        b = b + c; c = 2 * c - b;                   /* undo L2 */             \
        d = d + a; a = 2 * a - d;                   /* undo L1 */             \
    } while (0)

#define EXACT_HALF(v) ((v) * 0.5)
#define INT_HALF(v) floor_half(wrap32(v))

void zfpo_lift_forward_exact(double v[4])
{
    double a = v[0], b = v[1], c = v[2], d = v[3];
    LIFT_FORWARD(a, b, c, d, EXACT_HALF);
    v[0] = a; v[1] = b; v[2] = c; v[3] = d;
}
void zfpo_lift_inverse_exact(double v[4])
{
    double a = v[0], b = v[1], c = v[2], d = v[3];
    LIFT_INVERSE(a, b, c, d, EXACT_HALF);
    v[0] = a; v[1] = b; v[2] = c; v[3] = d;
}

/* Integer lifting on int32 values: every sum is formed exactly, then wrapped
 * to int32 (counted by the overflow counter) before it is halved or stored. */
static void lift_forward_int(int32_t *p, ptrdiff_t s)
{
    int64_t a = p[0], b = p[s], c = p[2 * s], d = p[3 * s];
    LIFT_FORWARD(a, b, c, d, INT_HALF);
    p[0] = (int32_t)wrap32(a); p[s] = (int32_t)wrap32(b);
    p[2 * s] = (int32_t)wrap32(c); p[3 * s] = (int32_t)wrap32(d);
}
static void lift_inverse_int(int32_t *p, ptrdiff_t s)
{
    int64_t a = p[0], b = p[s], c = p[2 * s], d = p[3 * s];
    LIFT_INVERSE(a, b, c, d, INT_HALF);
    p[0] = (int32_t)wrap32(a); p[s] = (int32_t)wrap32(b);
    p[2 * s] = (int32_t)wrap32(c); p[3 * s] = (int32_t)wrap32(d);
}

/* Note on the integer instantiation: every intermediate of LIFT_* is an
 * exact int64; INT_HALF wraps the value it halves, and the final stores wrap
 * again.  For blocks of finite float32 input the values never leave int32
 * (pinned by tests), so this equals plain int32 arithmetic. */

void zfpo_lift_forward(int32_t v[4]) { lift_forward_int(v, 1); }
void zfpo_lift_inverse(int32_t v[4]) { lift_inverse_int(v, 1); }

/* Separable transform of a block q[i + 4j + 16k]: along axis 0 (i) for every
 * line, then axis 1 (j), then axis 2 (k).  The inverse runs axes 2, 1, 0.
 * A 2-D block q[i + 4j] has the first two axes only. */
void zfpo_xform_forward(int dims, int32_t *q)
{
    if (dims == 1) { lift_forward_int(q, 1); return; }
    if (dims == 2) {
        for (int j = 0; j < 4; j++) lift_forward_int(q + 4 * j, 1);
        for (int i = 0; i < 4; i++) lift_forward_int(q + i, 4);
        return;
    }
    for (int k = 0; k < 4; k++)
        for (int j = 0; j < 4; j++) lift_forward_int(q + 4 * j + 16 * k, 1);
    for (int k = 0; k < 4; k++)
        for (int i = 0; i < 4; i++) lift_forward_int(q + i + 16 * k, 4);
    for (int j = 0; j < 4; j++)
        for (int i = 0; i < 4; i++) lift_forward_int(q + i + 4 * j, 16);
}
void zfpo_xform_inverse(int dims, int32_t *q)
{
    if (dims == 1) { lift_inverse_int(q, 1); return; }
    if (dims == 2) {
        for (int i = 0; i < 4; i++) lift_inverse_int(q + i, 4);
        for (int j = 0; j < 4; j++) lift_inverse_int(q + 4 * j, 1);
        return;
    }
    for (int j = 0; j < 4; j++)
        for (int i = 0; i < 4; i++) lift_inverse_int(q + i + 4 * j, 16);
    for (int k = 0; k < 4; k++)
        for (int i = 0; i < 4; i++) lift_inverse_int(q + i + 16 * k, 4);
    for (int k = 0; k < 4; k++)
        for (int j = 0; j < 4; j++) lift_inverse_int(q + 4 * j + 16 * k, 1);
}

/* ------------------------------------------------------------------------ */
/* Step 5: sequency order.  Coefficient (i,j,k) of a 3-D block is ranked by  */
/* total sequency i+j+k; ties by i*i+j*j+k*k; then by i + 4j + 16k (reading). */
/* A 2-D block is the same rule with k = 0.  1-D blocks keep their order.    */
/* ------------------------------------------------------------------------ */
void zfpo_sequency_order(int dims, int *order /* [4^dims] */)
{
    int S = 1 << (2 * dims);
    for (int t = 0; t < S; t++) order[t] = t;
    if (dims == 1) return;
    /* insertion sort on the key; plain and small */
    for (int a = 1; a < S; a++) {
        int v = order[a], b = a - 1;
        int vi = v & 3, vj = (v >> 2) & 3, vk = v >> 4;
        long vkey = (long)(vi + vj + vk) * 100000 + (vi * vi + vj * vj + vk * vk) * 100 + v;
        while (b >= 0) {
            int w = order[b];
            int wi = w & 3, wj = (w >> 2) & 3, wk = w >> 4;
            long wkey = (long)(wi + wj + wk) * 100000 + (wi * wi + wj * wj + wk * wk) * 100 + w;
            if (wkey <= vkey) break;
            order[b + 1] = w;
            b--;
        }
        order[b + 1] = v;
    }
}

/* ------------------------------------------------------------------------ */
/* Step 6: negabinary.  u = (q + 0xAAAAAAAA) xor 0xAAAAAAAA modulo 2^32, so   */
/* that bit k of u carries weight (-2)^k.                                     */
/* ------------------------------------------------------------------------ */
uint32_t zfpo_to_negabinary(int32_t q)
{
    return ((uint32_t)q + 0xAAAAAAAAu) ^ 0xAAAAAAAAu;
}
int32_t zfpo_from_negabinary(uint32_t u)
{
    return (int32_t)((u ^ 0xAAAAAAAAu) - 0xAAAAAAAAu);
}

/* ------------------------------------------------------------------------ */
/* Step 7: embedded bit-plane coding with group testing, one plane.          */
/* State n = number of leading coefficients already known significant.      */
/*  (i)  the bits of coefficients 0..n-1 are sent as they are;               */
/*  (ii) then repeatedly: send G = [some coefficient >= n has a 1 here].     */
/*       G = 0 ends the plane.  G = 1: send the bits of n, n+1, ... until a  */
/*       1 is sent; the last coefficient's 1 is implied (not sent) when it   */
/*       is the only one left.  That coefficient becomes significant.        */
/* Every sent bit spends one unit of *budget; at zero the plane stops.       */
/* Returns 0 when the plane completed, 1 when the budget ran out.            */
/* ------------------------------------------------------------------------ */
static int code_plane(bitw *w, int S, const unsigned *X, int *n_io, uint64_t *budget)
{
    int n = *n_io;
    int stopped = 0;
    for (int i = 0; i < n; i++) {
        if (*budget == 0) { stopped = 1; goto out; }
        put_bit(w, X[i]); (*budget)--;
    }
    while (n < S) {
        unsigned G = 0;
        if (*budget == 0) { stopped = 1; goto out; }
        for (int i = n; i < S; i++) G |= X[i];
        put_bit(w, G); (*budget)--;
        if (!G) break;
        while (n < S - 1) {
            if (*budget == 0) { stopped = 1; goto out; }
            put_bit(w, X[n]); (*budget)--;
            if (X[n]) break;
            n++;
        }
        n++;            /* coefficient n found (sent, or implied at S-1) */
    }
out:
    *n_io = n;
    return stopped;
}

/* Mirror of code_plane: fills X[] (zeroed by the caller). */
static int decode_plane(bitr *r, int S, unsigned *X, int *n_io, uint64_t *budget)
{
    int n = *n_io;
    int stopped = 0;
    for (int i = 0; i < n; i++) {
        if (*budget == 0) { stopped = 1; goto out; }
        X[i] = get_bit(r); (*budget)--;
    }
    while (n < S) {
        if (*budget == 0) { stopped = 1; goto out; }
        unsigned G = get_bit(r); (*budget)--;
        if (!G) break;
        while (n < S - 1) {
            if (*budget == 0) { stopped = 1; goto out; }
            unsigned b = get_bit(r); (*budget)--;
            if (b) break;
            n++;
        }
        X[n] = 1;       /* read as 1, or implied as the only one left */
        n++;
    }
out:
    *n_io = n;
    return stopped;
}

/* Test hook: bits one full plane costs with an unlimited budget. */
int zfpo_plane_bits(int S, uint64_t plane, int n_in, int *n_out)
{
    unsigned X[64];
    for (int i = 0; i < S; i++) X[i] = (unsigned)((plane >> i) & 1u);
    bitw w = {NULL, 0};
    uint64_t budget = UINT64_MAX;
    int n = n_in;
    code_plane(&w, S, X, &n, &budget);
    if (n_out) *n_out = n;
    return (int)w.pos;
}

/* Code planes 31..0 of u[0..S-1] into at most `budget` bits. */
static uint64_t encode_planes(bitw *w, int S, const uint32_t *u, uint64_t budget)
{
    uint64_t left = budget;
    int n = 0;
    for (int k = 31; k >= 0; k--) {
        unsigned X[64];
        for (int i = 0; i < S; i++) X[i] = (u[i] >> k) & 1u;
        if (code_plane(w, S, X, &n, &left)) break;
        if (left == 0) break;
    }
    return budget - left;
}
static uint64_t decode_planes(bitr *r, int S, uint32_t *u, uint64_t budget)
{
    uint64_t left = budget;
    int n = 0;
    for (int i = 0; i < S; i++) u[i] = 0;
    for (int k = 31; k >= 0; k--) {
        unsigned X[64];
        for (int i = 0; i < S; i++) X[i] = 0;
        int stopped = decode_plane(r, S, X, &n, &left);
        for (int i = 0; i < S; i++) u[i] |= (uint32_t)X[i] << k;
        if (stopped || left == 0) break;
    }
    return budget - left;
}

/* Test hooks over whole coefficient sets (u in coding order). */
uint64_t zfpo_encode_planes(int S, const uint32_t *u, uint64_t budget, uint8_t *out /* zeroed */)
{
    bitw w = {out, 0};
    return encode_planes(&w, S, u, budget);
}
uint64_t zfpo_decode_planes(int S, const uint8_t *in, uint64_t budget, uint32_t *u)
{
    bitr r = {in, 0};
    return decode_planes(&r, S, u, budget);
}

/* ------------------------------------------------------------------------ */
/* Steps 1-8 on one block of 4^dims float32 values v[i + 4j + 16k].          */
/* ------------------------------------------------------------------------ */
static int valid_rate(int dims, int rate)
{
    if (dims < 1 || dims > 3) return 0;
    if (rate < 1 || rate > 32) return 0;
    if (dims == 1 && rate < 3) return 0;   /* 4*rate must exceed the 9-bit header */
    return 1;
}

static void encode_block(bitw *w, int dims, int rate, const float *v)
{
    const int S = 1 << (2 * dims);
    const uint64_t maxbits = (uint64_t)S * (uint64_t)rate;   /* step 1 */
    const uint64_t start = w->pos;

    /* step 2: common exponent of the largest magnitude */
    double M = 0.0;
    for (int i = 0; i < S; i++) {
        double a = fabs((double)v[i]);
        if (a > M || a != a) M = a;                 /* NaN propagates */
    }
    int emax = 0;
    int zero = 1;
    if (M > 0.0 && isfinite(M)) {
        (void)frexp(M, &emax);                     /* M = f 2^emax, f in [0.5,1) */
        zero = (emax + 127 <= 0);                  /* reading: max below 2^-127 -> zero block */
    }
    if (zero) {
        /* reading: non-finite maxima are coded as a zero block too */
        put_bit(w, 0);
        w->pos = start + maxbits;                  /* zero fill */
        return;
    }
    put_bit(w, 1);
    unsigned e = (unsigned)(emax + 127);
    for (int b = 0; b < 8; b++) put_bit(w, (e >> b) & 1u);

    /* step 3: block floating point, q = trunc(x * 2^(30 - emax)) */
    int32_t q[64];
    for (int i = 0; i < S; i++) {
        double y = ldexp((double)v[i], 30 - emax);  /* exact */
        q[i] = (int32_t)y;                          /* C cast truncates toward 0 */
    }
    /* step 4 */
    zfpo_xform_forward(dims, q);
    /* steps 5 and 6 */
    int order[64];
    zfpo_sequency_order(dims, order);
    uint32_t u[64];
    for (int t = 0; t < S; t++) u[t] = zfpo_to_negabinary(q[order[t]]);
    /* step 7 */
    encode_planes(w, S, u, maxbits - 9);
    w->pos = start + maxbits;                       /* zero fill to exactly maxbits */
}

static void decode_block(bitr *r, int dims, int rate, float *v)
{
    const int S = 1 << (2 * dims);
    const uint64_t maxbits = (uint64_t)S * (uint64_t)rate;
    const uint64_t start = r->pos;
    if (!get_bit(r)) {
        for (int i = 0; i < S; i++) v[i] = 0.0f;
        r->pos = start + maxbits;
        return;
    }
    unsigned e = 0;
    for (int b = 0; b < 8; b++) e |= get_bit(r) << b;
    int emax = (int)e - 127;

    uint32_t u[64];
    decode_planes(r, S, u, maxbits - 9);            /* missing bits are 0 */
    int order[64];
    zfpo_sequency_order(dims, order);
    int32_t q[64];
    for (int t = 0; t < S; t++) q[order[t]] = zfpo_from_negabinary(u[t]);
    zfpo_xform_inverse(dims, q);
    for (int i = 0; i < S; i++)
        v[i] = (float)ldexp((double)q[i], emax - 30);   /* one rounding, to nearest even */
    r->pos = start + maxbits;
}

int zfpo_encode_block(int dims, int rate, const float *v, uint8_t *out /* zeroed */)
{
    if (!valid_rate(dims, rate)) return -1;
    bitw w = {out, 0};
    encode_block(&w, dims, rate, v);
    return 0;
}
int zfpo_decode_block(int dims, int rate, const uint8_t *in, float *v)
{
    if (!valid_rate(dims, rate)) return -1;
    bitr r = {in, 0};
    decode_block(&r, dims, rate, v);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Arrays.  A box of extent n[0] x n[1] x n[2] (axis 0 fastest) is read      */
/* through element strides s[0..2].  dims == 3: 4x4x4 blocks; dims == 2: 4x4 */
/* blocks over axes 0 and 1, each axis-2 slice on its own; dims == 1:        */
/* 4-value blocks along axis 0.  Blocks are stored back to back in raster    */
/* order of block indices, axis 0 fastest.  A partial block is completed by  */
/* repeating the last value along each short axis (reading); the repeated    */
/* values are coded and dropped again on decode.                            */
/* ------------------------------------------------------------------------ */
static int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

int64_t zfpo_block_count(int dims, const int64_t n[3])
{
    if (dims == 1) return ((n[0] + 3) / 4) * n[1] * n[2];
    if (dims == 2) return ((n[0] + 3) / 4) * ((n[1] + 3) / 4) * n[2];
    return ((n[0] + 3) / 4) * ((n[1] + 3) / 4) * ((n[2] + 3) / 4);
}
int64_t zfpo_stream_bytes(int dims, int rate, const int64_t n[3])
{
    int S = 1 << (2 * dims);
    int64_t bits = zfpo_block_count(dims, n) * S * rate;
    return (bits + 7) / 8;
}

int zfpo_encode_array(int dims, int rate, const float *base, const int64_t n[3],
                      const int64_t s[3], uint8_t *out, int64_t out_bytes)
{
    if (!valid_rate(dims, rate)) return -1;
    if (n[0] < 1 || n[1] < 1 || n[2] < 1) return 0;
    if (out_bytes < zfpo_stream_bytes(dims, rate, n)) return -2;
    memset(out, 0, (size_t)zfpo_stream_bytes(dims, rate, n));
    bitw w = {out, 0};
    float v[64];
    int64_t bx = (n[0] + 3) / 4;
    if (dims == 3) {
        int64_t by = (n[1] + 3) / 4, bz = (n[2] + 3) / 4;
        for (int64_t zb = 0; zb < bz; zb++)
            for (int64_t yb = 0; yb < by; yb++)
                for (int64_t xb = 0; xb < bx; xb++) {
                    for (int k = 0; k < 4; k++)
                        for (int j = 0; j < 4; j++)
                            for (int i = 0; i < 4; i++) {
                                int64_t x = imin64(4 * xb + i, n[0] - 1);
                                int64_t y = imin64(4 * yb + j, n[1] - 1);
                                int64_t z = imin64(4 * zb + k, n[2] - 1);
                                v[i + 4 * j + 16 * k] = base[x * s[0] + y * s[1] + z * s[2]];
                            }
                    encode_block(&w, 3, rate, v);
                }
    } else if (dims == 2) {
        int64_t by = (n[1] + 3) / 4;
        for (int64_t z = 0; z < n[2]; z++)
            for (int64_t yb = 0; yb < by; yb++)
                for (int64_t xb = 0; xb < bx; xb++) {
                    for (int j = 0; j < 4; j++)
                        for (int i = 0; i < 4; i++) {
                            int64_t x = imin64(4 * xb + i, n[0] - 1);
                            int64_t y = imin64(4 * yb + j, n[1] - 1);
                            v[i + 4 * j] = base[x * s[0] + y * s[1] + z * s[2]];
                        }
                    encode_block(&w, 2, rate, v);
                }
    } else {
        for (int64_t z = 0; z < n[2]; z++)
            for (int64_t y = 0; y < n[1]; y++)
                for (int64_t xb = 0; xb < bx; xb++) {
                    for (int i = 0; i < 4; i++) {
                        int64_t x = imin64(4 * xb + i, n[0] - 1);
                        v[i] = base[x * s[0] + y * s[1] + z * s[2]];
                    }
                    encode_block(&w, 1, rate, v);
                }
    }
    return 0;
}

int zfpo_decode_array(int dims, int rate, const uint8_t *in, const int64_t n[3],
                      float *base, const int64_t s[3])
{
    if (!valid_rate(dims, rate)) return -1;
    if (n[0] < 1 || n[1] < 1 || n[2] < 1) return 0;
    bitr r = {in, 0};
    float v[64];
    int64_t bx = (n[0] + 3) / 4;
    if (dims == 3) {
        int64_t by = (n[1] + 3) / 4, bz = (n[2] + 3) / 4;
        for (int64_t zb = 0; zb < bz; zb++)
            for (int64_t yb = 0; yb < by; yb++)
                for (int64_t xb = 0; xb < bx; xb++) {
                    decode_block(&r, 3, rate, v);
                    for (int k = 0; k < 4; k++)
                        for (int j = 0; j < 4; j++)
                            for (int i = 0; i < 4; i++) {
                                int64_t x = 4 * xb + i, y = 4 * yb + j, z = 4 * zb + k;
                                if (x < n[0] && y < n[1] && z < n[2])
                                    base[x * s[0] + y * s[1] + z * s[2]] = v[i + 4 * j + 16 * k];
                            }
                }
    } else if (dims == 2) {
        int64_t by = (n[1] + 3) / 4;
        for (int64_t z = 0; z < n[2]; z++)
            for (int64_t yb = 0; yb < by; yb++)
                for (int64_t xb = 0; xb < bx; xb++) {
                    decode_block(&r, 2, rate, v);
                    for (int j = 0; j < 4; j++)
                        for (int i = 0; i < 4; i++) {
                            int64_t x = 4 * xb + i, y = 4 * yb + j;
                            if (x < n[0] && y < n[1]) base[x * s[0] + y * s[1] + z * s[2]] = v[i + 4 * j];
                        }
                }
    } else {
        for (int64_t z = 0; z < n[2]; z++)
            for (int64_t y = 0; y < n[1]; y++)
                for (int64_t xb = 0; xb < bx; xb++) {
                    decode_block(&r, 1, rate, v);
                    for (int i = 0; i < 4; i++) {
                        int64_t x = 4 * xb + i;
                        if (x < n[0]) base[x * s[0] + y * s[1] + z * s[2]] = v[i];
                    }
                }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Variable-rate coding to an absolute error tolerance (3-D blocks).  The   */
/* paper names ZFP's accuracy mode and leaves it for future work (Sec.      */
/* II-C); the readings here:                                                 */
/*   minexp = floor(log2 tol); a block with exponent e_max codes its bit     */
/*   planes from 31 down to kmin = clamp(minexp - e_max + 22, 0, 32), with   */
/*   the same header, transform, order and group-tested coder as the fixed-  */
/*   rate mode, and at most 16 * 64 = 1024 bits (the rate-16 budget: a block */
/*   whose planes do not fit is cut there).  Dropping planes below kmin      */
/*   changes a coefficient by less than 2^kmin; the inverse transform's gain */
/*   is below 2^6 and its rounding adds a few units, so the reconstruction   */
/*   error stays below 2^(kmin + 7) * 2^(e_max - 30) = tol / 2 for blocks    */
/*   whose kmin is not clamped at 0 and whose bits are not cut.              */
/*   Zero blocks (the fixed-rate rule) take 1 bit; a block with kmin = 32    */
/*   takes its 9 header bits and no plane.                                   */
/* Stream of an array: per block (raster order, edge-replicated partial     */
/* blocks as in the fixed-rate arrays) its bit count L in lengths[], and     */
/* the blocks' bits back to back in payload (LSB first).  A block decodes    */
/* as the rate-16 block made of its L bits followed by zeros: zero bits      */
/* after the last coded plane read as planes with nothing in them.           */
/* ------------------------------------------------------------------------ */
int zfpo_accuracy_kmin(int emax, int minexp)
{
    int k = minexp - emax + 22;
    return k < 0 ? 0 : (k > 32 ? 32 : k);
}

static uint64_t encode_planes_down_to(bitw *w, int S, const uint32_t *u, uint64_t budget, int kstop)
{
    uint64_t left = budget;
    int n = 0;
    for (int k = 31; k >= kstop; k--) {
        unsigned X[64];
        for (int i = 0; i < S; i++) X[i] = (u[i] >> k) & 1u;
        if (code_plane(w, S, X, &n, &left)) break;
        if (left == 0) break;
    }
    return budget - left;
}

/* One block's bits in accuracy mode (prec == 0) or precision mode (prec in
 * 1..32: planes 31 down to 32 - prec, the mode that keeps a fixed number of
 * bit planes per block), written at w (buffer zeroed); returns L. */
static uint64_t encode_block_accuracy(bitw *w, const float *v, int minexp, int prec)
{
    const uint64_t start = w->pos;
    double M = 0.0;
    for (int i = 0; i < 64; i++) {
        double a = fabs((double)v[i]);
        if (a > M || a != a) M = a;
    }
    int emax = 0, zero = 1;
    if (M > 0.0 && isfinite(M)) {
        (void)frexp(M, &emax);
        zero = (emax + 127 <= 0);
    }
    if (zero) { put_bit(w, 0); return 1; }
    put_bit(w, 1);
    unsigned e = (unsigned)(emax + 127);
    for (int b = 0; b < 8; b++) put_bit(w, (e >> b) & 1u);
    const int kmin = prec > 0 ? 32 - prec : zfpo_accuracy_kmin(emax, minexp);
    if (kmin < 32) {
        int32_t q[64];
        for (int i = 0; i < 64; i++) q[i] = (int32_t)ldexp((double)v[i], 30 - emax);
        zfpo_xform_forward(3, q);
        int order[64];
        zfpo_sequency_order(3, order);
        uint32_t u[64];
        for (int t = 0; t < 64; t++) u[t] = zfpo_to_negabinary(q[order[t]]);
        encode_planes_down_to(w, 64, u, 64 * 16 - 9, kmin);
    }
    return w->pos - start;
}

int zfpo_accuracy_minexp(double tol)
{
    int e = 0;
    (void)frexp(tol, &e);          /* tol = m 2^e, m in [0.5, 1): floor(log2 tol) = e - 1 */
    return e - 1;
}

int64_t zfpo_accuracy_max_payload_bytes(const int64_t n[3])
{
    return zfpo_block_count(3, n) * 128;
}

static void gather3(const float *base, const int64_t n[3], const int64_t s[3],
                    int64_t xb, int64_t yb, int64_t zb, float *v)
{
    for (int k = 0; k < 4; k++)
        for (int j = 0; j < 4; j++)
            for (int i = 0; i < 4; i++) {
                int64_t x = imin64(4 * xb + i, n[0] - 1);
                int64_t y = imin64(4 * yb + j, n[1] - 1);
                int64_t z = imin64(4 * zb + k, n[2] - 1);
                v[i + 4 * j + 16 * k] = base[x * s[0] + y * s[1] + z * s[2]];
            }
}

static int encode_variable(const float *base, const int64_t n[3], const int64_t s[3], int minexp, int prec,
                           uint16_t *lengths, uint8_t *payload, int64_t payload_bytes, uint64_t *total_bits)
{
    if (n[0] < 1 || n[1] < 1 || n[2] < 1) { *total_bits = 0; return 0; }
    if (payload_bytes < zfpo_accuracy_max_payload_bytes(n)) return -2;
    memset(payload, 0, (size_t)payload_bytes);
    bitw w = {payload, 0};
    float v[64];
    int64_t bx = (n[0] + 3) / 4, by = (n[1] + 3) / 4, bz = (n[2] + 3) / 4, b = 0;
    for (int64_t zb = 0; zb < bz; zb++)
        for (int64_t yb = 0; yb < by; yb++)
            for (int64_t xb = 0; xb < bx; xb++) {
                gather3(base, n, s, xb, yb, zb, v);
                lengths[b++] = (uint16_t)encode_block_accuracy(&w, v, minexp, prec);
            }
    *total_bits = w.pos;
    return 0;
}

int zfpo_encode_accuracy(const float *base, const int64_t n[3], const int64_t s[3], double tol,
                         uint16_t *lengths, uint8_t *payload, int64_t payload_bytes, uint64_t *total_bits)
{
    if (!(tol > 0.0) || !isfinite(tol)) return -1;
    return encode_variable(base, n, s, zfpo_accuracy_minexp(tol), 0, lengths, payload, payload_bytes, total_bits);
}

/* Precision mode: every block keeps its top `prec` bit planes (1..32), same
 * stream layout and cut as the accuracy mode; decoded by zfpo_decode_accuracy. */
int zfpo_encode_precision(const float *base, const int64_t n[3], const int64_t s[3], int prec,
                          uint16_t *lengths, uint8_t *payload, int64_t payload_bytes, uint64_t *total_bits)
{
    if (prec < 1 || prec > 32) return -1;
    return encode_variable(base, n, s, 0, prec, lengths, payload, payload_bytes, total_bits);
}

int zfpo_decode_accuracy(const uint16_t *lengths, const uint8_t *payload, const int64_t n[3],
                         float *base, const int64_t s[3])
{
    if (n[0] < 1 || n[1] < 1 || n[2] < 1) return 0;
    bitr r = {payload, 0};
    float v[64];
    int64_t bx = (n[0] + 3) / 4, by = (n[1] + 3) / 4, bz = (n[2] + 3) / 4, b = 0;
    for (int64_t zb = 0; zb < bz; zb++)
        for (int64_t yb = 0; yb < by; yb++)
            for (int64_t xb = 0; xb < bx; xb++) {
                uint8_t blk[128];
                memset(blk, 0, sizeof blk);
                bitw bw = {blk, 0};
                const unsigned L = lengths[b++];
                if (L > 1024) return -1;
                for (unsigned i = 0; i < L; i++) put_bit(&bw, get_bit(&r));
                bitr br = {blk, 0};
                decode_block(&br, 3, 16, v);
                for (int k = 0; k < 4; k++)
                    for (int j = 0; j < 4; j++)
                        for (int i = 0; i < 4; i++) {
                            int64_t x = 4 * xb + i, y = 4 * yb + j, z = 4 * zb + k;
                            if (x < n[0] && y < n[1] && z < n[2])
                                base[x * s[0] + y * s[1] + z * s[2]] = v[i + 4 * j + 16 * k];
                        }
            }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* float64 fields (the paper cites CAMS data in float64, Sec. III; its own  */
/* fields are float32), 3-D blocks, fixed rate r bits per value (1..64).    */
/* The same steps with the double format's sizes (readings):                */
/*   e_max = frexp exponent of max|x|; zero block if max|x| is 0, below      */
/*   2^-1023 (e_max + 1023 <= 0) or non-finite: one 0 bit;                   */
/*   header: a 1 bit, then e_max + 1023 in 11 bits, LSB first;               */
/*   q = trunc(x 2^(62 - e_max)) as int64 (|q| < 2^62);                      */
/*   the same five-step lifting in int64 (floor halving), axes x, y, z;      */
/*   the same coefficient order; negabinary with 0xAAAA...AA (64 bits);      */
/*   bit planes 63 .. 0 with the same group-tested coder, cut at 64 r bits;  */
/*   decode x = q 2^(e_max - 62) rounded once to nearest even.               */
/* ------------------------------------------------------------------------ */
typedef __int128 i128;

static i128 wrap64(i128 v)
{
    const int64_t w = (int64_t)(uint64_t)(unsigned __int128)v;
    if ((i128)w != v) g_overflow++;
    return w;
}
static i128 floor_half128(i128 v) { return (v - (v & 1)) / 2; }
#define INT64_HALF(v) floor_half128(wrap64(v))

static void lift_forward_i64(int64_t *p, ptrdiff_t s)
{
    i128 a = p[0], b = p[s], c = p[2 * s], d = p[3 * s];
    LIFT_FORWARD(a, b, c, d, INT64_HALF);
    p[0] = (int64_t)wrap64(a); p[s] = (int64_t)wrap64(b);
    p[2 * s] = (int64_t)wrap64(c); p[3 * s] = (int64_t)wrap64(d);
}
static void lift_inverse_i64(int64_t *p, ptrdiff_t s)
{
    i128 a = p[0], b = p[s], c = p[2 * s], d = p[3 * s];
    LIFT_INVERSE(a, b, c, d, INT64_HALF);
    p[0] = (int64_t)wrap64(a); p[s] = (int64_t)wrap64(b);
    p[2 * s] = (int64_t)wrap64(c); p[3 * s] = (int64_t)wrap64(d);
}

void zfpo_xform_forward_i64(int64_t *q)
{
    for (int k = 0; k < 4; k++)
        for (int j = 0; j < 4; j++) lift_forward_i64(q + 4 * j + 16 * k, 1);
    for (int k = 0; k < 4; k++)
        for (int i = 0; i < 4; i++) lift_forward_i64(q + i + 16 * k, 4);
    for (int j = 0; j < 4; j++)
        for (int i = 0; i < 4; i++) lift_forward_i64(q + i + 4 * j, 16);
}
void zfpo_xform_inverse_i64(int64_t *q)
{
    for (int j = 0; j < 4; j++)
        for (int i = 0; i < 4; i++) lift_inverse_i64(q + i + 4 * j, 16);
    for (int k = 0; k < 4; k++)
        for (int i = 0; i < 4; i++) lift_inverse_i64(q + i + 16 * k, 4);
    for (int k = 0; k < 4; k++)
        for (int j = 0; j < 4; j++) lift_inverse_i64(q + 4 * j + 16 * k, 1);
}

static const uint64_t kNega64 = 0xAAAAAAAAAAAAAAAAull;

static void encode_block_f64(bitw *w, int rate, const double *v)
{
    const uint64_t maxbits = 64ull * (uint64_t)rate;
    const uint64_t start = w->pos;
    double M = 0.0;
    for (int i = 0; i < 64; i++) {
        double a = fabs(v[i]);
        if (a > M || a != a) M = a;
    }
    int emax = 0, zero = 1;
    if (M > 0.0 && isfinite(M)) {
        (void)frexp(M, &emax);
        zero = (emax + 1023 <= 0);
    }
    if (zero) { put_bit(w, 0); w->pos = start + maxbits; return; }
    put_bit(w, 1);
    unsigned e = (unsigned)(emax + 1023);
    for (int b = 0; b < 11; b++) put_bit(w, (e >> b) & 1u);
    int64_t q[64];
    for (int i = 0; i < 64; i++) q[i] = (int64_t)ldexp(v[i], 62 - emax);     /* exact, truncates */
    zfpo_xform_forward_i64(q);
    int order[64];
    zfpo_sequency_order(3, order);
    uint64_t u[64];
    for (int t = 0; t < 64; t++) u[t] = ((uint64_t)q[order[t]] + kNega64) ^ kNega64;
    uint64_t left = maxbits - 12;
    int n = 0;
    for (int k = 63; k >= 0 && left > 0; k--) {
        unsigned X[64];
        for (int i = 0; i < 64; i++) X[i] = (unsigned)((u[i] >> k) & 1u);
        if (code_plane(w, 64, X, &n, &left)) break;
    }
    w->pos = start + maxbits;
}

static void decode_block_f64(bitr *r, int rate, double *v)
{
    const uint64_t maxbits = 64ull * (uint64_t)rate;
    const uint64_t start = r->pos;
    if (!get_bit(r)) {
        for (int i = 0; i < 64; i++) v[i] = 0.0;
        r->pos = start + maxbits;
        return;
    }
    unsigned e = 0;
    for (int b = 0; b < 11; b++) e |= get_bit(r) << b;
    const int emax = (int)e - 1023;
    uint64_t u[64];
    for (int i = 0; i < 64; i++) u[i] = 0;
    uint64_t left = maxbits - 12;
    int n = 0;
    for (int k = 63; k >= 0 && left > 0; k--) {
        unsigned X[64];
        for (int i = 0; i < 64; i++) X[i] = 0;
        int stopped = decode_plane(r, 64, X, &n, &left);
        for (int i = 0; i < 64; i++) u[i] |= (uint64_t)X[i] << k;
        if (stopped) break;
    }
    int order[64];
    zfpo_sequency_order(3, order);
    int64_t q[64];
    for (int t = 0; t < 64; t++) q[order[t]] = (int64_t)((u[t] ^ kNega64) - kNega64);
    zfpo_xform_inverse_i64(q);
    for (int i = 0; i < 64; i++)
        v[i] = (double)ldexpl((long double)q[i], emax - 62);    /* q exact in long double: one rounding */
    r->pos = start + maxbits;
}

static int valid_rate_f64(int rate) { return rate >= 1 && rate <= 64; }

int64_t zfpo_stream_bytes_f64(int rate, const int64_t n[3])
{
    return (zfpo_block_count(3, n) * 64 * rate + 7) / 8;
}

int zfpo_encode_block_f64(int rate, const double *v, uint8_t *out /* zeroed */)
{
    if (!valid_rate_f64(rate)) return -1;
    bitw w = {out, 0};
    encode_block_f64(&w, rate, v);
    return 0;
}
int zfpo_decode_block_f64(int rate, const uint8_t *in, double *v)
{
    if (!valid_rate_f64(rate)) return -1;
    bitr r = {in, 0};
    decode_block_f64(&r, rate, v);
    return 0;
}

int zfpo_encode_array_f64(int rate, const double *base, const int64_t n[3], const int64_t s[3],
                          uint8_t *out, int64_t out_bytes)
{
    if (!valid_rate_f64(rate)) return -1;
    if (n[0] < 1 || n[1] < 1 || n[2] < 1) return 0;
    if (out_bytes < zfpo_stream_bytes_f64(rate, n)) return -2;
    memset(out, 0, (size_t)zfpo_stream_bytes_f64(rate, n));
    bitw w = {out, 0};
    double v[64];
    int64_t bx = (n[0] + 3) / 4, by = (n[1] + 3) / 4, bz = (n[2] + 3) / 4;
    for (int64_t zb = 0; zb < bz; zb++)
        for (int64_t yb = 0; yb < by; yb++)
            for (int64_t xb = 0; xb < bx; xb++) {
                for (int k = 0; k < 4; k++)
                    for (int j = 0; j < 4; j++)
                        for (int i = 0; i < 4; i++) {
                            int64_t x = imin64(4 * xb + i, n[0] - 1);
                            int64_t y = imin64(4 * yb + j, n[1] - 1);
                            int64_t z = imin64(4 * zb + k, n[2] - 1);
                            v[i + 4 * j + 16 * k] = base[x * s[0] + y * s[1] + z * s[2]];
                        }
                encode_block_f64(&w, rate, v);
            }
    return 0;
}

int zfpo_decode_array_f64(int rate, const uint8_t *in, const int64_t n[3], double *base, const int64_t s[3])
{
    if (!valid_rate_f64(rate)) return -1;
    if (n[0] < 1 || n[1] < 1 || n[2] < 1) return 0;
    bitr r = {in, 0};
    double v[64];
    int64_t bx = (n[0] + 3) / 4, by = (n[1] + 3) / 4, bz = (n[2] + 3) / 4;
    for (int64_t zb = 0; zb < bz; zb++)
        for (int64_t yb = 0; yb < by; yb++)
            for (int64_t xb = 0; xb < bx; xb++) {
                decode_block_f64(&r, rate, v);
                for (int k = 0; k < 4; k++)
                    for (int j = 0; j < 4; j++)
                        for (int i = 0; i < 4; i++) {
                            int64_t x = 4 * xb + i, y = 4 * yb + j, z = 4 * zb + k;
                            if (x < n[0] && y < n[1] && z < n[2])
                                base[x * s[0] + y * s[1] + z * s[2]] = v[i + 4 * j + 16 * k];
                        }
            }
    return 0;
}
