/*
 * zfpx.h -- C ABI of the GB300 (sm_103a) library for the fused pencil-
 * transposition pack + ZFP fixed-rate compression path.
 *
 * The method (paper Sec. I and Sec. IV-C/D): before each all-to-all of the
 * Spherical Harmonic Transform's pencil transpositions (Sec. II-B), every
 * rank compresses its outgoing buffer on the GPU with ZFP in fixed-rate mode
 * (Sec. II-C, Sec. IV-B: rate 8 or 16 bits per value, a fixed and
 * predictable message size), sends the streams, and decompresses on receipt.
 * Comparators: the plain float32 buffer and a float16 cast (Sec. I,
 * Sec. IV-D).  On one device every rank is simulated: the all-to-all is a
 * device-local permutation of fixed-size messages.
 *
 * Conventions (all entry points):
 *  - Pointers named d_* are DEVICE pointers owned by the caller; the library
 *    never frees them.  Pointers without the prefix are host pointers.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every d_* call only enqueues work on that stream and returns;
 *    the caller synchronises.
 *  - Return value 0 on success, a negative ZFPX_E* code otherwise; nothing
 *    is enqueued when an argument check fails.  zfpx_strerror() names codes.
 *  - Fields are float32 arrays indexed by (x, y, z) = (longitude, latitude,
 *    level); a view gives extents n[] and element strides stride[] (axis 0 =
 *    longitude, normally stride 1).  Strides are non-negative.
 *  - rate: ZFPX_RATE_F32 (0) plain float32, ZFPX_RATE_F16 (-16) float16
 *    cast, or a ZFP rate in bits per value; the GPU codec supports 8 and 16.
 *  - ZFP streams: every 4^d block takes exactly 4^d * rate bits, blocks back
 *    to back in raster order of block index (axis 0 fastest); bit p of a
 *    stream is bit (p % 8) of byte p / 8.  Partial blocks are completed by
 *    repeating the last value along each short axis; the repeated values are
 *    coded and dropped again on decode.
 */
#ifndef ZFPX_H
#define ZFPX_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define ZFPX_API __attribute__((visibility("default")))
#else
#define ZFPX_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define ZFPX_OK 0
#define ZFPX_EINVAL (-1)          /* bad argument: view, rate, dims, rank grid, NULL */
#define ZFPX_ESIZE (-2)           /* caller's buffer smaller than required */
#define ZFPX_ECUDA (-3)           /* a CUDA call or kernel launch failed */
#define ZFPX_ETIMEOUT (-4)        /* a bounded device-side wait gave up */
#define ZFPX_ENOMEM_BUDGET (-5)   /* request larger than the admission budget */
#define ZFPX_ENOMEM (-6)          /* host or device allocation failed */

#define ZFPX_RATE_F32 0
#define ZFPX_RATE_F16 (-16)

/* buffer layouts a call reads or writes */
#define ZFPX_LAYOUT_SEND 0        /* per source rank, messages in destination-peer order */
#define ZFPX_LAYOUT_RECV 1        /* per destination rank, in source-peer order */

/* float16 rounding of the comparator */
#define ZFPX_ROUND_NEAREST 0      /* IEEE round to nearest even; overflow to +-inf */
#define ZFPX_ROUND_ZERO 1         /* toward zero; overflow to +-65504 */

/* plan split modes */
#define ZFPX_SPLIT_BALANCED 0     /* the first (extent mod parts) parts get one more */
#define ZFPX_SPLIT_TABLE1 1       /* floor(extent / parts) each, remainder dropped (Table 1) */

typedef struct {
    int64_t n[3];       /* extents: longitude, latitude, level */
    int64_t stride[3];  /* element strides of the same axes */
} zfpx_view3;

typedef struct zfpx_plan_s *zfpx_plan;
typedef struct zfpx_graph_s *zfpx_graph;
typedef struct zfpx_batch_s *zfpx_batch;
typedef struct zfpx_server_s *zfpx_server;

/* One field of a batch on a grid of ragged rows, stored [level][point]: the
 * rows [row0, row1) of the grid (row0 = row1 = 0: all rows) on nlev levels.
 * d_src and d_dst point at level 0, first point of row row0. */
typedef struct {
    const float *d_src;       /* values to encode (device), NULL if the batch only decodes */
    float *d_dst;             /* decode target (device), NULL if it only encodes */
    int64_t lev_stride;       /* d_src elements between levels (>= the rows' points when nlev > 1) */
    int64_t dst_lev_stride;   /* d_dst elements between levels; 0 = lev_stride */
    int32_t nlev;             /* levels, >= 1 */
    int32_t dims;             /* 1: 4 points of a row; 3: 4 points x 4 rows x 4 levels */
    int32_t rate;             /* 8 or 16 */
    int32_t row0, row1;       /* dims 3: row0 % 4 == 0 and (row1 % 4 == 0 or row1 == nrows) */
    int32_t reserved;         /* 0 */
} zfpx_field;

ZFPX_API const char *zfpx_strerror(int code);

/* Number of kernels this library has launched since load (all devices). */
ZFPX_API uint64_t zfpx_launch_count(void);

/* ---- plan (Sec. II-B, pencil transpositions; Table 1) --------------------
 * Builds the message list of one transposition over a p_r x p_c rank grid,
 * rank id = row * p_c + col.
 *   transposition 0, z -> lambda (the all-to-all by rows): source (row j, col i)
 *     holds lon part i of p_c x lat part j of p_r x all levels; message
 *     (j,i) -> (j,k) is the box lon_i x lat_j x lev_k (levels split in p_c).
 *   transposition 1, lambda -> theta (the all-to-all by columns): source
 *     (row j, col k) holds all lon x lat_j x lev_k; message (j,k) -> (l,k) is
 *     lon_l (lon split in p_r) x lat_j x lev_k.
 * `src` describes the field the packs read (all simulated ranks' pencils
 * together, as one array); `dst` the field the unpacks write; their
 * extents must be equal, strides may differ.  dims = 3 (4x4x4 blocks), 2
 * (4x4 blocks over longitude and latitude, every level on its own: the block
 * shape for single-level fields, coded like the 3-D blocks with one axis
 * fewer, 16 r bits each) or 1 (4 values along longitude).  Every message starts at a multiple of 256
 * bytes in both layouts.  The plan is host-side; device tables are built on
 * first use per rate (or by zfpx_plan_prepare, which should precede any
 * stream capture).  *out receives a plan owned by the caller, freed with
 * zfpx_plan_destroy.  Size limits (the kernels' block and row indices are
 * 32-bit): every extent at most 2^31 - 8, and in every message
 * ceil(nx / 4) * ny * nz < 2^31 (nx, ny, nz the message box); a larger field
 * goes through more ranks or several calls.  At most 2^24 messages
 * (p_r p_c p_c for transposition 0, p_r p_c p_r for 1).  Errors: ZFPX_EINVAL
 * (bad argument or a size limit), ZFPX_ENOMEM (host tables). */
ZFPX_API int zfpx_plan_create(zfpx_plan *out, const zfpx_view3 *src, const zfpx_view3 *dst,
                     int pr, int pc, int transposition, int dims, int split_mode);
ZFPX_API void zfpx_plan_destroy(zfpx_plan plan);
/* Uploads the device tables for `rate` on the current device (synchronous). */
ZFPX_API int zfpx_plan_prepare(zfpx_plan plan, int rate);

ZFPX_API int zfpx_plan_num_messages(zfpx_plan plan);
/* Geometry of message i (send order): ranks, peers, and the box x0,nx,y0,ny,z0,nz. */
ZFPX_API int zfpx_plan_message(zfpx_plan plan, int i, int32_t ranks[4], int64_t box[6]);
/* Bytes of message (src, dst) at `rate` -- what rank src sends to rank dst,
 * the send-size query; 0 if the pair exchanges nothing. */
ZFPX_API size_t zfpx_message_bytes(zfpx_plan plan, int rate, int src, int dst);
/* Byte offset of message (src, dst) in the given layout; -1 if none. */
ZFPX_API int64_t zfpx_message_offset(zfpx_plan plan, int rate, int layout, int src, int dst);
/* Total bytes of a send (= receive) buffer at `rate`. */
ZFPX_API size_t zfpx_buffer_bytes(zfpx_plan plan, int rate);

/* ---- the fused codec path -------------------------------------------------
 * zfpx_pack_compress (Sec. I: the send buffer is compressed on the device
 * right ahead of the exchange; Sec. II-C fixed-rate ZFP):
 * gathers every message's box from d_src (the plan's src view), codes it at
 * `rate` (8 or 16) and writes it at its fixed offset of the chosen layout in
 * d_out (cap bytes).  ZFPX_LAYOUT_RECV writes each message straight into the
 * receiver's slot (the permutation folded into the addressing).
 * Errors: ZFPX_EINVAL, ZFPX_ESIZE (cap < zfpx_buffer_bytes), ZFPX_ECUDA. */
ZFPX_API int zfpx_pack_compress(zfpx_plan plan, int rate, const float *d_src, uint8_t *d_out,
                       size_t cap, int layout, void *stream);

/* zfpx_decompress_unpack (Sec. I: the receiver expands the streams before it
 * computes on them): decodes every message of d_in (len bytes, the
 * chosen layout) and scatters the values into d_dst through the plan's dst
 * view; padding values are dropped.  Errors as above.
 *
 * Neither call keeps state on the device between launches (the work split is
 * fixed by the launch shape), so launches with the same plan may run on
 * several streams at once, and graph replays need no reset. */
ZFPX_API int zfpx_decompress_unpack(zfpx_plan plan, int rate, const uint8_t *d_in, size_t len,
                           float *d_dst, int layout, void *stream);

/* Launch shape of the 3-D codec kernels: every warp codes `upw` consecutive
 * units of 32 blocks (encode != 0: compression, else decompression; rate 8
 * or 16); 0 restores the library's default.  Process-wide; results never
 * depend on it (the autotuner sets it).  Errors: ZFPX_EINVAL.
 * zfpx_get_units_per_warp returns the value in use. */
ZFPX_API int zfpx_set_units_per_warp(int encode, int rate, int upw);
ZFPX_API int zfpx_get_units_per_warp(int encode, int rate);

/* ---- comparators (Sec. I; Sec. IV-D, Table 1 columns Float32/Float16) ----- */
/* float32 -> float16 cast of every message (round_mode ZFPX_ROUND_*). */
ZFPX_API int zfpx_cast_fp16_pack(zfpx_plan plan, int round_mode, const float *d_src, uint16_t *d_out,
                        size_t cap_bytes, int layout, void *stream);
ZFPX_API int zfpx_fp16_unpack(zfpx_plan plan, const uint16_t *d_in, size_t len_bytes, float *d_dst,
                     int layout, void *stream);
/* plain float32 copy-pack and unpack */
ZFPX_API int zfpx_pack(zfpx_plan plan, const float *d_src, float *d_out, size_t cap_bytes, int layout,
              void *stream);
ZFPX_API int zfpx_unpack(zfpx_plan plan, const float *d_in, size_t len_bytes, float *d_dst, int layout,
                void *stream);

/* ---- the all-to-all on one device (Sec. II-B; Sec. IV-D) ------------------
 * recv[dst][src] <- send[src][dst] for every message of the plan at `rate`.
 * d_send and d_recv must not overlap; len = zfpx_buffer_bytes(plan, rate). */
ZFPX_API int zfpx_permute(zfpx_plan plan, int rate, const void *d_send, void *d_recv, size_t len,
                 void *stream);

/* ---- raw codec on one array (Sec. II-C) ------------------------------------
 * Encodes the array of extents n[] read through element strides stride[]
 * into d_out (cap bytes, at least zfpx_stream_bytes).  dims 1, 2 or 3,
 * rate 8 or 16; blocks back to back in raster order of block indices (axis 0
 * fastest; for dims 2 each level's blocks in turn).  The array is one message
 * of a one-rank plan, so the plan's size limits hold: ceil(n[0] / 4) * n[1] *
 * n[2] < 2^31 (about 8.6e9 values).  Errors: ZFPX_EINVAL, ZFPX_ESIZE,
 * ZFPX_ECUDA. */
ZFPX_API size_t zfpx_stream_bytes(int dims, int rate, const int64_t n[3]);
ZFPX_API int zfpx_encode(int dims, int rate, const float *d_in, const int64_t n[3],
                const int64_t stride[3], uint8_t *d_out, size_t cap, void *stream);
ZFPX_API int zfpx_decode(int dims, int rate, const uint8_t *d_in, size_t len, const int64_t n[3],
                const int64_t stride[3], float *d_out, void *stream);

/* ---- debug report of non-finite inputs (Sec. II-C) ------------------------
 * The paper's codec outline leaves infinities and NaNs in the input
 * unspecified.  The codec codes a block whose largest magnitude is not finite
 * as a zero block (a single 0 bit; it decodes to zeros) and never faults on
 * one; this call reports such inputs.  It adds to *d_count (a device counter that the caller owns, zeroes
 * and reads) the number of elements of the view (extents n[], element strides
 * stride[] >= 0, axis 0 fastest) whose exponent field is all ones, i.e. the
 * infinities and NaNs.  elem_bytes: 4 for float32, 8 for float64; d_src
 * aligned to it, d_count to 8 bytes.  Asynchronous on `stream`; it is a call
 * of its own, so the codec calls pay nothing for it.  An empty view adds 0 and
 * launches nothing.  Errors: ZFPX_EINVAL (NULL, a negative extent or stride,
 * elem_bytes not 4 or 8, misaligned pointers), ZFPX_ECUDA. */
ZFPX_API int zfpx_count_nonfinite(const void *d_src, int elem_bytes, const int64_t n[3], const int64_t stride[3],
                                  unsigned long long *d_count, void *stream);

/* ---- accuracy and precision modes: variable rate (3-D blocks) --------------
 * The ZFP mode the paper names and leaves for future work (Sec. II-C).  Every
 * 4x4x4 block (raster order, partial blocks edge-replicated as in the raw
 * codec) keeps its bit planes 31 .. kmin, kmin = clamp(floor(log2 tolerance)
 * - e_max + 22, 0, 32), at most 1024 bits (the rate-16 budget, which cuts
 * blocks whose planes do not fit): the reconstruction error of a block that
 * is not cut and whose kmin is not clamped at 0 stays within the tolerance.
 * A zero block takes 1 bit, a block below the tolerance its 9 header bits.
 * Output: d_lengths[b] = bits of block b (uint16, one per block) and
 * d_payload = the blocks' bits back to back, LSB first, in 64-bit words;
 * *d_total_bits (device) = their sum; the payload's used part is
 * 8 * ceil(total / 64) bytes.  Both calls need caller-owned device scratch
 * d_work (256-byte aligned) of zfpx_accuracy_workspace_bytes(n) bytes; the
 * encoder needs cap >= zfpx_accuracy_max_payload_bytes(n) (it zeroes that much
 * of d_payload).  Decode takes the lengths and the payload (len bytes, a
 * multiple of 8 covering the used part) and writes the array through stride.
 * Calls using the same d_work must not overlap on the GPU.  Errors:
 * ZFPX_EINVAL (NULL, extents < 1, tolerance not positive and finite,
 * misaligned pointers), ZFPX_ESIZE, ZFPX_ECUDA. */
ZFPX_API size_t zfpx_accuracy_workspace_bytes(const int64_t n[3]);
ZFPX_API size_t zfpx_accuracy_max_payload_bytes(const int64_t n[3]);
ZFPX_API int zfpx_encode_accuracy(const float *d_in, const int64_t n[3], const int64_t stride[3], double tolerance,
                                  uint16_t *d_lengths, uint8_t *d_payload, size_t cap, uint64_t *d_total_bits,
                                  void *d_work, size_t work_bytes, void *stream);
/* Precision mode: every block keeps its top `precision` bit planes (1..32), the
 * same cut, output and scratch as the accuracy mode; zfpx_decode_accuracy
 * decodes it. */
ZFPX_API int zfpx_encode_precision(const float *d_in, const int64_t n[3], const int64_t stride[3], int precision,
                                   uint16_t *d_lengths, uint8_t *d_payload, size_t cap, uint64_t *d_total_bits,
                                   void *d_work, size_t work_bytes, void *stream);
ZFPX_API int zfpx_decode_accuracy(const uint16_t *d_lengths, const uint8_t *d_payload, size_t len,
                                  const int64_t n[3], const int64_t stride[3], float *d_out, void *d_work,
                                  size_t work_bytes, void *stream);

/* ---- float64 fields: 3-D blocks, fixed rate (raw arrays) -----------------
 * The fixed-rate method with the double format's sizes, for the float64
 * fields the paper's data comes in (Sec. III): per 4x4x4 block a 1 bit and
 * the 11-bit biased exponent e_max + 1023 (e_max = the frexp exponent of the
 * block's largest magnitude; a zero block, one 0 bit, if that magnitude is
 * 0, below 2^-1023 or not finite), q = trunc(x 2^(62 - e_max)) as int64, the
 * five-step lifting in int64, the 3-D coefficient order, 64-bit negabinary
 * and group-tested bit planes 63 .. 0 cut at exactly 64 * rate bits.  Decode
 * rounds q 2^(e_max - 62) once to nearest even (subnormal results included).
 * rate = bits per value, 1 .. 32; the stream is the blocks' 8 * rate bytes
 * each, in raster block order (x fastest).  d_in/d_out: device arrays read or
 * written through stride (in elements, >= 0; any view), 8-byte aligned, and
 * the stream 8-byte aligned.  Errors: ZFPX_EINVAL
 * (NULL, rate, extents < 1, alignment), ZFPX_ESIZE (cap / len below
 * zfpx_stream_bytes_f64), ZFPX_ECUDA. */
ZFPX_API size_t zfpx_stream_bytes_f64(int rate, const int64_t n[3]);
ZFPX_API int zfpx_encode_f64(int rate, const double *d_in, const int64_t n[3], const int64_t stride[3],
                             uint8_t *d_out, size_t cap, void *stream);
ZFPX_API int zfpx_decode_f64(int rate, const uint8_t *d_in, size_t len, const int64_t n[3],
                             const int64_t stride[3], double *d_out, void *stream);

/* ---- the longitude transform (the FFT after the first transposition) ------
 * The spectral transform is an FFT in longitude and a Legendre transform in
 * latitude (Sec. II-A); the z -> lambda all-to-all makes every longitude row
 * local so that the FFT can run (Sec. II-B).  For every row x_0 .. x_{N-1} of
 * the [n2][n1][n0] float32 array d_in (n0 = N longitudes, row elements
 * contiguous: stride[0] == 1; stride[1], stride[2] even, d_in 8-byte aligned)
 * this writes F_m = (1/N) sum_j x_j exp(-2 pi i j m / N), m = 0 .. K-1, as
 * real parts to d_re and imaginary parts to d_im, both [n2][n1][K] float32
 * arrays through ostride (ostride[0] == 1; the same strides for both).
 * N even, N <= 8192, N / 2 a product of 2, 3 and 5; 1 <= K <= N/2 + 1.
 * Single-precision arithmetic; twiddles rounded once from double.  The first
 * call for a given N on a device builds that N's twiddle table (8 N bytes of
 * device memory, kept for the process; a synchronous upload, so make that
 * first call outside stream capture).  Errors: ZFPX_EINVAL (NULL, sizes,
 * strides, alignment), ZFPX_ECUDA. */
ZFPX_API int zfpx_rfft_lon(const float *d_in, const int64_t n[3], const int64_t stride[3], int K, float *d_re,
                           float *d_im, const int64_t ostride[3], void *stream);

/* ---- decompression fused with the longitude FFT (Sec. II-A; Sec. VI) ------
 * For a z -> lambda plan (transposition 0, dims 3): decodes the received
 * messages d_recv (len bytes, the receive layout of zfpx_pack_compress /
 * zfpx_permute at `rate` 8 or 16) and transforms every longitude row of the
 * assembled field straight into wavenumbers F_m = (1/N) sum_j x_j
 * exp(-2 pi i j m / N), m < K <= N/2 + 1 (N = the plan's n[0], even, at most
 * 8192, with prime factors 2, 3 and 5 only), real parts to d_re and imaginary
 * parts to d_im, float32 [n2][n1][>= K] with element strides ostride
 * (ostride[0] == 1).  The values equal, bit for bit, zfpx_decompress_unpack
 * followed by zfpx_rfft_lon on the decoded field; the float32 field is never
 * written to memory in between.  d_work: caller-owned device scratch
 * (16-byte aligned) of zfpx_decompress_rfft_workspace_bytes(plan) bytes, row
 * buffers that stay in L2; calls that share d_work must not overlap on the
 * GPU.  The first call per (plan, rate) uploads the plan's unit table (an
 * allocation, so make that first call before any stream capture).  Errors:
 * ZFPX_EINVAL (NULL, plan kind, sizes, strides, alignment, or a plan whose
 * messages to one receiver do not tile its rows), ZFPX_ESIZE, ZFPX_ECUDA,
 * ZFPX_ENOMEM. */
ZFPX_API size_t zfpx_decompress_rfft_workspace_bytes(zfpx_plan plan);
ZFPX_API int zfpx_decompress_rfft(zfpx_plan plan, int rate, const uint8_t *d_recv, size_t len, int K, float *d_re,
                                  float *d_im, const int64_t ostride[3], void *d_work, size_t work_bytes,
                                  void *stream);

/* ---- the Legendre transform (the latitude transform after the second
 * transposition) -------------------------------------------------------------
 * The spectral transform's latitude half (Sec. II-A: associated Legendre
 * functions, Gauss-Legendre quadrature), run on theta-pencils once the
 * lambda -> theta all-to-all has made every latitude column local (Sec. II-B).
 * For the wavenumber fields F_m(mu_j) (real and imaginary parts: float32
 * [n2 = levels][n1 = nlat][n0 >= T + 1 wavenumbers], the same strides for
 * both, stride[0] == 1; latitudes at the Gauss-Legendre nodes north to south)
 *     a_l^m = sum_j w_j Pbar_l^m(mu_j) F_m(mu_j),   0 <= m <= l <= T,
 * Pbar normalised to int_{-1}^{1} Pbar_l^m Pbar_l'^m dmu = delta_ll' with the
 * Condon-Shortley phase.  Output: per level, a_l^m at m (T+1) - m (m-1)/2 +
 * (l - m), real parts to d_are and imaginary parts to d_aim, levels
 * out_stride floats apart (>= (T+1)(T+2)/2).
 * zfpx_legendre_create builds the plan on the current device: the Gauss
 * nodes and weights and the table w_j Pbar_l^m(mu_j) over the northern half
 * (computed in double, rounded once) with its TF32 low parts for the tensor
 * cores (about 2 (T+1)(T+2) nlat bytes of device memory in all, a
 * synchronous upload); nlat even, at most 32768, T + 1 <= nlat.
 * zfpx_legendre_forward takes n[1] equal to the plan's nlat and 1 .. 2^20
 * levels, and needs caller-owned device scratch d_work (16-byte aligned) of
 * zfpx_legendre_workspace_bytes(plan, levels) bytes; calls that share d_work
 * must not overlap on the GPU.  Float32 in and out; the contraction runs on
 * the tensor cores (TF32 operands split into high and low parts, three
 * products per term, float32 accumulation), which keeps float32 accuracy.
 * Errors: ZFPX_EINVAL (NULL, sizes, strides, alignment, another device),
 * ZFPX_ESIZE, ZFPX_ECUDA.
 * zfpx_legendre_status reads (synchronously) whether any earlier forward on
 * the plan gave up on a bounded wait inside its kernel: ZFPX_OK, or
 * ZFPX_ETIMEOUT (that call's coefficients are incomplete). */
/* The Gauss-Legendre latitudes the transform expects: mu[i] = sin(latitude),
 * north to south, and the weights w[i] (sum 2), for n = 1 .. 32768 points, by
 * Newton's iteration on P_n in double precision (the nodes the plan uses).
 * Host arrays of n doubles each; no GPU work.  Errors: ZFPX_EINVAL. */
ZFPX_API int zfpx_gauss_legendre(int n, double *mu, double *w);
typedef struct zfpx_legendre_s *zfpx_legendre;
ZFPX_API int zfpx_legendre_create(zfpx_legendre *out, int nlat, int T);
ZFPX_API void zfpx_legendre_destroy(zfpx_legendre plan);
ZFPX_API size_t zfpx_legendre_workspace_bytes(zfpx_legendre plan, int64_t levels);
ZFPX_API int zfpx_legendre_forward(zfpx_legendre plan, const float *d_re, const float *d_im, const int64_t n[3],
                                   const int64_t stride[3], float *d_are, float *d_aim, int64_t out_stride,
                                   void *d_work, size_t work_bytes, void *stream);
ZFPX_API int zfpx_legendre_status(zfpx_legendre plan);

/* The accuracy mode on a transposition plan (dims 3): every message's box is
 * coded as above, so messages vary in size and the exchange becomes an
 * all-to-all-v, the per-message sizes first, then the payloads (on one GPU,
 * device-local copies).  Per plan: G = zfpx_plan_accuracy_blocks (blocks of all
 * messages), scratch d_work of zfpx_plan_accuracy_workspace_bytes (256-byte
 * aligned, shared by the three calls, which must not overlap on the GPU).
 *   pack_compress: d_lengths (G uint16, messages in send order, blocks in
 *     raster order), d_payload (cap >= 128 G bytes; message m starts on a
 *     64-bit word, messages back to back in send order), d_msg_words (one per
 *     message in send order: its payload in 64-bit words).
 *   exchange: moves lengths and payloads to the receive order (by destination
 *     rank, then source peer), both payload buffers of cap >= 128 G bytes.
 *   decompress_unpack: from the received lengths and payload (len bytes) and
 *     the same d_msg_words, writes the plan's destination view.
 * Errors: ZFPX_EINVAL (NULL, dims != 3, tolerance, alignment), ZFPX_ESIZE,
 * ZFPX_ECUDA. */
ZFPX_API size_t zfpx_plan_accuracy_blocks(zfpx_plan plan);
ZFPX_API size_t zfpx_plan_accuracy_workspace_bytes(zfpx_plan plan);
ZFPX_API int zfpx_pack_compress_accuracy(zfpx_plan plan, double tolerance, const float *d_src, uint16_t *d_lengths,
                                         uint8_t *d_payload, size_t cap, uint64_t *d_msg_words, void *d_work,
                                         size_t work_bytes, void *stream);
/* The precision mode on a plan (the same layout; exchange and decode as above). */
ZFPX_API int zfpx_pack_compress_precision(zfpx_plan plan, int precision, const float *d_src, uint16_t *d_lengths,
                                          uint8_t *d_payload, size_t cap, uint64_t *d_msg_words, void *d_work,
                                          size_t work_bytes, void *stream);
ZFPX_API int zfpx_exchange_accuracy(zfpx_plan plan, const uint64_t *d_msg_words, const uint16_t *d_len_send,
                                    const uint8_t *d_pay_send, uint16_t *d_len_recv, uint8_t *d_pay_recv, size_t cap,
                                    void *d_work, size_t work_bytes, void *stream);
ZFPX_API int zfpx_decompress_unpack_accuracy(zfpx_plan plan, const uint64_t *d_msg_words, const uint16_t *d_len_recv,
                                             const uint8_t *d_pay_recv, size_t len, float *d_dst, void *d_work,
                                             size_t work_bytes, void *stream);

/* ---- batched ragged-row fields in one persistent launch -------------------
 * Many fields with different level counts, block dimensionality and rate
 * (ZFP fixed rate, Sec. II-C) on one grid of ragged rows: rows back to back,
 * row r holding row_len[r] points -- the octahedral reduced Gaussian grid of
 * IFS-class models has 20 + 4i points per row, mirrored.
 *   dims 1: blocks of 4 consecutive points of one row of one level;
 *   dims 3: 4 points x 4 consecutive rows (a row-quad) x 4 consecutive
 *     levels over x < the longest row of the quad, shorter rows repeating
 *     their last point, a missing last row / level repeating the last one.
 * Stream of a field: items (dims 3: level quads, dims 1: levels) in level
 * order, inside an item the blocks in row (row-quad) order then along x;
 * every field at a 256-byte aligned offset (zfpx_batch_field_offset).
 * zfpx_batch_create copies row_len and the descriptors (host arrays) and
 * uploads the work list to the current device (it allocates; the encode and
 * decode calls do not).  Each of zfpx_batch_encode / zfpx_batch_decode is
 * one kernel launch over every field.  The device pointers in the field
 * descriptors must stay valid while the batch is used.
 * Errors: ZFPX_EINVAL, ZFPX_ESIZE, ZFPX_ECUDA, ZFPX_ENOMEM. */
ZFPX_API int zfpx_batch_create(zfpx_batch *out, const int64_t *row_len, int nrows, const zfpx_field *fields,
                               int nfields);
ZFPX_API void zfpx_batch_destroy(zfpx_batch batch);
/* Total stream bytes of the batch; offset and bytes of field f's stream. */
ZFPX_API size_t zfpx_batch_bytes(zfpx_batch batch);
ZFPX_API int64_t zfpx_batch_field_offset(zfpx_batch batch, int f);
ZFPX_API size_t zfpx_batch_field_bytes(zfpx_batch batch, int f);
/* Launch shape used by later calls: warps per CTA (2, 3, 4 or 8; default 3)
 * and CTAs per SM (0 = as many as fit, the default).  Picked by the autotuner;
 * results never depend on it. */
ZFPX_API int zfpx_batch_set_launch(zfpx_batch batch, int warps_per_cta, int ctas_per_sm);
/* Work-unit size of 1-D items: a warp claims 32 x blocks_per_lane_1d
 * consecutive 1-D blocks at a time, each lane coding blocks_per_lane_1d of
 * them (1..64, default 16; 3-D units stay 32 blocks, one per lane).  Larger
 * units spend fewer work claims and table searches per block, smaller ones
 * balance short batches better.  Rebuilds the batch's work tables after
 * waiting for the device to go idle.  Picked by the autotuner; results never
 * depend on it.  Errors: ZFPX_EINVAL, ZFPX_ECUDA, ZFPX_ENOMEM. */
ZFPX_API int zfpx_batch_set_unit_blocks(zfpx_batch batch, int blocks_per_lane_1d);
/* Work units a warp claims at a time from its kind's queue (1..64, default
 * 4): one atomic add per claim.  More units per claim spend fewer atomics,
 * fewer balance the end of a launch better.  Picked by the autotuner; results
 * never depend on it.  Errors: ZFPX_EINVAL. */
ZFPX_API int zfpx_batch_set_claim_units(zfpx_batch batch, int units_per_claim);
ZFPX_API int zfpx_batch_encode(zfpx_batch batch, uint8_t *d_out, size_t cap, void *stream);
ZFPX_API int zfpx_batch_decode(zfpx_batch batch, const uint8_t *d_in, size_t len, void *stream);

/* ---- serving: a request loop with continuous batching ---------------------
 * The paper's exchange as a service: messages (row x level slabs of fields
 * resident on the device, one zfpx_field each, d_dst unused) arrive one by
 * one and are compressed and decompressed (the sender's and the receiver's
 * side of Sec. I) as they come.  A request is admitted when its compressed
 * stream plus its decoded copy fit in the server's arena -- one device
 * allocation of arena_bytes, the HBM budget, made at creation; a request that
 * can never fit is refused by zfpx_server_submit with ZFPX_ENOMEM_BUDGET.
 * zfpx_server_pump admits waiting requests (first come, first served, at
 * most max_batch) into one batch -- one encode and one decode launch -- on the
 * next of nstreams streams whose previous batch has finished, so batches
 * overlap on the device; *launched = requests put in flight (0 if none).
 * zfpx_server_poll returns ids of finished requests (up to max); their
 * results (device pointers from zfpx_server_result) stay valid until
 * zfpx_server_release returns the memory.  A request's bytes and values do
 * not depend on which other requests share its batch.  Nothing is allocated
 * after creation.  One host thread per server.
 * zfpx_server_stats: [queued, streams busy, arena bytes used, arena bytes,
 * batches launched, finished-not-polled]. */
ZFPX_API int zfpx_server_create(zfpx_server *out, const int64_t *row_len, int nrows, size_t arena_bytes, int nstreams,
                                int max_batch);
ZFPX_API void zfpx_server_destroy(zfpx_server server);
ZFPX_API int zfpx_server_set_launch(zfpx_server server, int warps_per_cta, int ctas_per_sm);
/* The 1-D work-unit size of zfpx_batch_set_unit_blocks, for batches launched
 * from then on.  Errors: ZFPX_EINVAL. */
ZFPX_API int zfpx_server_set_unit_blocks(zfpx_server server, int blocks_per_lane_1d);
/* A batching window for zfpx_server_pump: a batch is launched once at least
 * min_requests requests wait, or once the oldest waiting one has waited
 * max_wait_us microseconds (1 and 0, the defaults, launch whatever waits as
 * soon as a stream is free).  A window trades latency for larger batches
 * when requests arrive slower than the device codes them.  min_requests <=
 * max_batch, 0 <= max_wait_us <= 1e7.  Errors: ZFPX_EINVAL. */
ZFPX_API int zfpx_server_set_batching(zfpx_server server, int min_requests, double max_wait_us);
/* The units per claim of zfpx_batch_set_claim_units, for batches launched from
 * then on.  Errors: ZFPX_EINVAL. */
ZFPX_API int zfpx_server_set_claim_units(zfpx_server server, int units_per_claim);
ZFPX_API int zfpx_server_submit(zfpx_server server, const zfpx_field *request, int64_t *id);
ZFPX_API int zfpx_server_pump(zfpx_server server, int *launched);
ZFPX_API int zfpx_server_poll(zfpx_server server, int64_t *done, int max, int *ndone);
ZFPX_API int zfpx_server_result(zfpx_server server, int64_t id, const uint8_t **d_stream, size_t *stream_bytes,
                                const float **d_values, size_t *values_bytes);
/* Synchronous copy of a finished request's stream and values to host memory
 * (either pointer may be NULL). */
ZFPX_API int zfpx_server_copy_result(zfpx_server server, int64_t id, uint8_t *h_stream, size_t stream_cap,
                                     float *h_values, size_t values_cap);
ZFPX_API int zfpx_server_release(zfpx_server server, int64_t id);
ZFPX_API int zfpx_server_stats(zfpx_server server, int64_t out[6]);
/* The request loop in native code: submits request i once arrivals[i]
 * seconds have passed since the call began (all at once if arrivals is NULL),
 * and between arrivals pumps (a batch on every free stream), polls and
 * releases finished requests, until every request has finished.  t_done[i]:
 * the time from the start at which the loop saw request i finished, or -1 if
 * it was refused (ZFPX_ENOMEM_BUDGET: larger than the arena).  info (may be
 * NULL): [wall seconds from the first arrival to the last completion, batches
 * launched, most streams busy at once, requests refused].  The results are
 * released as they finish (use submit / pump / poll to keep them).  Errors:
 * ZFPX_EINVAL, and those of submit, pump and poll. */
ZFPX_API int zfpx_server_run(zfpx_server server, const zfpx_field *reqs, int n, const double *arrivals,
                             double *t_done, double *info);

/* ---- capturing any sequence of calls into a CUDA graph ---------------------
 * zfpx_capture_begin starts stream capture on `stream` (which must not be the
 * legacy default stream); every zfpx call enqueued on it until
 * zfpx_capture_end is recorded, not run; zfpx_capture_end instantiates the
 * graph.  Plans and batches used must have their device tables uploaded
 * before the capture starts (zfpx_plan_prepare; batches upload at creation). */
ZFPX_API int zfpx_capture_begin(void *stream);
ZFPX_API int zfpx_capture_end(zfpx_graph *out, void *stream);

/* ---- a transposition that allocates nothing --------------------------------
 * No counterpart in the paper: this serves callers that cannot allocate
 * device memory where they call -- inside another framework's memory pool or
 * allocator, in loops that must not pay for an allocation, with a fixed
 * device memory map.  It does what zfpx_pack_compress (ZFPX_LAYOUT_RECV)
 * followed by zfpx_decompress_unpack do, d_src -> d_dst through the plan at
 * `rate` (8 or 16), with the same result, but it keeps
 * the plan's message table and the compressed messages in one library-owned
 * device array of ZFPX_NOALLOC_SCRATCH_BYTES (64 MiB), reserved on every GPU
 * that loads the library until the process exits, and calls no allocation
 * routine; the plan
 * needs no zfpx_plan_prepare.  The first call on each device looks the array
 * up with that device current.  Every call shares the array, so calls that
 * overlap on the GPU (other streams, other host threads) race; calls in order
 * on one stream do not.  The message table is copied from pageable host
 * memory, so the call returns after the copy has read it, and the call
 * cannot be recorded into a CUDA graph: on a capturing stream it returns
 * ZFPX_EINVAL and enqueues nothing.  Errors: ZFPX_EINVAL, ZFPX_ESIZE (table
 * plus compressed messages larger than the array), ZFPX_ECUDA. */
#define ZFPX_NOALLOC_SCRATCH_BYTES (64u << 20)
ZFPX_API int zfpx_transpose_noalloc(zfpx_plan plan, int rate, const float *d_src, float *d_dst, void *stream);

/* ---- a transposition pipelined per piece (Sec. III-E, Sec. V-B) ----------
 * The paper's time model adds compression, exchange and decompression in
 * series and notes that pipelining them per block would do better.  A
 * pipeline splits the plan's messages into `pieces` pieces by destination
 * peer (piece k: peers d of the communicator with floor(d K / P) = k, K =
 * min(pieces, P)), and zfpx_pipeline_run compresses piece k+1 (stream A)
 * while piece k is moved to the receive layout (stream B, the device-local
 * all-to-all) and piece k-1 is decompressed and unpacked (stream C), ordered
 * by events.  The stream `stream` waits for the last piece; the streams of the
 * pipeline wait for what `stream` had enqueued before the call.  Results are
 * byte for byte those of zfpx_pack_compress (send layout), zfpx_permute and
 * zfpx_decompress_unpack: d_send and d_recv (buf_bytes each, >=
 * zfpx_buffer_bytes) end up as they would, and d_dst gets the same values.
 * Creation allocates the pieces' device tables, three streams and events
 * (run allocates nothing); one pipeline's runs must not overlap on the GPU
 * (they share its streams and events; runs in order on one stream do not).
 * The plan must outlive the pipeline.  Errors: ZFPX_EINVAL, ZFPX_ESIZE,
 * ZFPX_ECUDA, ZFPX_ENOMEM. */
typedef struct zfpx_pipeline_s *zfpx_pipeline;
ZFPX_API int zfpx_pipeline_create(zfpx_pipeline *out, zfpx_plan plan, int rate, int pieces);
/* Pieces actually used (K above). */
ZFPX_API int zfpx_pipeline_pieces(zfpx_pipeline pipeline);
ZFPX_API int zfpx_pipeline_run(zfpx_pipeline pipeline, const float *d_src, uint8_t *d_send, uint8_t *d_recv,
                               size_t buf_bytes, float *d_dst, void *stream);
ZFPX_API void zfpx_pipeline_destroy(zfpx_pipeline pipeline);

/* ---- the transposition pair as one CUDA graph (Sec. II-B; Sec. VI) -------
 * Records, on a private stream, pack+compress -> all-to-all -> decompress+
 * unpack with `first` (src field -> d_mid) and then with `second` (d_mid ->
 * d_dst): six kernels, or four with fold_permute != 0 (compress writes the
 * receive layout directly).  The plans must share extents; `first`'s dst
 * view and `second`'s src view both describe d_mid.  d_send / d_recv are
 * caller-owned scratch of buf_bytes each, at least the larger
 * zfpx_buffer_bytes of the two plans.  All pointers must stay valid for the
 * graph's lifetime.  Creation uploads the plans' device tables first, so it
 * allocates; launching does not.  Errors: ZFPX_EINVAL, ZFPX_ESIZE,
 * ZFPX_ECUDA, ZFPX_ENOMEM. */
ZFPX_API int zfpx_pair_graph_create(zfpx_graph *out, zfpx_plan first, zfpx_plan second, int rate,
                                    const float *d_src, float *d_mid, float *d_dst, uint8_t *d_send,
                                    uint8_t *d_recv, size_t buf_bytes, int fold_permute);
/* Enqueues one replay of the graph on `stream`. */
ZFPX_API int zfpx_graph_launch(zfpx_graph graph, void *stream);
/* Kernels recorded in the graph. */
ZFPX_API int zfpx_graph_num_kernels(zfpx_graph graph);
ZFPX_API void zfpx_graph_destroy(zfpx_graph graph);

#ifdef __cplusplus
}
#endif
#endif /* ZFPX_H */
