/*
 * dctf.h - C ABI of the GB300 block-DCT-domain filtering library (libdctf.so).
 *
 * The library applies a 2-D filter mask to the N x N block-DCT coefficients
 * of an image without returning to pixels.  The whole filter (mask, anchor,
 * per-block zero padding or border replication) is folded into one N^2 x N^2
 * operator M = (C kron C) H (C kron C)^T, built on the GPU in FP64 once per
 * mask, and then y_b = M x_b is computed for every block b.
 *
 *   Paper: "Block DCT filtering using vector processing" (arXiv 1710.07193).
 *   Sec. II.A, Eq. 1-3 : orthonormal DCT-II, BLOCK = C block C^T.
 *   Sec. II.B, Eq. 5-11: zero-padded filtering as sums of matrix products.
 *   Sec. II.C, Eq. 13-20: border replication added as further products.
 *   Eq. 7              : a spatial product moves to the DCT domain by
 *                        conjugation with C; for the vectorised block the
 *                        whole filter H becomes M = K H K^T, K = C kron C.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - N (block side) is 4, 8 or 16; a block has N2 = N*N coefficients.
 *  - Coefficient (u, v) of a block (u vertical, v horizontal frequency) is
 *    element u*N + v; a batch is [nblocks][N2], contiguous, blocks in any
 *    order (raster order of the image by convention).
 *  - The mask is a row-major mh x mw array of doubles with 1 <= mh, mw <= N;
 *    anchor = {row, col} is the mask entry over the output pixel.  The filter
 *    is a correlation: out(i,j) = sum_{r,c} w[r][c] x(i+r-ar, j+c-ac), the
 *    reading of Eq. 5 that the printed matrices of Eq. 6-18 implement.
 *    Each block is padded on its own (pixels of other blocks are never read).
 *  - Device pointers must be 16-byte aligned.  nblocks == 0 is a no-op.
 *  - Calls taking a stream are asynchronous on it; their return value covers
 *    argument checks and launch errors only.  Device-side failures (a bounded
 *    wait that ran out) are latched in the operator's status word, read with
 *    dctf_operator_status.
 *  - Every call returns DCTF_OK or an error code, never aborts; the message
 *    of the last error on the calling thread is dctf_last_error().
 *  - The caller owns every coefficient buffer; an operator owns its device
 *    memory until dctf_release_operator.
 */
#ifndef DCTF_H
#define DCTF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *dctf_stream_t;

typedef enum {
    DCTF_OK = 0,
    DCTF_EINVAL = 1,        /* bad argument: nothing was launched          */
    DCTF_ENOMEM = 2,        /* device or host allocation failed            */
    DCTF_ECUDA = 3,         /* a CUDA runtime call failed                  */
    DCTF_EBUDGET = 4,       /* request larger than the server's HBM budget */
    DCTF_ETIMEOUT = 5,      /* a bounded wait ran out (host or device)     */
    DCTF_EUNSUPPORTED = 6   /* valid but not supported (e.g. N, precision) */
} dctf_status;

typedef enum { DCTF_ZERO = 0, DCTF_REPLICATE = 1 } dctf_boundary;

/* Arithmetic of dctf_apply.  Every variant accumulates in FP32 and applies
 * the input DC coefficient's contribution as a separate FP32 rank-1 term.
 *  FP32_SIMT : plain FP32 FMA on CUDA cores (comparison kernel).
 *  F16X3     : tcgen05 tensor cores, FP16 hi/lo split of x and M,
 *              hi*hi + hi*lo + lo*hi.  |x| must stay below 65504.
 *              n = 8 and n = 16.
 *  BF16X6    : tcgen05, x and M in three BF16 pieces each, the six
 *              products x_i m_j with i + j <= 2.  n = 16.
 *  TF32X3    : tcgen05, TF32 hi/lo split, hi*hi + hi*lo + lo*hi.  n = 16.
 *  TF32X1    : tcgen05, x and M rounded to TF32 once, one product; about
 *              3 decimal digits, NOT within the 1e-3 coefficient bar (for
 *              comparison).  n = 16.
 *  BF16X3    : tcgen05, BF16 hi/lo split of x and M (the first two BF16X6
 *              pieces), hi*hi + hi*lo + lo*hi: the three-term split with
 *              BF16 pieces, ~16 significant bits, so NOT within the 1e-3
 *              coefficient bar (max 1-3e-3 on the 16x16 workload; 2e-4 in
 *              the pixel domain); the cost of F16X3 without its
 *              |x| < 65504 limit.  n = 16.
 *  KRON_FP32 : the paper's form (Sec. II.B Eq. 11-12, Sec. II.C Eq. 20):
 *              M = sum_t A_t kron B_t with one term per rank of the mask,
 *              applied as sandwich products Y = sum_t A_t X B_t^T in FP32
 *              on CUDA cores; r * 2 n^3 multiply-adds per block instead of
 *              n^4 (8x fewer for a separable mask at n = 16).  Needs an
 *              operator built with DCTF_BUILD_KRON; n = 4, 8, 16.
 *  KRON_F16X3: the same sandwich products on tcgen05 tensor cores with the
 *              F16X3 split (Sec. II.B Eq. 11-12, Sec. II.C Eq. 20): per
 *              term, Z_t = X B_t^T, then Y = sum_t A_t Z_t, both FP16 hi/lo
 *              products accumulated in FP32, Z re-split between the two;
 *              |x| must stay below 65504.  n = 16; runs in place.
 * The dense tensor-core variants of 16x16 blocks do not run in place.
 * dctf_operator_set_precision returns DCTF_EUNSUPPORTED for a variant that
 * has no kernel for the operator's n. */
typedef enum {
    DCTF_FP32_SIMT = 0,
    DCTF_F16X3 = 1,
    DCTF_BF16X6 = 2,
    DCTF_TF32X1 = 3,
    DCTF_TF32X3 = 4,
    DCTF_KRON_FP32 = 5,
    DCTF_BF16X3 = 6,
    DCTF_KRON_F16X3 = 7
} dctf_precision;

typedef struct dctf_operator dctf_operator;

/* Build the operator for one mask (Sec. II.B-C; M = K H K^T by Eq. 7).
 *  mask     host, row-major mh*mw doubles, copied (not kept).
 *  anchor   host {row, col}, 0-based inside the mask.
 *  n        4, 8 or 16.   boundary  DCTF_ZERO or DCTF_REPLICATE.
 *  stream   the FP64 build kernels run on it; *out may be used on that
 *           stream at once, on others after synchronising with it.
 * Allocates device memory on the current device (cudaMalloc).  The
 * precision starts as DCTF_F16X3 where tensor-core kernels exist for n,
 * else DCTF_FP32_SIMT.  EINVAL for a bad mask/anchor/n/boundary/out. */
dctf_status dctf_build_operator(const double *mask, int mh, int mw,
                                const int anchor[2], int n,
                                dctf_boundary boundary, dctf_stream_t stream,
                                dctf_operator **out);

/* As dctf_build_operator, with flags.  DCTF_MASK_CONVOLUTION applies the
 * mask as a convolution, out(i,j) = sum_{r,c} w[r][c] x(i-r+ar, j-c+ac)
 * (the other natural reading of Eq. 5), i.e. a correlation with the mask
 * rotated by 180 degrees and the anchor mirrored to (mh-1-ar, mw-1-ac). */
enum { DCTF_MASK_CONVOLUTION = 1u };
/* DCTF_BUILD_KRON: also keep the operator's Kronecker factors (every
 * rebuild recomputes them, all on the device in FP64): the mask is split
 * into rank(w) separable terms by Gaussian elimination with complete
 * pivoting (terms below 1e-13 of the largest entry are dropped), and the
 * DCT-domain 1-D filters of each term are formed (kept in FP64 and FP32;
 * for n = 16 also as FP16 tensor-core pieces).  Enables DCTF_KRON_FP32 and,
 * for n = 16, DCTF_KRON_F16X3. */
enum { DCTF_BUILD_KRON = 2u };
dctf_status dctf_build_operator_ex(const double *mask, int mh, int mw,
                                   const int anchor[2], int n,
                                   dctf_boundary boundary, uint32_t flags,
                                   dctf_stream_t stream, dctf_operator **out);

/* Rebuild an existing operator for a new mask of the same n, in place, on
 * `stream` (the paper's point that the prepared matrices are simply rebuilt
 * when the mask changes, Sec. I and IV).  Allocates nothing; the mask travels
 * in the kernel parameters, so the call can be captured in a CUDA graph.
 * Work already queued on other streams that reads the operator must finish
 * first. */
dctf_status dctf_operator_rebuild(dctf_operator *op, const double *mask,
                                  int mh, int mw, const int anchor[2],
                                  dctf_boundary boundary, dctf_stream_t stream);

/* Choose the arithmetic of later dctf_apply calls.  EUNSUPPORTED if no
 * kernel exists for (n, p).  Not synchronised with concurrent applies. */
dctf_status dctf_operator_set_precision(dctf_operator *op, dctf_precision p);

/* Flags for dctf_operator_set_flags.
 * DCTF_APPLY_INPUTS_READY: the caller guarantees that the input of every
 *   dctf_apply through this operator, and the operator itself, are already
 *   in place when the apply is queued (not written by the kernel queued
 *   just before it on the stream).  The 8x8 and 16x16 tensor-core applies
 *   (DCTF_KRON_F16X3 included) are then launched with programmatic stream
 *   serialisation: their CTAs start on SMs the previous kernel has left and
 *   begin reading while that kernel finishes.  No output is written before
 *   the previous kernel has completed.  Ignored by the other kernels. */
enum { DCTF_APPLY_INPUTS_READY = 1u };

/* Set the DCTF_APPLY_* flags of later dctf_apply calls (0 clears them). */
dctf_status dctf_operator_set_flags(dctf_operator *op, uint32_t flags);

/* Read back (synchronously, after the build finished) the FP64 operator M
 * (n2*n2, row-major: row = output coefficient) and, if H_host is not NULL,
 * the spatial operator H (n2*n2, row = output pixel i*n+j).  For tests. */
dctf_status dctf_operator_download(const dctf_operator *op, double *M_host,
                                   double *H_host);

/* Device status word of the operator: 0 when every kernel that used it ran
 * to completion; else the code of the first bounded wait that ran out
 * (bits 0-7 the role, bits 8-31 the tile).  Synchronises the device.  With
 * clear != 0 the word is reset to 0 afterwards. */
dctf_status dctf_operator_status(dctf_operator *op, uint32_t *code, int clear);

/* Number of Kronecker terms of an operator built with DCTF_BUILD_KRON (the
 * numerical rank of its mask; 0 for an all-zero mask), as the device build
 * found it: synchronises the device and reads it back.  EUNSUPPORTED for an
 * operator built without the flag. */
dctf_status dctf_operator_kron_rank(const dctf_operator *op, int *rank);

void dctf_release_operator(dctf_operator *op);

/* y_b = M x_b for b < nblocks (Eq. 11 zero padding, Eq. 20 replication).
 *  coeffs, out  device [nblocks][n2] FP32; out == coeffs (in place) allowed
 *               except for 16x16 blocks with a tensor-core precision; no
 *               other overlap.
 * Arithmetic per dctf_operator_set_precision. */
dctf_status dctf_apply(const dctf_operator *op, const float *coeffs,
                       int64_t nblocks, float *out, dctf_stream_t stream);

/* Filtered uint8 pixels straight from the block-DCT coefficients, one pass
 * (no counterpart kernel in the paper; its Sec. III validation converts the
 * filtered coefficients back to uint8 pixels).  The pixel operator
 * G = H K^T = K^T M (Eq. 3 applied after Eq. 7, K^T K = I) takes a block's
 * coefficients to its filtered pixels; each pixel is rounded half away from
 * zero and saturated to [0, 255].
 *  coeffs  device [nblocks][64] FP32, nblocks = (height/8)*(width/8), raster
 *          block order, 16-byte aligned.
 *  image   device uint8, height rows of `pitch` bytes (pitch >= width, a
 *          multiple of 8; 8-byte aligned); only the height x width pixels
 *          are written.  Must not overlap coeffs.
 * 8x8 operators only (EUNSUPPORTED otherwise); arithmetic F16X3 on tensor
 * cores whatever the operator's precision setting; honours
 * DCTF_APPLY_INPUTS_READY.  Asynchronous on `stream`. */
dctf_status dctf_apply_pixels(const dctf_operator *op, const float *coeffs,
                              int height, int width, uint8_t *image,
                              int64_t pitch, dctf_stream_t stream);

/* dctf_apply (y_b = M x_b, Eq. 11 / Eq. 20) for coefficients in the
 * image-plane layout (a JPEG decoder's coefficient plane): an FP32 array
 * shaped like the pixel image, where coefficient (u, v) of block (by, bx)
 * sits at row 8 by + u, column 8 bx + v.  The kernel reads and writes it with
 * 2-D TMA boxes of 256 floats x 8 rows (32 blocks of one block row; no
 * layout conversion pass).  Same arithmetic as dctf_apply (F16X3 tensor
 * cores).
 *  coeffs, out  device FP32, height rows of pitch / out_pitch floats
 *               (pitches >= width, multiples of 4; 16-byte aligned); only
 *               the height x width coefficients are written.  out == coeffs
 *               (in place, equal pitches) allowed; no other overlap.
 * 8x8 operators only (EUNSUPPORTED otherwise); honours
 * DCTF_APPLY_INPUTS_READY.  Asynchronous on `stream`. */
dctf_status dctf_apply_planar(const dctf_operator *op, const float *coeffs,
                              int height, int width, int64_t pitch, float *out,
                              int64_t out_pitch, dctf_stream_t stream);

/* As dctf_apply (y_b = M x_b, Eq. 11 / Eq. 20), with FP64 input
 * coefficients (FP32 output), FP32 SIMT arithmetic; for the small
 * FP64-coefficient workload. */
dctf_status dctf_apply_f64in(const dctf_operator *op, const double *coeffs,
                             int64_t nblocks, float *out,
                             dctf_stream_t stream);

/* End-to-end call for callers holding the data in HOST memory (the same
 * y_b = M x_b as dctf_apply, Eq. 11 / Eq. 20).  host_in, host_out: [nblocks][N*N] FP32 in
 * host memory, owned by the caller; host_out == host_in allowed, no other
 * overlap (EINVAL).  Two routes, chosen per call:
 *  - 8x8 DCTF_F16X3 with both buffers page-locked and mapped (cudaHostAlloc,
 *    cudaHostRegister; see dctf_host_buffer_direct) and 16-byte aligned: ONE
 *    host-direct launch of the tensor-core kernel, which reads host_in and
 *    writes host_out over the host link itself (no device staging), with the
 *    same arithmetic and result as dctf_apply;
 *  - otherwise host_in is copied to the device, applied and copied back in
 *    8 MB chunks pipelined over four internal streams and device buffers
 *    owned by the operator (allocated by the first such call, 8 x 8 MB).
 * The internal streams are blocking streams: the work starts after work
 * already queued on the legacy default stream (e.g. a rebuild).
 * Synchronous: returns after host_out is written.  Never uses programmatic
 * dependent launch.  Calls on the same operator from several host threads
 * are serialised (the streams and staging are per operator). */
dctf_status dctf_apply_host(dctf_operator *op, const float *host_in,
                            int64_t nblocks, float *host_out);

/* 1 if [p, p + bytes) is host memory that kernels can read and write
 * directly: page-locked, mapped into the device address space, inside one
 * allocation (dctf_apply_host then takes its host-direct route); 0
 * otherwise (pageable memory, device memory, NULL, bytes < 0).  Host-side
 * query, no device work. */
int dctf_host_buffer_direct(const void *p, int64_t bytes);

/* ---------------------------------------------------------------------
 * Grouped apply: many images, each with its own operator, in ONE persistent
 * launch (the same y_b = M x_b of Eq. 11 / Eq. 20 for every block of every
 * item; 8x8 blocks, F16X3 tensor-core arithmetic).  All blocks of all items
 * are split evenly over the persistent CTAs; each CTA switches operators at
 * item boundaries without stalling (operator slots are loaded one segment
 * ahead).
 *
 * DCTF_IO_I16 items hold JPEG-style quantised coefficients: the kernel
 * dequantises x[k] = in[k] * q_in[k] on load and requantises
 * out[k] = sat_int16(round_half_away(y[k] / q_out[k])) on store, so int16
 * data goes from HBM to HBM in one pass. */
typedef enum { DCTF_IO_F32 = 0, DCTF_IO_I16 = 1 } dctf_io;

typedef struct {
    const dctf_operator *op;  /* n = 8 operator (kept alive by the caller)     */
    const void *in;           /* device [nblocks][64] float, or int16 for I16  */
    void *out;                /* same shape and type; == in allowed, no other  */
                              /* overlap                                       */
    int64_t nblocks;          /* >= 0; 0 makes the item a no-op                */
    const uint16_t *q_in;     /* device [64] quantisation table (I16), or NULL */
    const uint16_t *q_out;    /* device [64] output table (I16), or NULL       */
} dctf_group_item;

typedef struct dctf_group dctf_group;

/* Encode every item's TMA descriptors and upload them (synchronous, allocates
 * device memory).  The items' buffers and operators must stay valid while the
 * group is used.  Launch parameters start from the autotuner's cached choice
 * for this size class, else one CTA per SM and 128-row tiles. */
dctf_status dctf_group_create(const dctf_group_item *items, int nitems,
                              dctf_io io, dctf_group **out);

/* One persistent launch over every item, asynchronous on `stream`; no host
 * work, so it can be captured in a CUDA graph and replayed. */
dctf_status dctf_group_launch(const dctf_group *g, dctf_stream_t stream);

/* Set the flags of later launches of the group (0 clears them).
 * DCTF_APPLY_INPUTS_READY: the caller guarantees that every item's input and
 *   operator are already in place when a launch is queued (not written by
 *   the kernel queued just before it on the stream: launching a group whose
 *   items are not in place twice in a row is fine, one with an in-place
 *   item is not).  The launch then uses programmatic
 *   stream serialisation: its CTAs start on SMs the previous kernel has left
 *   and begin reading while that kernel finishes; no output is written
 *   before the previous kernel has completed.  EINVAL for unknown flags. */
dctf_status dctf_group_set_flags(dctf_group *g, uint32_t flags);

/* Autotuner: time each candidate (CTA count x tile height x shared-memory
 * layout, i.e. input stages x operator slots) in `reps` rounds of four
 * back-to-back launches on this group (it really runs the group: no item
 * may be in place; EINVAL otherwise), keep the fastest median for this group and cache it for its (device, kind, size
 * class).  If the environment variable DCTF_TUNE_CACHE names a file, the
 * cache is loaded from it when the first group is created and written back
 * after each tuning.  Synchronises `stream`. */
dctf_status dctf_group_tune(dctf_group *g, dctf_stream_t stream, int reps);

/* The launch parameters in use: CTA count, tile height (64 or 128), input
 * stages and operator slots of the shared-memory layout.  Any output
 * pointer may be NULL. */
dctf_status dctf_group_config(const dctf_group *g, int *grid, int *tile_rows, int *stages,
                              int *slots);

/* Set the launch parameters by hand (grid 0: one CTA per SM).  The
 * (stages, slots) layouts that exist: FP32 coefficient groups (3,2) (2,2)
 * (4,1); int16 groups (4,2) (6,2) (8,1); pixel groups (4,2) (5,2) (6,1).
 * EUNSUPPORTED for another layout; every layout gives the same bits. */
dctf_status dctf_group_set_config(dctf_group *g, int grid, int tile_rows, int stages, int slots);

/* Device status word of the group's launches (as dctf_operator_status). */
dctf_status dctf_group_status(dctf_group *g, uint32_t *code, int clear);

void dctf_group_destroy(dctf_group *g);

/* One-shot form: create, launch on `stream`, wait for it, destroy.  Not for
 * stream capture (it synchronises). */
dctf_status dctf_apply_grouped(const dctf_group_item *items, int nitems,
                               dctf_io io, dctf_stream_t stream);

/* Grouped fused pixel output: many images, each with its own 8x8 operator,
 * from block-DCT coefficients to filtered uint8 pixels in ONE persistent
 * launch (dctf_apply_pixels per item: the pixel operator H K^T, Eq. 3 after
 * Eq. 7, round half away from zero and saturate, Sec. III).  Each item:
 *   coeffs : device [ (height/8) * (width/8) ][64] FP32, raster block order,
 *            16-byte aligned (caller-owned, read only);
 *   image  : device uint8, `height` rows of `pitch` bytes, 8-byte aligned;
 *            only the height x width pixels are written; must not overlap
 *            coeffs;
 *   height, width: positive multiples of 8; pitch >= width, multiple of 8.
 * The group is used like a coefficient group: dctf_group_launch (graph-
 * capturable), dctf_group_tune (needs no in-place care: inputs are never
 * written), dctf_group_config, dctf_group_status, dctf_group_destroy.
 * EINVAL on a bad item (nothing is allocated), EUNSUPPORTED for an operator
 * that is not 8x8. */
typedef struct {
    const dctf_operator *op;  /* n = 8 operator (kept alive by the caller)     */
    const float *coeffs;
    int height, width;
    uint8_t *image;
    int64_t pitch;            /* bytes per image row                          */
} dctf_pixel_item;

dctf_status dctf_group_create_pixels(const dctf_pixel_item *items, int nitems,
                                     dctf_group **out);

/* ---------------------------------------------------------------------
 * Serving: a continuous-batching request loop for JPEG-style quantised
 * planes (the library's serving form of the per-block filter; the paper has
 * no serving system).  A request carries 1-4 int16 planes [nblocks][64] with
 * one quantisation table each (used to dequantise the input and requantise
 * the output) and one 8x8-block mask.  A worker thread admits waiting
 * requests in arrival order while a batch slot is free and their device
 * memory fits in the HBM budget, reuses or builds their operators (device
 * cache keyed by mask, anchor and boundary; FP64 build), and runs each batch
 * as grouped launches with dequantise / requantise fused (one for the planes
 * it reads and writes in host memory itself, one for planes staged in HBM); up to
 * max_inflight batches overlap on the device.  Results do not depend on the
 * batch a request lands in. */
typedef struct {
    size_t hbm_budget_bytes;        /* device arena for request planes (>= 1 MiB) */
    int max_inflight;               /* batches in flight at once (1..8)           */
    int max_batch_requests;         /* requests per batch (>= 1)                  */
    int op_cache_capacity;          /* cached operators (>= 1)                    */
    int inject_build_failure_every; /* test hook: fail every k-th build (0 off)   */
    int staged_only;                /* nonzero: every request takes the staged    */
                                    /* route (HBM arena, admission by the budget), */
                                    /* page-locked planes included                 */
} dctf_server_cfg;

typedef struct {
    int nplanes;                    /* 1..4                                        */
    const int16_t *in[4];           /* host [nblocks][64], read during the call... */
    int16_t *out[4];                /* ...and written before wait returns          */
    int64_t nblocks[4];             /* > 0                                         */
    const uint16_t *q[4];           /* host [64] quantisation table per plane: the */
                                    /* input is dequantised with it                */
    const double *mask;             /* host row-major mh x mw, copied at submit    */
    int mh, mw;                     /* 1..8                                        */
    int anchor[2];
    dctf_boundary boundary;
    const uint16_t *q_out[4];       /* host [64] table the output is requantised   */
                                    /* with, or NULL for the plane's q (copied at  */
                                    /* submit)                                     */
} dctf_request;

typedef struct {
    double p50_ms, p99_ms, mean_ms, max_ms;  /* submit -> result in host buffer */
    double wall_s;                           /* first submit -> last completion */
    uint64_t completed, failed, batches, blocks, cache_hits, cache_misses;
    int max_batch_requests_seen;
    size_t hbm_in_use;
    uint64_t direct_requests;                /* completed on the host-direct route */
    uint64_t budget_waits;                   /* requests that waited for HBM: at the
                                                head of the queue, with a batch slot
                                                free, they did not fit the budget's
                                                free space until others finished  */
    size_t hbm_peak;                         /* most budget bytes in use at once  */
} dctf_stats;

typedef struct dctf_server dctf_server;

/* Allocate the HBM arena, pinned staging of the same size and the batch
 * slots on the current device; start the worker thread. */
dctf_status dctf_server_create(const dctf_server_cfg *cfg, dctf_server **out);

/* Queue a request: every plane is dequantised with its table q, filtered
 * block by block (y_b = M x_b, Eq. 11 / Eq. 20) and requantised with its
 * table q_out (q when q_out is NULL).  Its
 * host buffers must stay valid until dctf_server_wait returns for its
 * ticket.  Routes, chosen per request at submit:
 *  - host-direct (unless the server was created staged_only): every
 *    plane's input and output is page-locked, mapped
 *    memory (cudaHostAlloc, cudaHostRegister), 16-byte aligned, and no two
 *    of the request's buffers overlap except a plane filtered in place
 *    (in == out).  The batch kernel reads and writes these planes over the
 *    host link itself; the request takes no HBM from the budget.
 *  - staged: otherwise.  Page-locked buffers are copied by DMA directly,
 *    others go through the server's pinned staging; EBUDGET if the planes
 *    can never fit the HBM budget.
 * Both routes give the same bits. */
dctf_status dctf_server_submit(dctf_server *s, const dctf_request *req,
                               uint64_t *ticket);

/* Wait up to timeout_ms for a request: DCTF_OK once its outputs are written,
 * ETIMEOUT if still running (the ticket stays valid), or the request's own
 * error (the server keeps running).  A finished ticket is then retired. */
dctf_status dctf_server_wait(dctf_server *s, uint64_t ticket, int timeout_ms);

dctf_status dctf_server_stats(dctf_server *s, dctf_stats *out);

/* Start a new statistics window: clears the latencies and every counter of
 * dctf_stats (hbm_peak restarts at the bytes in use); the operator cache,
 * queued and running requests are untouched (requests still running when
 * it is called count in the new window, with their original submit time).
 * For measuring a steady state after a warm-up. */
dctf_status dctf_server_reset_stats(dctf_server *s);

/* Finish every queued and running request, then free everything. */
void dctf_server_destroy(dctf_server *s);

/* Blockwise forward DCT of a uint8 image (Sec. II.A, Eq. 1): block (by, bx)
 * in raster order b = by*(width/n) + bx gets BLOCK = C block C^T, written as
 * coeffs[b][u*n + v].  image: device, height x width bytes, row pitch `pitch`
 * >= width; height and width multiples of n.  FP64 arithmetic; the FP32
 * variant rounds the result once.  Asynchronous on `stream`. */
dctf_status dctf_forward_dct(const uint8_t *image, int height, int width,
                             int64_t pitch, int n, float *coeffs,
                             dctf_stream_t stream);
dctf_status dctf_forward_dct_f64(const uint8_t *image, int height, int width,
                                 int64_t pitch, int n, double *coeffs,
                                 dctf_stream_t stream);

/* Forward DCT (Sec. II.A, Eq. 1) followed by JPEG-style quantisation with a
 * per-coefficient table q (device, n*n entries; the quantisation is codec
 * practice, not part of the paper): coeffs[b][k] = sat_int16(
 * round_half_away(BLOCK[k] / q[k])).  Prepares int16 input for the
 * quantised grouped path. */
dctf_status dctf_forward_dct_i16(const uint8_t *image, int height, int width,
                                 int64_t pitch, int n, const uint16_t *q,
                                 int16_t *coeffs, dctf_stream_t stream);

/* Inverse of dctf_forward_dct followed by the uint8 conversion of Sec. III:
 * block = C^T BLOCK C (Eq. 3), rounded half away from zero and saturated to
 * [0, 255], written into a device image of the given pitch.  FP64 inside. */
dctf_status dctf_inverse_dct_u8(const float *coeffs, int height, int width,
                                int n, uint8_t *image, int64_t pitch,
                                dctf_stream_t stream);

/* Allocation-free build: the same FP64 operator M (and optionally the
 * spatial operator H) that dctf_build_operator makes for one mask, written
 * into memory the caller provides; the library allocates nothing.  The
 * paper has no counterpart: this exists for callers that cannot call
 * cudaMalloc -- code inside a framework whose pool owns all device memory,
 * real-time paths where cudaMalloc's implicit device synchronisation is not
 * allowed, plug-ins that are handed only the buffers they read and write.
 *  M_out  device, n2*n2 doubles (row = output coefficient), 16-byte aligned.
 *  H_out  device, n2*n2 doubles (row = output pixel i*n+j), or NULL.
 * Same mask, anchor and boundary arguments and checks as
 * dctf_build_operator; asynchronous on `stream`.  The build's scratch is a
 * static 1 MiB device array inside the library (2 n^4 doubles: enough for
 * the largest block, n = 16); a block side beyond it (n > 16) is rejected
 * with DCTF_EINVAL and a message naming the scratch limit.  The first call
 * in a CUDA context (the first on a device, or the first after a device
 * reset) looks up that array's device address, so make it before any
 * stream capture.  Every call shares the array, which keeps the last
 * call's contents: calls that overlap on the GPU (different streams, or
 * several host threads) race and must be serialised by the caller. */
dctf_status dctf_build_matrix_noalloc(const double *mask, int mh, int mw,
                                      const int anchor[2], int n,
                                      dctf_boundary boundary, double *M_out,
                                      double *H_out, dctf_stream_t stream);

/* Self-test of the device-side failure handling the tensor-core kernels
 * use (no counterpart in the paper): one CTA waits, with a bound of
 * limit_us microseconds (1..100000), on a barrier nothing ever completes.
 * The waiting role must give up, record its code (0x101) and raise the
 * CTA's abort flag; a second role waiting elsewhere must leave through that
 * flag (other_role_aborted = 1).  The kernel returns normally: nothing
 * faults or hangs.  Synchronous; returns DCTF_ETIMEOUT when the timeout was
 * detected as designed. */
dctf_status dctf_selftest_wait_timeout(uint32_t limit_us, uint32_t *code,
                                       uint32_t *other_role_aborted);

/* Message of the last failed call on this thread ("" if none). */
const char *dctf_last_error(void);

/* Library version, major*10000 + minor*100 + patch. */
int dctf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DCTF_H */
