/*
 * kf.h -- C ABI of the GB300 (sm_103a) multi-scale shape-filter bank.
 *
 * Kennedy, "Digital filters with vanishing moments for shape analysis"
 * (arXiv:1912.07133).  A low-pass blur (repeated-pole IIR "Filter D",
 * Sec. 4.3 / Table IV; discrete Butterworth IIR "Filter E", Sec. 4.4;
 * colored Savitzky-Golay FIR "Filter C", Sec. 4.2) is cascaded with the
 * derivative filters of Table I and a scale-space extremum detector (Sec. 5,
 * eqs 26-27).  Every stage runs in the library's CUDA kernels.
 *
 * Conventions
 *   - Status codes: 0 (KF_OK) or a negative KF_E* value.  No C++ exception
 *     crosses this boundary.  kf_last_error() describes the last failure of a
 *     context (thread-unsafe per context; use one context per thread).
 *   - Pointers named "device" must be CUDA device pointers on the context's
 *     device; "host" pointers are ordinary host memory.  The caller owns every
 *     pointer it passes; the library never frees them.  The context owns its
 *     workspace (intermediate planes, carries, candidate list).
 *   - Images are row-major: element (x, y) of a frame is data[y * pitch + x],
 *     0 <= x < width, 0 <= y < height, pitch >= width (in elements).
 *   - Scales are blob radii lambda in pixels; the filters use
 *     sigma = lambda / 2 (Sec. 5).
 */
#ifndef KF_H
#define KF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define KF_OK 0
#define KF_EINVAL -1     /* invalid argument (sizes, enums, sigma, pointers)   */
#define KF_ECOND -2      /* a filter design failed (singular / ill-conditioned) */
#define KF_ENOMEM -3     /* device allocation failed                            */
#define KF_ECUDA -4      /* a CUDA runtime call or kernel launch failed         */
#define KF_ETIMEOUT -5   /* a bounded device-side wait gave up                  */
#define KF_EOVERFLOW -6  /* output capacity too small; *count holds the need    */
#define KF_ENODEV -7     /* no usable CUDA device                               */
#define KF_ERERUN -8     /* the context's candidate list overflowed during the
                            last bank call; its capacity has been raised: run
                            kf_filter_bank again (*count holds the need)       */
#define KF_ERANGE -9     /* with f16 storage, a plane value exceeded 65504: the
                            responses of that call are not finite; scale the
                            input down (value_scale) or store bf16 / f32       */

/* ---- enumerations -------------------------------------------------------- */
#define KF_IIR_REPEATED_POLE 0 /* Filter D, Sec. 4.3 / Table IV                  */
#define KF_IIR_BUTTERWORTH 1   /* Filter E, Sec. 4.4                             */
#define KF_FIR_COLORED_SG 2    /* Filter C, Sec. 4.2                             */
#define KF_FIR_GAUSSIAN 3      /* Filter A, Sec. 3.1 (the paper's Gaussian FIR
                                  comparison blur)                              */
#define KF_NTYPES 4

/* Element types.  Input frames: any of the four; each element is converted
 * to f32 and multiplied by the frame's value_scale.  Intermediate planes
 * (kf_bank_opts.storage): f32, f16 or bf16; every recursion, tap sum and
 * response is computed in f32 whatever the storage. */
#define KF_DTYPE_F32 0
#define KF_DTYPE_F16 1  /* IEEE binary16                                       */
#define KF_DTYPE_BF16 2 /* bfloat16                                            */
#define KF_DTYPE_U16 3  /* unsigned 16-bit counts (input only)                 */

#define KF_RESP_LAPLACIAN 0 /* R_L = -sigma^2 (D20 + D02)                        */
#define KF_RESP_HESSIAN 1   /* R_H = sigma^4 (D20 D02 - D11^2), eq (26); bright
                               maxima only.  R_H and Threshold #2 run the
                               derivative bank: each needed derivative (D20,
                               D02, D11; D10, D01 for eq 27) is blurred as its
                               own channel (Table I taps first), then one
                               kernel forms R and detects.  Not with gating
                               or graph replay (calls run eagerly).          */

#define KF_BOUNDARY_HOLD 0 /* frame edges held to +-infinity (Appendix, A32)     */
#define KF_BOUNDARY_ZERO 1 /* frame extended by zeros (the FIR initialisation
                              of Sec. 5); FIR blurs (Filters A, C) with the
                              Laplacian response and no offset limit only    */

#define KF_GATE_OFF 0        /* no proposal gating                               */
#define KF_GATE_DILATED 1    /* marked tiles and their 8 neighbours              */
#define KF_GATE_TILES 2      /* marked tiles only                                */

#define KF_SCHED_BATCHED 0   /* one persistent launch per pass for all frames   */
#define KF_SCHED_PER_FRAME 1 /* every pass launched once per frame              */

#define KF_NEIGH_ALL_SCALES 0 /* extremum over 3 x 3 x (all scales)            */
#define KF_NEIGH_ADJACENT 1   /* extremum over 3 x 3 x (scale -1, 0, +1)       */

#define KF_MAX_SCALES 16
#define KF_MAX_ORDER 8
#define KF_MAX_FIR_K 160

/* ---- data structures ------------------------------------------------------ */

/* Coefficients of one designed blur (host-side copy of the FP64 design).
 * IIR (types 0, 1): three-term DE of eqs (A6)-(A10): y = y+ + y- + b0 x with
 *   y+(n) = sum_{m=1..K} bplus[m] x(n-m) - sum_{m=1..K} aplus[m] y+(n-m),
 *   y- the mirror image (b- = b+, a- = a+), aplus[0] = 1, bplus[0] = 0.
 * FIR (type 2): taps h[0..K], h(-m) = h(m), eq (A5).
 * dc_gain and moment2 are the realised sum h(m) and sum m^2 h(m) (design
 * self-check; 1 and 0 by construction, eq 7). */
typedef struct {
  int32_t type, order, K, reserved;
  double scale;  /* lambda (px) */
  double sigma;  /* lambda / 2 */
  double param;  /* D: pole p = exp(-1/sigma); E: cut-off omega_c; C: omega_c */
  double b0;
  double bplus[KF_MAX_ORDER + 1];
  double aplus[KF_MAX_ORDER + 1];
  double h[KF_MAX_FIR_K + 1];
  double dc_gain;
  double moment2;
} kf_coeffs;

/* One input frame (device memory). */
typedef struct {
  const void *data;    /* device pointer, dtype elements, aligned to the element */
  int32_t width;       /* 1 .. 8192                                            */
  int32_t height;      /* >= 1                                                 */
  int64_t pitch;       /* elements between rows, >= width                      */
  int32_t dtype;       /* KF_DTYPE_*                                           */
  float value_scale;   /* input multiplier (e.g. 1/4095 for 12-bit counts); 0 = 1 */
} kf_frame;

/* Options of one filter-bank call. */
typedef struct {
  int32_t response;      /* KF_RESP_*                                          */
  int32_t boundary;      /* KF_BOUNDARY_HOLD, or KF_BOUNDARY_ZERO for the FIR
                            blurs with the Laplacian response               */
  int32_t neighbourhood; /* KF_NEIGH_*                                         */
  int32_t storage;       /* element type of the one-sided planes between the
                            row and column passes: KF_DTYPE_F32 / F16 / BF16.
                            16-bit planes halve their traffic; they hold
                            sigma^2 x the row-blurred derivative, so their
                            values have the magnitude of R at every scale.
                            Responses and the detector stay f32.            */
  double threshold;      /* Threshold #1: |R| > threshold to be a candidate    */
  int32_t fir_kmax;      /* cap on the colored-SG half-length (0 -> 96)        */
  int32_t profile;       /* 1: record CUDA events around every kernel of the
                            call on the context stream (kf_kernel_times)       */
  float *responses;      /* optional device output, f32: for frame f, scale s,
                            R at (x, y) is responses[off_f + (s*H + y)*W + x],
                            off_f = sum over earlier frames of nscales*H*W.
                            NULL: not written.                                 */
  int32_t schedule;      /* KF_SCHED_BATCHED: each pass is one launch over
                            the work items of all frames of the call (the IIR
                            row pass one launch per block-width class);
                            KF_SCHED_PER_FRAME: every pass launched frame by
                            frame.  Same results either way.                 */
  int32_t graph;         /* 1: replay the call's launches from a CUDA graph.
                            The first call of a geometry runs eagerly; the
                            second captures the launches (status reset + all
                            passes) and every later call of the same geometry
                            replays them after uploading the frame table
                            (frame pointers, pitches, value scales and
                            response pointers may change between calls).
                            Geometry = type, order, scales, fir_kmax,
                            storage, threshold, neighbourhood, schedule,
                            frame count and each frame's width and height.
                            Ignored when profile = 1.                        */
  int32_t gate;          /* KF_GATE_*: proposal gating (needs
                            kf_proposal_set_weights, <= 8 scales, the batched
                            schedule).  Per frame the proposal network marks
                            64 x 64 tiles whose logit of some scale exceeds
                            logit(gate_threshold) in the tile
                            (KF_GATE_TILES) or in the tile or one of its 8
                            neighbours (KF_GATE_DILATED); only column-pass tiles
                            overlapping marked tiles run (all scales: the
                            extremum over scales stays exact), and for the FIR
                            bank only the row-pass rows they read.  Every blob
                            reported is the full bank's blob; blobs in unmarked
                            tiles are not found, and responses there are not
                            written.                                          */
  float gate_threshold;  /* probability threshold of the gate, in (0, 1)     */
  float offset_limit;    /* Threshold #2 (Sec. 5): > 0 keeps only candidates
                            whose eq (27) offset sqrt(dx^2 + dy^2) is at most
                            this many pixels; 0: off                          */
  int32_t gate_reuse;    /* gated calls: 1 reuses the tile marks of the
                            previous gated call on this context instead of
                            running the proposal network again (the marks
                            depend on the frames, the weights, the scale count,
                            the gate mode and threshold, not on the filter
                            type): the call must have the same frame count and
                            sizes, scale count, gate mode and threshold, with
                            no weight change since, else KF_EINVAL; the caller
                            guarantees that the frames hold the same values.
                            0: evaluate the network.                         */
  int64_t reserved[1];
} kf_bank_opts;

/* One detection (Threshold #1 extremum). */
typedef struct {
  int32_t frame, x, y, scale;
  int32_t polarity;  /* +1 bright (maximum of R), -1 dark (minimum of R_L) */
  float response;    /* R at (x, y, scale) */
  float dx, dy;      /* sub-pixel offset of the extremum by eq (27) (the
                        derivative bank: R_H or offset_limit > 0; else 0) */
} kf_blob;

/* Shape of one blob (Sec. 5: the blurred image's Hessian H = [[D20, D11],
 * [D11, D02]] at the detection read as minus the Fisher information of the
 * blob taken as a pdf, P = (-pol H)^-1 its covariance, pol = +1 for a bright
 * blob (D20 + D02 < 0), -1 for a dark one).  16 bytes. */
typedef struct {
  float p1, p2;  /* eigenvalues of P, p1 >= p2 (pixels^2); NaN where -pol H is
                    not positive definite (a saddle)                           */
  float theta;   /* orientation of the p1 axis: radians from +x towards +y, in
                    (-pi/2, pi/2] (undefined when p1 = p2)                     */
  float det;     /* |H| = D20 D02 - D11^2 (1 / pixels^4)                       */
} kf_blob_shape;

/* Per-kernel device time of the last profiled kf_filter_bank call. */
typedef struct {
  char name[32];     /* kernel name                                   */
  int32_t launches;  /* launches of this kernel in the call            */
  float ms;          /* summed CUDA-event time of those launches (ms)  */
} kf_kernel_time;

typedef struct kf_ctx kf_ctx;

/* ---- entry points --------------------------------------------------------- */

/* Fill *opts with defaults: Laplacian response, hold boundary, all-scales
 * neighbourhood, f32 storage, threshold 0.05, fir_kmax 96, no responses.
 * Returns KF_OK or KF_EINVAL (NULL). */
int kf_bank_opts_default(kf_bank_opts *opts);

/* Create a context on CUDA device `device`, issuing all work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *ctx receives the
 * handle (host).  Errors: KF_EINVAL (ctx NULL), KF_ENODEV, KF_ECUDA. */
int kf_create(kf_ctx **ctx, int device, void *cuda_stream);

/* Free the context and its workspace (synchronises its stream).  NULL is a
 * no-op. */
void kf_destroy(kf_ctx *ctx);

/* Message for the last failure on this context ("" if none); valid until the
 * next call on the context.  ctx NULL gives the message of the last
 * context-less call (kf_design). */
const char *kf_last_error(const kf_ctx *ctx);

/* Design one blur in FP64 on the current CUDA device (Sec. 4; the same
 * design kernel kf_filter_bank runs) and copy it to *out (host, caller-owned).
 *   type  KF_IIR_REPEATED_POLE: order = K^lpf = L_D + Lpi with L_D = 1
 *         (3 = Table IV, 4 = the fourth-order blur); p = exp(-1/sigma)
 *         (Sec. 4.3).
 *         KF_IIR_BUTTERWORTH: order = L_B / 2 = L_D + 1 (2 for D = 3);
 *         omega_c = sqrt(2 ln 2) / sigma, bilinear transform (Sec. 4.4).
 *         KF_FIR_COLORED_SG: order = L_D (1 or 2); K = ceil(5 sigma)
 *         (ceil(7 sigma) for L_D = 2) capped at 96, omega_c = 3 / sigma
 *         (Sec. 4.2).
 *         KF_FIR_GAUSSIAN: order = 1; the Gaussian of eq 9 (d = 0) sampled
 *         at |m| <= K = ceil(5 sigma) (capped at 96) and renormalised to
 *         unit dc gain (eq 11) (Sec. 3.1).
 *   scale lambda in pixels, sigma = lambda / 2 (Sec. 5).
 * Errors: KF_EINVAL (bad type/order, sigma <= 0, colored SG with
 * 3/sigma >= pi), KF_ECOND (design solve failed), KF_ENODEV, KF_ECUDA. */
int kf_design(int type, int order, double scale, kf_coeffs *out);

/* Run the bank on `nframes` frames (host array of descriptors pointing to
 * device images) for `nscales` scales (host array of lambdas, ascending not
 * required, <= KF_MAX_SCALES) with one blur type/order: designs (FP64
 * kernel), separable blur of the derivative-filtered frame (Table I taps),
 * response and the scale-space extremum detector (Sec. 5).  Candidates with
 * |R| > opts->threshold are kept in the context for kf_detect_blobs; a new
 * call replaces them.  Asynchronous on the context stream: the frames must
 * stay valid until the stream reaches this work.
 * All frames of a call stay resident in the context's workspace (their
 * one-sided planes, edge rows and carries): a call of many large frames needs
 * S x (sum of frame pixels) plane elements; split the batch if KF_ENOMEM.
 * Errors: KF_EINVAL (arguments, unsupported option), KF_ECOND, KF_ENOMEM,
 * KF_ECUDA. */
int kf_filter_bank(kf_ctx *ctx, const kf_frame *frames, int nframes,
                   const double *scales, int nscales, int type, int order,
                   const kf_bank_opts *opts);

/* Copy the candidates of the last kf_filter_bank call with |R| > threshold
 * into out[0..capacity) (host, caller-owned), sorted by (frame, scale, y, x);
 * *count (host) receives the number of such blobs; entries of out past
 * *count may be overwritten.  threshold must be >= the bank's
 * opts->threshold.  Synchronises the context stream (once per call: the
 * ordering, the count and the copy share one synchronisation; pinned `out`
 * memory copies fastest).
 * Errors: KF_EINVAL, KF_EOVERFLOW (capacity < *count; the first `capacity`
 * blobs are written), KF_ERERUN (the device-side candidate list of the last
 * call overflowed; capacity raised, run the bank again), KF_ERANGE (f16
 * storage overflowed in the last call), KF_ETIMEOUT, KF_ECUDA. */
int kf_detect_blobs(kf_ctx *ctx, double threshold, kf_blob *out,
                    int64_t capacity, int64_t *count);

/* Shapes of the blobs kf_detect_blobs(ctx, threshold, ...) returns, in the
 * same order: out[0..capacity) (host, caller-owned), *count (host) the number
 * of blobs.  Needs a last kf_filter_bank call that ran the derivative bank
 * (opts.response = KF_RESP_HESSIAN or opts.offset_limit > 0): the derivatives
 * are read from its planes at each blob's scale and pixel.  Synchronises the
 * context stream.
 * Errors: KF_EINVAL (no derivative-bank result, bad arguments, threshold
 * below the bank's), KF_EOVERFLOW (capacity < *count; the first `capacity`
 * shapes are written), and those of kf_detect_blobs. */
int kf_blob_shapes(kf_ctx *ctx, double threshold, kf_blob_shape *out, int64_t capacity, int64_t *count);

/* ---- the D = 5 derivative bank (L_D = 2) ----------------------------------
 * Sec. 4 with D = 2 L_D + 1 = 5: every derivative D_{dx,dy} (eq 3) with
 * dx + dy <= 4 of the quartic model (eq 1) at each scale, estimated by
 * separable filters whose moments vanish up to order 4: the differentiator
 * g_d of Sec. 4.1 (eqs 12-17, pure-delay basis, dc constraints; the five-point
 * central differences) along x and along y, cascaded with a blur flat at dc
 * to order 4.  Channel c of a set holds (dx, dy) with n = dx + dy, c =
 * n (n + 1) / 2 + dy: (0,0); (1,0) (0,1); (2,0) (1,1) (0,2); (3,0) (2,1)
 * (1,2) (0,3); (4,0) (3,1) (2,2) (1,3) (0,4).  x is the column index, y the
 * row index; the frame is held beyond its edges (the hold boundary). */
#define KF_QUARTIC_CHANNELS 15

/* D_{dx,dy} of one frame at nscales scales.
 *   frame   one device frame (any KF_DTYPE_*, value_scale applied), width
 *           <= 8192
 *   scales  host, nscales values lambda > 0 (sigma = lambda / 2), 1..16
 *   type, order  the blur: KF_IIR_REPEATED_POLE with order = K^lpf = L_D +
 *           Lbar_pi in 3..6 (L_D = 2 design of Sec. 4.3; at least one Nyquist
 *           constraint, without which the design is the unit impulse),
 *           KF_IIR_BUTTERWORTH with order = L_B / 2 in 3..6 (flat to order
 *           L_B - 1 >= 5), or
 *           KF_FIR_COLORED_SG with order = L_D = 2 (K = ceil(7 sigma) <= 96,
 *           omega_c = 3 / sigma, Sec. 4.2)
 *   out     device, f32, caller-owned: nscales x 15 planes of H x W,
 *           out[((s * 15 + c) * H + y) * W + x]
 *   profile 1: time every kernel launch with CUDA events (the stream is
 *           synchronised after each channel); kf_kernel_times then returns
 *           the per-kernel totals of this call.  0: no timing.
 * Runs on the context stream (asynchronous unless profiling; out is complete
 * when the stream is).  Uses the context's bank: afterwards kf_detect_blobs
 * has no result until the next kf_filter_bank call.  The recursive blurs run
 * on 32-row column segments unless kf_set_segment_length or kf_autotune
 * chose a length for the type.
 * Errors: KF_EINVAL (bad arguments, a type or order without vanishing
 * moments to order 4), KF_ECOND (design), KF_ECUDA. */
int kf_quartic_bank(kf_ctx *ctx, const kf_frame *frame, const double *scales, int nscales, int type,
                    int order, float *out, int profile);

/* Steered derivatives (Sec. 2, after eq 3): with x~ = x cos(phi) + y sin(phi)
 * and y~ = -x sin(phi) + y cos(phi), the coefficients beta (eq 2: beta_{dx,dy}
 * = D_{dx,dy} / (dx! dy!)) of the polynomial in (x~, y~) are re-expressed as
 * the coefficients of the same polynomial in (x, y); each total order maps
 * to itself.  in, out: device f32, nsets sets of 15 channel planes of npix
 * pixels each (the layout of kf_quartic_bank's out: nsets = nscales, npix =
 * H W); out may equal in.  Asynchronous on the context stream.
 * Errors: KF_EINVAL (NULL pointers, npix < 1, nsets < 1), KF_ECUDA. */
int kf_quartic_steer(kf_ctx *ctx, const float *in, int64_t npix, int nsets, double phi, float *out);

/* Kernel launches and, when the call ran with opts->profile = 1, per-kernel
 * CUDA-event times of the last kf_filter_bank call (or of the last
 * kf_quartic_bank call with profile = 1, until the next kf_filter_bank call): fills out[0..cap) (host,
 * caller-owned) and sets *n (host) to the number of distinct kernels.
 * Synchronises the context stream.  Without profiling, ms is 0.
 * Errors: KF_EINVAL (NULL arguments, no bank call yet), KF_ECUDA. */
int kf_kernel_times(kf_ctx *ctx, kf_kernel_time *out, int cap, int *n);

/* Passes of a bank (launch-shape tuning).  Recursive banks: row pass (with
 * the edge rows), column segment states, carry fold, column pass + detector.
 * FIR bank: row pass, column pass + detector. */
#define KF_PASS_ROW 0
#define KF_PASS_SEG 1
#define KF_PASS_FOLD 2
#define KF_PASS_DET 3
#define KF_NPASS 4

/* Launch shape of one pass of one filter type on this context.  Every pass is
 * a grid of blocks that take the call's work items (rows, column tiles, ...)
 * in turn:
 *   grid_mult = 0  one block per work item (the default);
 *   grid_mult = k  at most k x (blocks resident per SM for this kernel and
 *                  block size) x (SMs) blocks, each looping over items;
 *   grid_mult = -b at most b blocks per SM (b = 1..16, capped at the blocks
 *                  resident per SM) x (SMs): the pass takes a share of every
 *                  SM and leaves the rest to kernels of other streams (banks
 *                  of other contexts running at the same time).
 * The tensor-core FIR column pass is always one block per SM and ignores the
 * setting.  Results do not depend on the shape.  Errors: KF_EINVAL
 * (grid_mult outside -16..64). */
int kf_set_launch_shape(kf_ctx *ctx, int type, int pass, int grid_mult);

/* Column segment length (scan block length of the column recursions) of a
 * recursive bank on this context: 32 or 64 rows (default 64).  Shorter
 * segments halve the column pass's shared-memory tile and registers (more
 * resident blocks) at the cost of twice as many carries.  Results agree to
 * FP32 rounding.  Errors: KF_EINVAL. */
int kf_set_segment_length(kf_ctx *ctx, int type, int rows);

/* Column pass of a recursive bank on this context (Sec. 5: the column blur
 * of the separable filter, both one-sided recursions of eq A6 along y).
 *   KF_COLUMN_SINGLE_READ: each plane tile is read from device
 *     memory once; the carries of the recursions between tiles are exchanged
 *     while the tiles stay in shared memory (clusters of 8 tiles of 32 rows;
 *     between clusters through end states published in device memory and
 *     folded in a fixed order, so results repeat bit for bit).  Used for
 *     calls whose tallest frame's column strips fit on the GPU at once, with
 *     the segment passes otherwise.  With gating, every tile is still read
 *     (the carries need it); the final pass and the detector run on the
 *     selected tiles.
 *   KF_COLUMN_SEGMENTS (default): the segment end states, the carry fold
 *     and the final column pass as three passes (the planes are read twice;
 *     no pass waits on another block, and on the measured workloads this is
 *     the faster form).
 * kf_autotune times both and keeps the faster.  Results agree to FP32
 * rounding.  Errors: KF_EINVAL. */
#define KF_COLUMN_SINGLE_READ 0
#define KF_COLUMN_SEGMENTS 1
int kf_set_column_pass(kf_ctx *ctx, int type, int mode);

/* Failure-detection test hook.  polls > 0: the column pass of the recursive
 * banks issues no copy to its shared-memory load barrier, so that its bounded
 * wait (at most `polls` polls, each parking the warp for about a microsecond)
 * gives up on every tile: the next kf_filter_bank call then makes
 * kf_detect_blobs return KF_ETIMEOUT (no asynchronous copy is left in flight,
 * and the context stays usable).  polls = 0 restores the normal loads and
 * waits.  ctx NULL sets the hook of kf_responses_noalloc, which then returns
 * KF_ETIMEOUT.  Paper: none (tests of the failure path).
 * Errors: KF_EINVAL (polls outside 0..2^20). */
int kf_set_wait_limit(kf_ctx *ctx, int polls);

/* Autotuner: run the bank on these frames (as kf_filter_bank would, opts as
 * there) once per candidate shape (grid_mult 1, 2, 4, 0) and, for the
 * recursive banks, per column pass (segments of 64 rows, of 32 rows, the
 * single-read pass); time every pass with CUDA events on the context
 * stream; keep for `type` the column pass with the smallest sum of per-pass
 * best times and for each pass its fastest shape.  chosen (host, KF_NPASS +
 * 1 entries, may be NULL) receives the shapes (passes the type or the
 * chosen column pass lacks: -1) and, last, the segment length (0: the
 * single-read column pass; -1 for the FIR bank); ms_out (host, KF_NPASS x
 * 4, may be NULL) the per-pass times of the shape candidates at the chosen
 * column pass (ms).
 * Leaves the last candidate's result as the context's bank result.
 * Synchronises the context stream.  Errors: those of kf_filter_bank. */
int kf_autotune(kf_ctx *ctx, const kf_frame *frames, int nframes,
                const double *scales, int nscales, int type, int order,
                const kf_bank_opts *opts, int32_t *chosen, float *ms_out);

/* ---- proposal network (gating) --------------------------------------------
 * A small convolutional network, with no counterpart in the paper, predicts
 * per 64 x 64-pixel tile and scale whether the bank can find a blob there;
 * kf_filter_bank with opts->gate = 1 then runs the detector's work only on
 * tiles it marks (plus their neighbours).  Definition (all products with the
 * bf16 rounding of the FP32 master weights, all sums in FP32):
 *   pooled p = 8 x 8 block means of the frame times its value scale
 *              (ceil(H/8) x ceil(W/8); partial blocks average what they hold)
 *   a1 = relu(conv3x3(p; 1 -> 16)), a2 = relu(conv3x3(a1; 16 -> 16)),
 *   o3 = conv3x3(a2; 16 -> 8)   (cross-correlation, zero padding, + bias)
 *   logit[c][ty][tx] = max of o3[c] over pooled pixels [8ty, 8ty+8) x [8tx, 8tx+8)
 * Channel c is scale c of the bank (banks of up to 8 scales).
 * Parameters: KF_NET_NPARAM floats W1[16][1][3][3] b1[16] W2[16][16][3][3]
 * b2[16] W3[8][16][3][3] b3[8].  Training: mean over logits of
 * pw t softplus(-z) + (1 - t) softplus(z), Adam (0.9, 0.999, 1e-8). */
#define KF_NET_NPARAM 3640
#define KF_NET_CHANNELS 8

/* Set the FP32 master weights (host array of KF_NET_NPARAM) and reset the
 * Adam state.  Errors: KF_EINVAL, KF_ENOMEM, KF_ECUDA. */
int kf_proposal_set_weights(kf_ctx *ctx, const float *weights);

/* Copy the FP32 master weights to weights (host, KF_NET_NPARAM); synchronises
 * the context stream.  Errors: KF_EINVAL (NULL, no weights set), KF_ECUDA. */
int kf_proposal_get_weights(kf_ctx *ctx, float *weights);

/* Pooled frames: for frame f, ceil(H/8) x ceil(W/8) floats, frames back to
 * back in `pooled` (device, caller-owned).  Asynchronous.
 * Errors: KF_EINVAL, KF_ECUDA. */
int kf_proposal_pool(kf_ctx *ctx, const kf_frame *frames, int nframes, float *pooled);

/* Logits of n pooled images pooled[n][h][w] (device) into
 * logits[n][8][ceil(h/8)][ceil(w/8)] (device).  Asynchronous.
 * Errors: KF_EINVAL (no weights), KF_ENOMEM, KF_ECUDA. */
int kf_proposal_logits(kf_ctx *ctx, const float *pooled, int n, int h, int w, float *logits);

/* Loss and gradient on a batch: pooled[n][h][w] and labels (0/1 bytes)
 * [n][8][ceil(h/8)][ceil(w/8)] (device); *loss and grad[KF_NET_NPARAM]
 * (host, either may be NULL) receive the mean loss and its gradient with
 * respect to the bf16 weights.  Synchronises the context stream when an output
 * is requested.  Errors: KF_EINVAL, KF_ENOMEM, KF_ECUDA. */
int kf_proposal_grad(kf_ctx *ctx, const float *pooled, const uint8_t *labels, int n, int h, int w,
                     float pos_weight, float *grad, float *loss);

/* One Adam step of the masters on a batch (as kf_proposal_grad); *loss (host,
 * may be NULL: no synchronisation) receives the batch loss before the step.
 * Errors: KF_EINVAL, KF_ENOMEM, KF_ECUDA. */
int kf_proposal_train_step(kf_ctx *ctx, const float *pooled, const uint8_t *labels, int n, int h, int w,
                           float pos_weight, float lr, float *loss);

/* Training labels from the last kf_filter_bank call: for frame f, bytes
 * [S][ceil(H/64)][ceil(W/64)] (frames back to back, device, caller-owned),
 * 1 where a candidate with |R| > threshold has its centre in the tile.
 * Zeroes the array first.  threshold >= the bank threshold.
 * Errors: KF_EINVAL, KF_ERERUN (candidate list overflowed), KF_ECUDA. */
int kf_proposal_labels(kf_ctx *ctx, double threshold, uint8_t *labels);

/* Size of the static scratch that kf_responses_noalloc uses (MiB). */
#define KF_NOALLOC_SCRATCH_MB 32

/* kf_responses_noalloc: the response planes R of one frame through a
 * recursive bank, with no device allocation by the library.  The paper has
 * no counterpart to this entry point; it exists for callers that cannot call
 * cudaMalloc -- programs whose device memory is owned by a host framework's
 * pool allocator, and real-time loops that forbid allocation after start-up
 * because cudaMalloc can synchronise the device and can fail under memory
 * pressure.  The caller passes the frame and the output; every intermediate
 * lives in one static device array of KF_NOALLOC_SCRATCH_MB MiB that each GPU
 * which loads the library holds until the process exits.
 *   frame      one frame descriptor (device data) of any KF_DTYPE_* (f32,
 *              f16, bf16 or u16), each element times value_scale (0 = 1),
 *              as for kf_filter_bank; width <= 8192
 *   scales     host array of nscales blob radii lambda (px), 1..16
 *   type       KF_IIR_REPEATED_POLE (order 2..6) or KF_IIR_BUTTERWORTH
 *              (order 1..6); the FIR bank is not offered here
 *   responses  device output, nscales*H*W floats: R at (x, y) of scale s is
 *              responses[(s*H + y)*W + x] (same values as opts->responses of
 *              kf_filter_bank for this frame)
 *   cuda_stream cudaStream_t for all work (NULL = legacy default stream)
 * The frame's planes, edge rows and column carries must fit the scratch;
 * larger frames (roughly more than 4M pixel-scales) are rejected with
 * KF_EINVAL and a message naming the sizes (kf_last_error(NULL)).
 * Every call looks up the device address of the scratch on the current
 * device (cudaGetSymbolAddress; no allocation).  Every call shares the one
 * scratch array and finds the previous call's contents there: the library
 * clears what must start at zero, but calls that overlap on the GPU (e.g. on
 * two streams) race -- serialise them.  The call is synchronous: it waits on
 * the stream once after the designs (checked on the host) and once after the
 * filter kernels (to read their status), so it cannot be called while its
 * stream is being captured into a CUDA graph.
 * Errors: KF_EINVAL, KF_ECOND, KF_ENODEV, KF_ECUDA, KF_ETIMEOUT (a bounded
 * device wait gave up: the responses are incomplete). */
int kf_responses_noalloc(const kf_frame *frame, const double *scales, int nscales, int type,
                         int order, float *responses, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* KF_H */
