/*
 * fastttc.h - C ABI of the GB300 (sm_103a) FastConv and time-to-contact library.
 *
 * Paper: "Accelerated Convolutions for Efficient Multi-Scale Time to Contact
 * Computation in Julia" (Amini, Horn, Edelman).
 *
 * General conventions
 *  - Every entry point returns an ft_status (or a plain int where stated).  No C++
 *    exception and no abort ever crosses this boundary.
 *  - All arguments are validated on the host before anything is launched; an
 *    invalid call launches nothing and leaves every output untouched.
 *  - Pointers named "device" must point to memory of the current CUDA device; the
 *    caller owns every buffer passed in.  The library allocates device memory only
 *    in ttc_ctx_create (freed by ttc_ctx_destroy); no other call allocates.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Device work is enqueued asynchronously on it; no call synchronises
 *    the device.  Results are valid once the stream has reached the call.
 *  - A CUDA launch failure is reported as FT_ERR_CUDA (the CUDA error string is
 *    available from ft_last_cuda_error()).
 *  - Arrays are row-major (C order, last dimension fastest).
 */
#ifndef FASTTTC_H
#define FASTTTC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FT_OK = 0,
    FT_ERR_INVALID_ARG = 1,   /* null pointer, bad enum value, negative size */
    FT_ERR_SHAPE = 2,         /* dimensions inconsistent or too small for the request */
    FT_ERR_UNSUPPORTED = 3,   /* valid request beyond the library's limits */
    FT_ERR_WORKSPACE = 4,     /* request larger than the context was created for */
    FT_ERR_CUDA = 5,          /* a CUDA runtime call failed */
    FT_ERR_TIMEOUT = 6        /* a bounded wait inside a kernel gave up (see fastconv_check) */
} ft_status;

#define FT_MAX_NDIM 8         /* fastconv_nd: largest rank */
#define FT_MAX_LEVELS 7       /* ttc_*: largest number of pyramid levels */

/* Human-readable name of a status code (static string). */
const char *ft_status_string(int status);
/* Text of the last CUDA error seen by this library in the calling thread, or "". */
const char *ft_last_cuda_error(void);
/* Library version, major * 10000 + minor * 100 + patch. */
int ft_version(void);

/* ------------------------------------------------------------------------ */
/* FastConv: direct n-dimensional full convolution (Sec. IV-C, Eq. conv2)    */
/* ------------------------------------------------------------------------ */

/*
 * Output extent of the full convolution (Sec. IV: the operation FastConv replaces
 * is the full linear convolution): out_dims[d] = dims[d] + kdims[d] - 1.
 * Host only.  dims, kdims: nd host int64 values, each >= 1; out_dims: nd values
 * written on success.  Errors: FT_ERR_INVALID_ARG (null), FT_ERR_SHAPE (nd outside
 * [1, FT_MAX_NDIM] or an extent < 1).
 */
ft_status fastconv_out_dims(int nd, const int64_t *dims, const int64_t *kdims, int64_t *out_dims);

/*
 * Full n-D convolution, FP32 (Eq. conv2 read as the full linear convolution):
 *     out[p] = sum over r of kernel[r] * input[p - r],
 * over every kernel index r with p - r inside the input (zero outside).
 *   input  : device, prod(dims) floats, row-major contiguous.
 *   dims   : host, nd extents (each >= 1).
 *   kernel : device, prod(kdims) floats, row-major contiguous.
 *   kdims  : host, nd extents (each >= 1).  A kernel larger than the input is allowed.
 *   out    : device, prod(dims + kdims - 1) floats; every element is written.
 *   nd     : rank, 1 <= nd <= FT_MAX_NDIM.
 * Accumulation is FP32 in a fixed order.  input/kernel must not overlap out.
 * Some kernels receive their input tiles from the copy engine and wait for them with
 * a time limit; a wait that gives up leaves part of `out` unwritten and is reported by
 * the next fastconv_check.
 * Errors: FT_ERR_INVALID_ARG, FT_ERR_SHAPE, FT_ERR_UNSUPPORTED (output or kernel
 * with more than 2^62 elements), FT_ERR_CUDA.
 */
ft_status fastconv_nd(const float *input, const int64_t *dims, int nd,
                      const float *kernel, const int64_t *kdims, float *out, void *stream);

/*
 * fastconv_nd for inputs of other element types (Sec. IV-C: FastConv covers many signal
 * types): in_dtype FT_U8, FT_I16, FT_F16, FT_BF16 (or FT_F32, which is fastconv_nd).
 * The kernel and the output stay FP32; every input value is widened to FP32 exactly.
 * Planes of more than one row with kernels of at most 17 columns whose input rows are
 * 16-byte aligned whole 16-byte units are staged in the input's own type by the copy
 * engine and widened in the kernel; any other request converts the input into
 * `scratch` (device, prod(dims) floats) first and runs the FP32 path.
 * Errors: as fastconv_nd; FT_ERR_INVALID_ARG (bad in_dtype), FT_ERR_WORKSPACE (scratch
 * needed but NULL).
 */
ft_status fastconv_nd_typed(const void *input, int in_dtype, const int64_t *dims, int nd, const float *kernel,
                            const int64_t *kdims, float *out, float *scratch, void *stream);

/*
 * Full convolution by FFT, for large kernels (Sec. IV-C, IV-D: above a kernel size
 * threshold the FFT method is faster, and FastConv switches to it).  Ranks 1-3.  Both
 * operands are zero-padded to FFT extents F_d >= N_d + K_d - 1 (products of 2, 3, 5, 7),
 * transformed real-to-complex (cuFFT), multiplied pointwise, transformed back and
 * cropped to out.
 * Error: normwise, about FP32 rounding times log2(prod F) times ||input||_2 ||kernel||_2
 * per element, unlike the per-element bound of the direct path.
 *
 * fastconv_fft_plan_create: the transforms for input dims and kernel kdims (host
 *   arrays, as fastconv_nd) on the current device.  This is the call that allocates
 *   (cuFFT's plan data): make it once per shape, before any timed loop or stream
 *   capture.  *workspace_bytes (nullable) receives the bytes a call needs: the padded
 *   operands, their spectra and cuFFT's work area.  The plan is owned by the caller
 *   until fastconv_fft_plan_destroy.  Errors: FT_ERR_INVALID_ARG, FT_ERR_SHAPE,
 *   FT_ERR_UNSUPPORTED (rank > 3, more than 2^30 output values), FT_ERR_CUDA.
 * fastconv_fft: one convolution with a plan; allocates nothing and does not
 *   synchronise.  workspace: device, 256-byte aligned, at least
 *   fastconv_fft_plan_workspace(plan) bytes, owned by this call until the stream has
 *   passed it (calls on different streams need different workspaces; one plan serves
 *   them all, the binding of a stream and work area to it is serialised per plan).
 *   The current device must be the plan's.  Errors: FT_ERR_INVALID_ARG,
 *   FT_ERR_WORKSPACE, FT_ERR_CUDA (also for cuFFT errors).
 */
typedef struct fastconv_fft_plan fastconv_fft_plan;
ft_status fastconv_fft_plan_create(const int64_t *dims, int nd, const int64_t *kdims, fastconv_fft_plan **plan,
                                   size_t *workspace_bytes);
void fastconv_fft_plan_destroy(fastconv_fft_plan *plan);
size_t fastconv_fft_plan_workspace(const fastconv_fft_plan *plan);
ft_status fastconv_fft(fastconv_fft_plan *plan, const float *input, const float *kernel, float *out,
                       void *workspace, size_t workspace_bytes, void *stream);

/*
 * Host only: 1 when the FFT path is expected to be faster than the direct path for
 * this request, 0 otherwise: 2-D requests whose kernel has at least FT_FFT_MIN_TAPS
 * taps and whose output has at least FT_FFT_MIN_OUTPUT values.  The crossover was
 * measured on GB300 for 1080 x 1920 images only; 3-D kernels and small images keep the
 * direct path (and its per-element error bound).
 */
#define FT_FFT_MIN_TAPS 961          /* 31 x 31: direct 86 us at 25 x 25 and 117 us at 31 x 31, FFT 109 us */
#define FT_FFT_MIN_OUTPUT 1000000    /* output values: about a 1080 x 1920 image */
int fastconv_prefers_fft(const int64_t *dims, int nd, const int64_t *kdims);

/*
 * Full n-D convolution with a separable kernel k = f_0 (x) f_1 (x) ... (x) f_{nd-1}
 * (outer product of one vector per axis; the paper's Future Work: directional
 * derivatives, Gaussians and block averages are separable): one 1-D full convolution
 * per axis, in axis order, so an output costs sum(kdims) multiply-adds instead of
 * prod(kdims).  Same result as fastconv_nd with the outer-product kernel, up to the
 * order of the FP32 sums.
 *   factors: host array of nd device pointers; factors[d] holds kdims[d] floats.
 *   scratch: device, prod(dims + kdims - 1) floats (may be NULL when nd == 1); the
 *            passes alternate between scratch and out so that the last one writes out.
 *   input, out, scratch must not overlap.  Other arguments as fastconv_nd.
 * Errors: as fastconv_nd; FT_ERR_INVALID_ARG (a null factor, missing scratch, aliased
 * buffers).
 */
ft_status fastconv_separable(const float *input, const int64_t *dims, int nd, const float *const *factors,
                             const int64_t *kdims, float *out, float *scratch, void *stream);

/*
 * Host only: tests whether a kernel (host, prod(kdims) floats, row-major) is the outer
 * product of one vector per axis, within rel_tol * max|k| at every entry.  On success
 * writes the factors to `factors` (host, sum(kdims) floats: factor 0, then factor 1,
 * ...) and returns 1; returns 0 when the kernel is not separable, -1 on invalid
 * arguments (null pointers, nd outside [1, FT_MAX_NDIM], an extent < 1, more than 2^26
 * entries, rel_tol < 0).  The factors are the kernel's fibres through its largest
 * entry, the first one scaled so that their product reproduces the kernel.
 */
int fastconv_factor(const float *kernel, const int64_t *kdims, int nd, double rel_tol, float *factors);

/*
 * Synchronises `stream`, then reports (and clears) the device-wide FastConv status
 * word of the current device: FT_ERR_TIMEOUT if a bounded wait of a FastConv kernel
 * gave up since the last check (its output is incomplete), FT_OK otherwise.  No
 * counterpart in the paper.  Errors: FT_ERR_CUDA.
 */
ft_status fastconv_check(void *stream);

/*
 * Test switch for the timeout paths (no counterpart in the paper).  While on (nonzero),
 * kernels that wait for copy-engine transfers and are launched afterwards expect 16
 * more bytes than their copies deliver: every copy still lands, but each bounded wait
 * gives up after about 2 s of GPU clock, the kernel reports it (FT_FLAG_TIMEOUT in the
 * TTC records, FT_ERR_TIMEOUT from fastconv_check) and returns; results of those calls
 * are incomplete.  Off (0) restores normal operation.  Process-wide; not for production.
 */
void ft_test_stall_tma_waits(int on);

/* ------------------------------------------------------------------------ */
/* Time to contact (Sec. V-A, V-B)                                           */
/* ------------------------------------------------------------------------ */

/* element types: frames (FT_U8, FT_F32) and FastConv inputs (all five) */
typedef enum { FT_U8 = 0, FT_F32 = 1, FT_I16 = 2, FT_F16 = 3, FT_BF16 = 4 } ft_dtype;
typedef enum { FT_MODE_TTC = 0, FT_MODE_FOE = 1 } ft_mode;

/* Per-result flags (information, not errors). */
#define FT_FLAG_SINGULAR 1   /* normal equations singular: A, B, C, TTC, FOE are NaN */
#define FT_FLAG_C_ZERO 2     /* C == 0: TTC = +inf, FOE = NaN */
#define FT_FLAG_RECEDING 4   /* C < 0: the camera moves away; TTC is negative */
#define FT_FLAG_TIMEOUT 8    /* a bounded wait inside the kernels expired: this call's sums are incomplete */
#define FT_FLAG_BOUNDS 16    /* only in builds with FASTTTC_CHECK=1 (FT_CHECK): a kernel of this call found a
                                read outside its frame or a write outside its image; the access was skipped */

/*
 * One solve result for one frame pair at one pyramid level (152 bytes).
 *  sums : the ten least-squares sums of Sec. V-A over all 2x2x2 cubes of the
 *         level, in the units of the level-l image (block means of the input
 *         brightness) and level-l pixels, in this order:
 *         0 Ex^2, 1 Ex Ey, 2 Ey^2, 3 G Ex, 4 G Ey, 5 G^2, 6 Ex Et, 7 Ey Et, 8 G Et, 9 Et^2.
 *  A, B, C : solution of the normal equations (mode FT_MODE_TTC: A = B = 0).
 *  ttc  : 1/C in frame intervals (Eq. final_TTC).
 *  x0, y0 : focus of expansion -A/C, -B/C, converted to level-0 pixels, measured
 *         from the image centre ((W-1)/2, (H-1)/2), x right, y down.
 *  resid : sum over cubes of (A Ex + B Ey + C G + Et)^2 divided by sum Et^2.
 *  n    : number of cubes summed, (H_l - 1) (W_l - 1).
 */
typedef struct {
    double sums[10];
    double A, B, C;
    double ttc, x0, y0;
    double resid;
    int64_t n;
    int32_t level;
    int32_t flags;
} ttc_level_result;

/*
 * The 2x2x2 derivative estimates of Sec. II / V-A at level 0, materialised.
 * For the cube with corner (i, j) (rows i, i+1; columns j, j+1; frames prev, cur):
 *   Ex = mean of the four x first differences, Ey = mean of the four y first
 *   differences, Et = mean of the four t first differences (cur - prev),
 *   G  = x Ex + y Ey with x = j + 1/2 - (W-1)/2, y = i + 1/2 - (H-1)/2.
 *   prev, cur : device, H rows of W pixels of `dtype`, row stride pitch_bytes.
 *   Ex, Ey, Et : device, (H-1) x (W-1) floats each, contiguous.
 *   G : device, (H-1) x (W-1) floats, or NULL to skip it.
 * For FT_U8 frames Ex, Ey and Et are exact (integer sums / 4).
 * Errors: FT_ERR_INVALID_ARG, FT_ERR_SHAPE (H or W < 2, pitch_bytes < W * pixel
 * size or not a multiple of the pixel size), FT_ERR_CUDA.
 */
ft_status ttc_derivatives(const void *prev, const void *cur, int dtype, int H, int W,
                          int64_t pitch_bytes, float *Ex, float *Ey, float *Et, float *G,
                          void *stream);

/*
 * A context owns the device workspace for the per-tile partial sums (allocated
 * here, once) for requests up to max_H x max_W frames, max_levels levels and
 * max_pairs frame pairs per call.  One context must not be used by two host
 * threads at once; different contexts are independent.
 * Errors: FT_ERR_INVALID_ARG, FT_ERR_SHAPE, FT_ERR_CUDA (allocation failed).
 */
typedef struct ttc_ctx ttc_ctx;
ft_status ttc_ctx_create(ttc_ctx **ctx, int max_H, int max_W, int max_levels, int max_pairs);
void ttc_ctx_destroy(ttc_ctx *ctx);
/* Bytes of device workspace the context holds. */
size_t ttc_ctx_workspace_bytes(const ttc_ctx *ctx);

/*
 * Multi-scale TTC/FOE for one frame pair (Sec. V-A, V-B): for each level
 * l = 0 .. levels-1, the level-l images are the l-fold 2x2 block means of prev and
 * cur (floor cropping: H_l = floor(H / 2^l)); the ten sums are taken over all
 * (H_l - 1)(W_l - 1) cubes of level l with x, y measured from the level-0 image
 * centre expressed in level-l pixels, (W - 2^l) / 2^(l+1) and (H - 2^l) / 2^(l+1);
 * then the 3x3 normal equations (mode FT_MODE_FOE) or the TTC-only equation
 * (FT_MODE_TTC: C = -sum(G Et) / sum(G^2)) are solved in FP64.
 *   prev, cur : device frames, H x W pixels of `dtype`, row stride pitch_bytes.
 *   out : device, `levels` results, out[l] for level l.
 * Per-cube products are formed in FP32 and summed pairwise in FP32 within each
 * tile; tiles are merged in FP64 in a fixed order (results are deterministic).
 * uint8 frames of 2..5 levels with 16-byte aligned frames and pitch take the
 * all-levels kernel (one launch for every level, then the merge/solve); other
 * requests take one pass per level.
 * Errors: FT_ERR_INVALID_ARG, FT_ERR_SHAPE (a level smaller than 2 x 2, pitch),
 * FT_ERR_UNSUPPORTED (levels > FT_MAX_LEVELS), FT_ERR_WORKSPACE (request larger
 * than the context), FT_ERR_CUDA.
 */
ft_status ttc_solve(ttc_ctx *ctx, const void *prev, const void *cur, int dtype, int H, int W,
                    int64_t pitch_bytes, int levels, int mode, ttc_level_result *out,
                    void *stream);

/*
 * ttc_solve for one frame pair without allocating any device memory.  The paper has
 * no counterpart: this entry point exists for callers that cannot call cudaMalloc
 * after start-up -- hard real-time control loops (an allocation can block for an
 * unbounded time), safety-certified vehicle software that forbids dynamic allocation,
 * and plug-ins whose host process owns all device memory through its own allocator.
 * The caller still passes and owns prev, cur and out (same meaning, layout and
 * results as ttc_solve, in place of a context).
 *
 * Scratch: a fixed array of FT_NOALLOC_SCRATCH_BYTES in the library's device memory,
 * held by every GPU that loads the library until the process exits.  It covers any
 * single pair up to 1920 x 1080 with up to FT_MAX_LEVELS levels in either dtype;
 * larger requests are rejected with FT_ERR_WORKSPACE before anything is launched.
 * The first call on a device looks up the array's device address for that device
 * (with that device current), and a call looks it up again when the device's current
 * context has changed since; make the first call before any stream capture.
 * Every call uses the same array and leaves the last call's contents in it: nothing
 * there needs to start at zero (each call writes every value it reads), but calls
 * whose work overlaps on the GPU (other streams, other host threads) race on it, so
 * serialise them.  Errors: as ttc_solve, plus FT_ERR_WORKSPACE for oversized requests.
 */
#define FT_NOALLOC_SCRATCH_BYTES (8u * 1024u * 1024u)
ft_status ttc_solve_noalloc(const void *prev, const void *cur, int dtype, int H, int W, int64_t pitch_bytes,
                            int levels, int mode, ttc_level_result *out, void *stream);

/*
 * Gradient magnitude and direction of one image (Sec. II, Eq. Emag and Eq. Eangle): at
 * every 2x2 block centre, Ex = 1/2 [(E(x+1,y) - E(x,y)) + (E(x+1,y+1) - E(x,y+1))] and
 * Ey likewise down the rows (the Sec. II mask and its transpose; x: column, y: row),
 *     mag = sqrt(Ex^2 + Ey^2),  dir = atan2(Ey, Ex) in [-pi, pi]  (FP32).
 *   image : device, H rows of W pixels (FT_U8 or FT_F32), row stride pitch_bytes.
 *   mag, dir : device, (H-1) x (W-1) floats each, row-major contiguous; either may be
 *              NULL (not both).
 * Errors: FT_ERR_INVALID_ARG (null image, both outputs null, bad dtype), FT_ERR_SHAPE
 * (H or W < 2, pitch), FT_ERR_UNSUPPORTED (more than 524280 rows), FT_ERR_CUDA.
 */
ft_status ttc_gradient(const void *image, int dtype, int H, int W, int64_t pitch_bytes, float *mag, float *dir,
                       void *stream);

/*
 * ttc_gradient for n images of one size in one launch (a batch of frames):
 *   images : device, image i at images + i * image_stride_bytes (each H rows of W pixels,
 *            row stride pitch_bytes);
 *   mag, dir : device, n x (H-1) x (W-1) floats each (image i's outputs at
 *              i * (H-1) * (W-1)), either may be NULL (not both).
 * Errors: those of ttc_gradient, and FT_ERR_SHAPE for n < 1 or an image stride smaller
 * than H rows (image_stride_bytes < (H-1) * pitch_bytes + W * pixel size, for n > 1),
 * FT_ERR_UNSUPPORTED for n > 65535.
 */
ft_status ttc_gradient_batch(const void *images, int n, int64_t image_stride_bytes, int dtype, int H, int W,
                             int64_t pitch_bytes, float *mag, float *dir, void *stream);

/*
 * The same for the T-1 consecutive pairs (t, t+1) of a video of T frames stored
 * frame_stride_bytes apart: out[(t * levels) + l] for pair t, level l (device,
 * (T-1) * levels results).  Sec. V-B: the estimate is produced at every frame.
 * A video whose pairs give more than 64 level-0 tiles of 64 x 256 cubes per CTA of
 * the grid (two per SM) takes one pass per level, each frame's pyramid built once;
 * shorter ones take the all-levels kernel under the conditions of ttc_solve (results
 * of the two agree within rounding; the choice depends only on the request).
 */
ft_status ttc_solve_sequence(ttc_ctx *ctx, const void *frames, int64_t frame_stride_bytes, int T,
                             int dtype, int H, int W, int64_t pitch_bytes, int levels, int mode,
                             ttc_level_result *out, void *stream);

/*
 * ttc_solve_sequence for a video in host memory, results to host memory (no
 * counterpart in the paper: the end-to-end path of a camera pipeline).  The pairs are
 * processed in chunks of FT_SEQ_CHUNK_PAIRS (fewer if the context was created for fewer
 * pairs): the chunks' frames (one frame shared by consecutive chunks is copied twice) go
 * to two device buffers of the context on two copy streams of the context, each chunk
 * is computed on `stream` as soon as its copy has landed, so uploads overlap compute.
 * Tile plans are those of the whole sequence, and for float frames a chunk after the
 * first also computes (without reporting) the levels - 1 pairs before it, so that its
 * frames' pyramids are rounded as in the whole sequence: the records are bitwise those
 * of ttc_solve_sequence on the same frames (device copies with the same strides),
 * except for float frames on a context created for at most levels - 1 pairs.
 *   frames: host, T frames frame_stride_bytes apart (page-locked memory lets the copies
 *           run asynchronously; pageable memory works but each copy then blocks);
 *           must stay valid and unchanged until `stream` reaches the end of the call.
 *   out:    host, (T-1) * levels records (page-locked for an asynchronous copy), valid
 *           once `stream` has reached the end of the call.
 * The call allocates nothing: the two device buffers and the records buffer are sized
 * beforehand by ttc_ctx_reserve_host for at least this request (same frame stride, T,
 * dtype, H, W, pitch and levels, or smaller), the copy streams and their events are
 * made by ttc_ctx_create.  Successive calls on one context may use different streams:
 * a call's uploads wait until the previous call has finished with the buffers.
 * Errors: as ttc_solve_sequence, FT_ERR_SHAPE (frame stride shorter than a frame),
 * FT_ERR_WORKSPACE (buffers not reserved for this request), FT_ERR_CUDA.
 *
 * ttc_ctx_reserve_host: sizes the context's host-sequence buffers for requests up to
 * the given one (the same arguments as ttc_solve_sequence_host); allocates only when
 * they must grow, and then first waits (on the host) for this context's last
 * host-sequence call to finish with them -- no device-wide synchronisation, so other
 * streams and contexts keep running.  Freed by ttc_ctx_destroy.  Errors: FT_ERR_INVALID_ARG,
 * FT_ERR_SHAPE, FT_ERR_WORKSPACE (larger than the context), FT_ERR_CUDA.
 */
#define FT_SEQ_CHUNK_PAIRS 64
ft_status ttc_ctx_reserve_host(ttc_ctx *ctx, int64_t frame_stride_bytes, int T, int dtype, int H, int W,
                               int64_t pitch_bytes, int levels);
ft_status ttc_solve_sequence_host(ttc_ctx *ctx, const void *frames, int64_t frame_stride_bytes, int T,
                                  int dtype, int H, int W, int64_t pitch_bytes, int levels, int mode,
                                  ttc_level_result *out, void *stream);

/*
 * The two stages of ttc_solve_sequence, for callers that time or overlap them.
 * ttc_partial_sums runs the fused pyramid + stencil + G + product + tile-reduction
 * kernel and leaves FP32 per-tile partial sums in the context; ttc_reduce_solve
 * merges them in FP64 and solves.  ttc_reduce_solve uses the geometry of the last
 * ttc_partial_sums call on the same context and must follow it on the same stream.
 */
ft_status ttc_partial_sums(ttc_ctx *ctx, const void *frames, int64_t frame_stride_bytes, int T,
                           int dtype, int H, int W, int64_t pitch_bytes, int levels, void *stream);
ft_status ttc_reduce_solve(ttc_ctx *ctx, int mode, ttc_level_result *out, void *stream);

/*
 * Batches of independent frame pairs of different sizes (no counterpart in the paper:
 * many cameras at once).  ttc_batch_prepare takes the pairs (host array of
 * descriptors; the frames are device memory owned by the caller and must stay valid
 * and unchanged in address until the last ttc_batch_run that uses them), checks them,
 * lays out the context workspace, and uploads a work list and per-pair descriptors on
 * `stream` (one small kernel that reads them from the context's page-locked staging
 * memory, which has two halves: a prepare waits on the host only for the upload of the
 * prepare before the previous one).  ttc_batch_run then performs, for every pair and level, the same
 * computation as ttc_solve (same results up to rounding; identical for a pair alone
 * or in any batch with the same tile plan).  uint8 pairs of 2..5 levels whose frames
 * and pitch are 16-byte aligned take one launch of the all-levels kernel (every level
 * of every such pair, work list of strips of level-0 tiles; the tile plan does not
 * apply to them, and their results equal those of ttc_solve bitwise); other pairs
 * take two launches per level; one merge/solve launch follows.  It only launches
 * kernels (after zeroing the context's status word), so a caller may capture it in a
 * CUDA graph and replay it.
 * out: device, npairs * levels results, out[p * levels + l].
 * ttc_batch_autotune times, on the prepared batch, 64-row and 16-row tiles for every
 * level, keeps the faster per level for later prepares on this context, prepares
 * again with it, and writes the chosen rows per tile to rows_per_tile (host, levels
 * ints, nullable).  It synchronises `stream`.
 * Errors: FT_ERR_INVALID_ARG (null, bad dtype/mode, no prepared batch), FT_ERR_SHAPE
 * (a pair too small for `levels`, pitch), FT_ERR_WORKSPACE (more pairs, levels, or
 * larger frames than the context was created for), FT_ERR_CUDA.
 */
typedef struct {
    const void *prev;        /* device, H rows of W pixels, row stride pitch_bytes */
    const void *cur;         /* device, same geometry as prev */
    int H, W;
    int64_t pitch_bytes;
    /* Per-frame pyramids owned by the caller (both nullable; see ttc_pyramid_layout).
     * prev_pyramid: levels 1 .. levels-1 of `prev`, as an earlier ttc_batch_run wrote
     * them into a cur_pyramid of the same H, W, dtype and levels; read only (pairs of
     * the all-levels kernel form every level from the frames and do not read it).
     * cur_pyramid: receives levels 1 .. levels-1 of `cur`.  A null pointer puts that
     * frame's pyramid in the context workspace instead (or nowhere, for pairs of the
     * all-levels kernel).  The two must differ, and no block may be one pair's
     * cur_pyramid and another pair's prev_pyramid in the same batch (the results of
     * such a batch are unspecified).  16-byte aligned. */
    const void *prev_pyramid;
    void *cur_pyramid;
} ttc_pair_desc;
ft_status ttc_batch_prepare(ttc_ctx *ctx, const ttc_pair_desc *pairs, int npairs, int dtype, int levels,
                            void *stream);
ft_status ttc_batch_run(ttc_ctx *ctx, int mode, ttc_level_result *out, void *stream);
ft_status ttc_batch_autotune(ttc_ctx *ctx, int mode, ttc_level_result *out, int reps, int *rows_per_tile,
                             void *stream);

/*
 * Layout of one frame's pyramid block (levels 1 .. levels-1 of the 2x2 block-sum
 * pyramid of Sec. V-B, no counterpart as a buffer in the paper): level l is an image of
 * floor(H/2^l) rows of floor(W/2^l) pixels, uint16 exact sums of 4^l pixels for uint8
 * frames up to level 4 and float beyond (float means for float frames), starting at
 * byte offsets[l] of the block with row stride pitches[l].  offsets and pitches: host,
 * levels entries each (entry 0 is set to 0), nullable; *bytes: the block size (0 when
 * levels == 1).  A serving loop keeps two blocks per stream and swaps them each frame,
 * so that each frame's pyramid is built once.
 * Errors: FT_ERR_INVALID_ARG (null bytes, bad dtype), FT_ERR_SHAPE (frame too small
 * for `levels`), FT_ERR_UNSUPPORTED (levels > FT_MAX_LEVELS).
 */
ft_status ttc_pyramid_layout(int H, int W, int levels, int dtype, int64_t *offsets, int64_t *pitches,
                             int64_t *bytes);

/*
 * Fixes the tile height of every level for later ttc_batch_prepare calls on this
 * context (no counterpart in the paper).  rows_per_tile: host, levels entries, each 16
 * or 64; null clears the plan (automatic choice per batch).  With a fixed plan, the
 * results of a pair do not depend on the other pairs of its batch.
 * Errors: FT_ERR_INVALID_ARG (null context, bad entry, levels < 1),
 * FT_ERR_UNSUPPORTED (levels > FT_MAX_LEVELS).
 */
ft_status ttc_batch_set_plan(ttc_ctx *ctx, const int *rows_per_tile, int levels);

/*
 * Serving runtime (no counterpart in the paper, which processes one camera): many
 * camera streams with continuous batching over ttc_batch_prepare / ttc_batch_run.
 * Each admitted stream owns three device frame slots and two pyramid blocks (its last
 * two frames' levels 1..L-1; see ttc_pyramid_layout), so each frame is uploaded once
 * and its pyramid built once.  ttc_server_step launches a tick when fewer than two are
 * in flight: at most one waiting frame per stream (oldest arrival first, at most
 * max_batch pairs), uploaded from the caller's host memory (frames under 1 MB in
 * page-locked memory whose rows and pitch are whole 16-byte words by one gather kernel
 * on the server's gather stream that reads that memory directly; the others by one
 * copy each on the server's copy stream), then one batch on the server's compute stream with the
 * records copied to page-locked host memory; it also reports every frame whose fate is
 * settled.  The multi-scale rule (Sec. V-B) picks each result's level on the host.
 *   ttc_server_create: dtype FT_U8 or FT_F32 frames; levels, mode, rule as elsewhere;
 *     max_batch pairs per tick; max_streams open streams; max_pending waiting frames per
 *     stream (a new frame beyond that drops the oldest); hbm_budget_bytes bounds the
 *     server's device memory (context, result buffers and every stream's buffers);
 *     rows_per_tile: host, levels entries (16 or 64), nullable (64 everywhere): the
 *     fixed tile plan, so a stream's records do not depend on the other streams.
 *   ttc_server_admit: a stream of H x W frames; FT_ERR_WORKSPACE when the budget, the
 *     stream count or the server's maximum frame size would be exceeded.
 *   ttc_server_submit: a frame (host, H rows of W pixels, row stride pitch_bytes; page-
 *     locked memory for asynchronous uploads) that must stay valid and unchanged until
 *     its report; seq and t_arrival are returned in the report unchanged.
 *   ttc_server_remove: the stream goes away; its waiting frames are reported dropped, its
 *     frames in flight discarded, its buffers freed once no tick in flight uses them.  A
 *     stream's first frame (after admission) has no result.
 *   ttc_server_step: wait != 0 blocks until at least one report is ready when a tick is
 *     in flight; writes up to max_done reports (host) and their count.
 * Errors: FT_ERR_INVALID_ARG (null, bad id or enum), FT_ERR_SHAPE (pitch), FT_ERR_WORKSPACE,
 * FT_ERR_CUDA.  A server is driven from one host thread.
 */
typedef enum {
    FT_SERVED_RESULT = 1,       /* records[0..levels-1] and level are valid */
    FT_SERVED_FIRST_FRAME = 0,  /* the stream's first frame: it only became the resident frame */
    FT_SERVED_DROPPED = -1,     /* never processed (queue overflow or stream removed) */
    FT_SERVED_DISCARDED = -2    /* processed, but its stream was removed meanwhile */
} ft_served_status;
typedef struct {
    ttc_level_result records[FT_MAX_LEVELS];
    double t_arrival;
    int64_t seq;
    int stream;
    int status;                 /* ft_served_status */
    int level;                  /* chosen level, -1 when none */
    int pad;
} ttc_served;
typedef struct ttc_server ttc_server;
ft_status ttc_server_create(ttc_server **srv, int max_H, int max_W, int levels, int mode, int rule, int dtype,
                            int max_batch, int max_streams, int max_pending, int64_t hbm_budget_bytes,
                            const int *rows_per_tile);
void ttc_server_destroy(ttc_server *srv);
ft_status ttc_server_stream_bytes(const ttc_server *srv, int H, int W, int64_t *bytes);
ft_status ttc_server_admit(ttc_server *srv, int H, int W, int *stream_id);
ft_status ttc_server_remove(ttc_server *srv, int stream_id);
ft_status ttc_server_submit(ttc_server *srv, int stream_id, const void *frame, int64_t pitch_bytes, int64_t seq,
                            double t_arrival);
ft_status ttc_server_step(ttc_server *srv, int wait, ttc_served *done, int max_done, int *n_done);

/*
 * Load generator for measuring the serving runtime (no counterpart in the paper): keeps
 * each of the nstreams admitted streams `ids` supplied with a waiting frame, taken in turn
 * from its nframes host frames (frames[i * nframes + k], row pitch pitches[i]; page-locked
 * memory lets the uploads run asynchronously), and steps the server until `pairs` results
 * (FT_SERVED_RESULT) have come back, keeping two ticks in flight (the next tick's uploads
 * overlap the kernels of the one being waited for).  Every tick then carries one pair per
 * stream, so the rate is set by the runtime and the device rather than by the caller.  The
 * ticks still in flight at the end complete before the call returns (their pairs count,
 * so *served may exceed `pairs`) and the server is idle again.  Reports are consumed;
 * *seconds (wall clock), *served, *p50_ms and *p99_ms (submission to report) are written
 * when non-null.  Errors: FT_ERR_INVALID_ARG, and those of submit and step.
 */
ft_status ttc_server_drive(ttc_server *srv, const int *ids, int nstreams, const void *const *frames,
                           const int64_t *pitches, int nframes, int64_t pairs, double *seconds, int64_t *served,
                           double *p50_ms, double *p99_ms);
int ttc_server_in_flight(const ttc_server *srv);        /* ticks in flight */
int64_t ttc_server_ticks(const ttc_server *srv);        /* ticks launched so far */
int ttc_server_waiting(const ttc_server *srv, int stream_id);   /* the stream's waiting frames; all waiting
                                                                   frames and unreturned reports if < 0 */
int64_t ttc_server_bytes_in_use(const ttc_server *srv);
int ttc_server_launches(const ttc_server *srv);         /* kernels of the last batch run */

/*
 * Timing hook (no counterpart in the paper): when start and end are non-null
 * (cudaEvent_t values passed as void*), every later ttc_partial_sums /
 * ttc_solve_sequence / ttc_solve on this context records `start` on its stream just
 * before the launches of the level-0 pass and `end` just after them, so that a
 * caller can time the dominant pass alone.  NULL, NULL turns it off.
 * Errors: FT_ERR_INVALID_ARG (null context, or exactly one event null).
 */
ft_status ttc_ctx_set_level0_events(ttc_ctx *ctx, void *start, void *end);
/* Number of kernels the last ttc_partial_sums on this context launched (0 before any). */
int ttc_ctx_last_launch_count(const ttc_ctx *ctx);

/*
 * Multi-scale selection (Sec. V-B), host only: start at the finest usable level
 * and move one level coarser while the next level is usable and its key is
 * smaller ("improved (ie. reduced)"); rule 0: key = TTC; rule 1: key = resid.
 * A level is usable when flags has neither FT_FLAG_SINGULAR nor FT_FLAG_C_ZERO
 * and TTC > 0.  host_results: `levels` results of one pair, level order.
 * Returns the chosen level, -1 if no level is usable, -2 on invalid arguments.
 */
int ttc_select_level(const ttc_level_result *host_results, int levels, int rule);

#ifdef __cplusplus
}
#endif

#endif /* FASTTTC_H */
