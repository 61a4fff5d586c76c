/* dwt2.h -- C ABI of the GB300 (sm_103a) 2-D discrete wavelet transform library (libdwt2.so).
 *
 * The library computes the 2-D DWT with the non-separable lifting scheme of Barina et al.,
 * "The Parallel Algorithm for the 2-D Discrete Wavelet Transform" (Sec. 3, Eq. 5): per lifting
 * pair one spatial predict step and one spatial update step, which act on the polyphase quad
 * [LL, HL, LH, HH] of Sec. 2.  Every decomposition level is one kernel that reads its input
 * plane once from HBM and writes the four subbands once.
 *
 * Conventions
 *   - Images are row-major: H rows x W columns, a row pitch in bytes.  "Horizontal" (the paper's
 *     m / z_m axis, filters P and U) runs along a row, "vertical" (n / z_n, P* and U*) along a
 *     column.
 *   - Polyphase quad at (n, m): LL = x[2n][2m], HL = x[2n][2m+1], LH = x[2n+1][2m],
 *     HH = x[2n+1][2m+1] (Sec. 2, the vector order of Eq. 3 and Eq. 5).
 *   - Level j maps the h x w plane LL_{j-1} (LL_0 = the image) to LL_j ceil(h/2) x ceil(w/2),
 *     HL_j ceil(h/2) x floor(w/2), LH_j floor(h/2) x ceil(w/2), HH_j floor(h/2) x floor(w/2)
 *     (the Mallat recursion on LL cited in Sec. 2).
 *   - Boundaries: whole-sample symmetric extension, x[-k] = x[k], x[N-1+k] = x[N-1-k]
 *     (repeated for signals shorter than the filter); an axis of length 1 passes through.
 *   - Wavelets (the paper evaluates CDF 5/3, Sec. 4, and states the scheme holds for any
 *     wavelet, Sec. 5; it prints no coefficients):
 *       DWT2_CDF53_INT  reversible integer CDF 5/3: d = x_o - floor((x_e + x_e') / 2),
 *                       s = x_e + floor((d' + d + 2) / 4); the fused steps keep the floors of
 *                       the step order of Eq. 3 (P, P*, U, U*), so results are bit-exact with
 *                       that order.  Exact while every intermediate fits in int32: inputs with
 *                       |x| <= 2^24 are safe for every level count.
 *       DWT2_CDF53_F32  CDF 5/3 in fp32: P(z) = -1/2 (1 + z), U(z) = 1/4 (1 + z^-1), no scaling.
 *       DWT2_CDF97_F32  CDF 9/7 in fp32, two lifting pairs (alpha, beta, gamma, delta) of the
 *                       Daubechies-Sweldens factorisation, then low-pass * 1/K and high-pass
 *                       * K/2 per axis (low-pass DC gain 1, high-pass Nyquist gain 1), i.e.
 *                       LL / K^2, HL / 2, LH / 2, HH * K^2 / 4.
 *       DWT2_DD97_F32   Deslauriers-Dubuc 9/7 in fp32 (the interpolating wavelet with a
 *                       four-tap predict): d[m] = x_o - (9/16 (s[m] + s[m+1]) - 1/16 (s[m-1] +
 *                       s[m+2])), the cubic interpolation of the odd sample, then
 *                       s[m] += 1/4 (d[m-1] + d[m]); no scaling.
 *       DWT2_DD137_F32  Deslauriers-Dubuc 13/7 in fp32: the same predict, then
 *                       s[m] += 9/32 (d[m-1] + d[m]) - 1/32 (d[m-2] + d[m+1]); no scaling.
 *     The Deslauriers-Dubuc wavelets run the non-separable scheme of Eq. 5 (their spatial steps
 *     with these P, U) in dwt2_forward, dwt2_inverse, the uniform batch entry points and
 *     dwt2_forward_static and the batched plans (forward and inverse directions), and the
 *     two-pass separable comparator (DWT2_SCHEME_SEP_TWOPASS, fp32); the other comparators and
 *     the adjoints return DWT2_EUNSUPPORTED for them.
 *   - All arithmetic of the float wavelets is fp32.  DWT2_BF16 / DWT2_F16 are storage types
 *     only: values are widened on load and rounded to nearest-even on store.  With 16-bit
 *     band storage the intermediate LL planes (workspace) and the final LL_J stay fp32.
 *
 * Memory and streams
 *   - Every pointer argument named img, coeffs, g_img, g_coeffs or workspace is a DEVICE pointer,
 *     owned by the caller; the library never allocates device memory on these paths.
 *   - stream is a cudaStream_t handle passed as void* (NULL = the legacy default stream).
 *     Every transform call is asynchronous on that stream; the buffers must stay alive until
 *     the stream has executed it.
 *   - Errors: functions return dwt2_status.  Invalid arguments are rejected before any launch
 *     (DWT2_EINVAL / DWT2_EUNSUPPORTED); a failed launch returns DWT2_ECUDA, with the CUDA error
 *     text available from dwt2_last_error().  Nothing in the library aborts, traps or throws.
 *   - Device-side waits (pipeline barriers inside a kernel) are bounded in time.  A wait that
 *     gives up records DWT2_ETIMEOUT in the workspace status word; dwt2_check_status() reads it.
 */
#ifndef DWT2_H
#define DWT2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DWT2_CDF53_INT = 0,
    DWT2_CDF53_F32 = 1,
    DWT2_CDF97_F32 = 2,
    DWT2_DD97_F32 = 3,
    DWT2_DD137_F32 = 4
} dwt2_wavelet;

/* Element types.  DWT2_I32 is the only type of the integer wavelet; the float wavelets take
 * DWT2_F32, DWT2_BF16 or DWT2_F16 storage. */
typedef enum {
    DWT2_I32 = 0,
    DWT2_F32 = 1,
    DWT2_BF16 = 2,
    DWT2_F16 = 3
} dwt2_dtype;

typedef enum {
    DWT2_OK = 0,
    DWT2_EINVAL = 1,        /* invalid argument (null/unaligned pointer, size, level count) */
    DWT2_EUNSUPPORTED = 2,  /* valid but unsupported combination (e.g. bf16 with the int wavelet) */
    DWT2_ENOMEM = 3,        /* workspace (or host memory of a plan) too small */
    DWT2_ECUDA = 4,         /* a CUDA call failed; see dwt2_last_error() */
    DWT2_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
    DWT2_EINTERNAL = 6
} dwt2_status;

/* The GPU evaluation schemes.  DWT2_SCHEME_NONSEP is the product (Eq. 5).  The separable schemes
 * are comparators of the paper's separable lifting (Eq. 3):
 *   DWT2_SCHEME_SEP_FUSED    one pass per level like NONSEP, but evaluating the four separable
 *                            steps P, P*, U, U* of Eq. 3 one after the other;
 *   DWT2_SCHEME_SEP_TWOPASS  the customary GPU separable transform: a row kernel (all
 *                            horizontal lifting steps) and then a column kernel (all vertical
 *                            ones), two HBM round trips per level.  For the integer wavelet
 *                            this rounds in rows-then-columns order, which differs from Eq. 3's
 *                            order in the last bits of some coefficients.
 *   DWT2_SCHEME_ADAPTED      the adapted non-separable scheme (Sec. 3, Fig. 3): P = P0 + P1,
 *                            U = U0 + U1 with the constant monomials P0, U0 applied as local
 *                            steps (no neighbouring quad read) before the fused steps with P1,
 *                            U1.  Float wavelets only (DWT2_EUNSUPPORTED for the integer one).
 *   DWT2_SCHEME_CONV         the separable convolution (Eq. 4): the whole 1-D analysis filter
 *                            bank along rows as one step, then along columns, each followed by
 *                            the subsampling (one pass per level).  Float wavelets only. */
typedef enum {
    DWT2_SCHEME_NONSEP = 0,
    DWT2_SCHEME_SEP_FUSED = 1,
    DWT2_SCHEME_SEP_TWOPASS = 2,
    DWT2_SCHEME_ADAPTED = 3,
    DWT2_SCHEME_CONV = 4
} dwt2_scheme;

/* One subband plane inside the caller's coefficient buffer. */
typedef struct {
    int64_t offset_bytes; /* from the start of the coefficient buffer; a multiple of 256 */
    int32_t h, w;         /* rows, columns (either may be 0, e.g. HL of a 1-column plane) */
    int32_t pitch_bytes;  /* row pitch, a multiple of 16 */
    int32_t dtype;        /* dwt2_dtype of the elements */
    int32_t level;        /* 1..levels */
    char kind;            /* 'A' = LL, 'H' = HL, 'V' = LH, 'D' = HH */
    char reserved[3];
} dwt2_band;

/* Human-readable text of a status code (static storage). */
const char* dwt2_status_string(int status);

/* Text of the last CUDA error seen by the calling thread ("" if none). */
const char* dwt2_last_error(void);

/* Largest valid level count for an H x W image: the number of halvings (rounding up) that
 * bring the longer side to 1, at least 1.  Returns 0 for H < 1 or W < 1. */
int dwt2_max_levels(int H, int W);

/* Layout of the coefficient buffer for (H, W, levels, band_dtype).
 * bands: caller array of 1 + 3 * levels entries (may be NULL to query only coeff_bytes), filled
 *        in band-list order LL_levels, then HL_j, LH_j, HH_j for j = levels .. 1.
 * coeff_bytes: total size of the coefficient buffer.
 * LL_levels is DWT2_I32 for the integer wavelet and DWT2_F32 otherwise; the other bands have
 * band_dtype.  band_dtype DWT2_I32 selects the integer layout.
 * Returns DWT2_EINVAL for invalid sizes or level counts. */
int dwt2_layout(int H, int W, int levels, int band_dtype, dwt2_band* bands, size_t* coeff_bytes);

/* Bytes of device workspace that dwt2_forward / dwt2_inverse / the adjoints need for these
 * arguments: a 256-byte status header plus two ping-pong planes for the intermediate LL levels
 * (fp32 for the float wavelets, int32 for the integer one).  Returns 0 for invalid arguments.
 * The workspace header must be zeroed before first use (dwt2_workspace_init). */
size_t dwt2_workspace_bytes(int H, int W, int levels, int wavelet, int band_dtype);

/* Zero the 256-byte status header of a workspace (asynchronous on stream). */
int dwt2_workspace_init(void* workspace, size_t ws_bytes, void* stream);

/* Synchronise stream, read the status word of the workspace header and clear it.  Returns
 * DWT2_OK, or DWT2_ETIMEOUT if any kernel since the last check gave up a bounded wait. */
int dwt2_check_status(void* workspace, void* stream);

/* Forward transform (Eq. 5, the non-separable lifting scheme), levels 1..levels.
 * img: device pointer to H x W elements of img_dtype with row pitch img_pitch_bytes (a multiple
 *      of the element size, >= W * element size); 16-byte-aligned pitch and base take the TMA
 *      load path, others a plain-load path with identical results.
 *      img_dtype: DWT2_I32 for the integer wavelet; DWT2_F32 or band_dtype for the float ones.
 * coeffs: device buffer of dwt2_layout(...)'s coeff_bytes, 256-byte aligned.
 * workspace: device buffer of at least dwt2_workspace_bytes(...) bytes, 256-byte aligned.
 * The call only enqueues work on stream. */
int dwt2_forward(const void* img, int64_t img_pitch_bytes, int H, int W, int img_dtype,
                 void* coeffs, void* workspace, size_t ws_bytes, int wavelet, int levels,
                 int band_dtype, void* stream);

/* Forward transform with a chosen scheme (DWT2_SCHEME_*); DWT2_SCHEME_NONSEP is dwt2_forward.
 * The separable schemes support DWT2_F32 / DWT2_I32 storage only.  DWT2_SCHEME_SEP_TWOPASS
 * needs dwt2_workspace_bytes_scheme(...) bytes of workspace (an extra full-size plane). */
int dwt2_forward_scheme(const void* img, int64_t img_pitch_bytes, int H, int W, int img_dtype,
                        void* coeffs, void* workspace, size_t ws_bytes, int wavelet, int levels,
                        int band_dtype, int scheme, void* stream);
size_t dwt2_workspace_bytes_scheme(int H, int W, int levels, int wavelet, int band_dtype,
                                   int scheme);

/* Inverse transform: the exact inverse of each fused step, in reverse order (Eq. 5 inverted:
 * the inverse spatial update [1 -U -U* UU*; 0 1 0 -U*; 0 0 1 -U; 0 0 0 1], then the inverse
 * spatial predict [1 0 0 0; -P 1 0 0; -P* 0 1 0; PP* -P* -P 1]), levels levels..1.
 * coeffs (input) as laid out by dwt2_layout; img (output) H x W of img_dtype with pitch
 * img_pitch_bytes.  Integer: bit-exact reconstruction of dwt2_forward's input. */
int dwt2_inverse(const void* coeffs, void* img, int64_t img_pitch_bytes, int H, int W,
                 int img_dtype, void* workspace, size_t ws_bytes, int wavelet, int levels,
                 int band_dtype, void* stream);

/* Adjoints (transposes) of the float transforms, for gradients (the float CDF wavelets, DWT2_F32
 * image and band storage only; the integer and the Deslauriers-Dubuc wavelets return
 * DWT2_EUNSUPPORTED).
 *   dwt2_forward_adjoint  applies W^T, the transpose of dwt2_forward: g_coeffs (laid out by
 *                         dwt2_layout) -> g_img (H x W).  Levels levels..1, each level the
 *                         transposed fused steps in reverse order: the transpose of the spatial
 *                         update (U*^T then U^T), then of the spatial predict (P*^T then P^T).
 *   dwt2_inverse_adjoint  applies W^-T, the transpose of dwt2_inverse: g_img -> g_coeffs.
 *                         Levels 1..levels.
 * The whole-sample symmetric boundary of the forward becomes, in the transpose, taps that add
 * twice into the sample a mirrored read used twice, and no reads from beyond the edge.  Padding
 * bytes of g_coeffs (between and after band rows) are neither read nor written.  Workspace and
 * stream as for dwt2_forward / dwt2_inverse. */
int dwt2_forward_adjoint(const void* g_coeffs, void* g_img, int64_t g_img_pitch_bytes, int H,
                         int W, int img_dtype, void* workspace, size_t ws_bytes, int wavelet,
                         int levels, int band_dtype, void* stream);
int dwt2_inverse_adjoint(const void* g_img, int64_t g_img_pitch_bytes, int H, int W, int img_dtype,
                         void* g_coeffs, void* workspace, size_t ws_bytes, int wavelet, int levels,
                         int band_dtype, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Uniform batches: N images of the same H x W, wavelet, levels and types, transformed by the
 * same per-level kernels as the single-image calls (one launch per level covers all N images; the
 * image index is the third grid dimension).  Each image's result equals, bit for bit, what the
 * single-image call gives for it.  The paper transforms one image at a time (Sec. 4); batching
 * changes only how many images a launch covers, not the arithmetic.
 *   img / g_img               image z at img + z * img_batch_bytes, rows img_pitch_bytes apart;
 *                             img_batch_bytes >= H * img_pitch_bytes when N > 1.
 *   coeffs / g_coeffs         image z's coefficients, laid out by dwt2_layout(H, W, levels,
 *                             band_dtype), at coeffs + z * coeff_batch_bytes; coeff_batch_bytes
 *                             >= that layout's total bytes and a multiple of 16 when N > 1
 *                             (a contiguous (N, total/4) float32 tensor qualifies, since the
 *                             layout's total is a multiple of 256 bytes).
 *   N                         1..65535 (the batch strides are ignored when N == 1).
 *   workspace, ws_bytes       at least dwt2_workspace_bytes_batch(N, H, W, levels, wavelet,
 *                             band_dtype) bytes, 16-byte aligned, prepared by dwt2_workspace_init;
 *                             images share the status word at its start and each has its own
 *                             region for the intermediate LL planes.
 * Errors as for the single-image calls (DWT2_EINVAL for a bad N or batch stride); the adjoint
 * entries are float-only as above.  Tensor maps address the batch as a third dimension, so a
 * batch stride that is not a multiple of 16 bytes selects the plain-load path. */
size_t dwt2_workspace_bytes_batch(int N, int H, int W, int levels, int wavelet, int band_dtype);
int dwt2_forward_batch(const void* img, int64_t img_pitch_bytes, int64_t img_batch_bytes, int N,
                       int H, int W, int img_dtype, void* coeffs, int64_t coeff_batch_bytes,
                       void* workspace, size_t ws_bytes, int wavelet, int levels, int band_dtype,
                       void* stream);
int dwt2_inverse_batch(const void* coeffs, int64_t coeff_batch_bytes, void* img,
                       int64_t img_pitch_bytes, int64_t img_batch_bytes, int N, int H, int W,
                       int img_dtype, void* workspace, size_t ws_bytes, int wavelet, int levels,
                       int band_dtype, void* stream);
int dwt2_forward_adjoint_batch(const void* g_coeffs, int64_t coeff_batch_bytes, void* g_img,
                               int64_t g_img_pitch_bytes, int64_t g_img_batch_bytes, int N, int H,
                               int W, int img_dtype, void* workspace, size_t ws_bytes, int wavelet,
                               int levels, int band_dtype, void* stream);
int dwt2_inverse_adjoint_batch(const void* g_img, int64_t g_img_pitch_bytes,
                               int64_t g_img_batch_bytes, int N, int H, int W, int img_dtype,
                               void* g_coeffs, int64_t coeff_batch_bytes, void* workspace,
                               size_t ws_bytes, int wavelet, int levels, int band_dtype,
                               void* stream);

/* ---------------------------------------------------------------------------------------------
 * Batched plans: many images of any sizes, every level, ONE persistent kernel launch replayed
 * from a CUDA graph.  The work is a list of tiles (image, level, strip of 240 quad columns,
 * block of rows) in level-major order; CTAs claim tiles from a counter, and a tile of level j of
 * an image waits (bounded in time) until the same image's level j-1 (forward flow) or j+1
 * (inverse flow) has completed.
 *   imgs[i].img     image (forward, inverse adjoint: input; inverse, forward adjoint: output),
 *                   H x W of img_dtype with row pitch img_pitch_bytes (multiple of 4 bytes);
 *   imgs[i].coeffs  coefficient buffer laid out by dwt2_layout(H, W, levels, band_dtype),
 *                   16-byte aligned (output of forward, input of inverse).
 *   img_dtype       DWT2_I32 (integer wavelet) or DWT2_F32; band_dtype as for dwt2_forward
 *                   (adjoint directions: DWT2_F32 only).
 *   workspace       device buffer of dwt2_plan_workspace_bytes(...), 256-byte aligned, header
 *                   zeroed (dwt2_workspace_init); it holds every image's intermediate LL planes.
 *   tune_cache      path of a text file of tuned schedules, or NULL.  With a path, the first
 *                   plan of a kind (GPU, direction, wavelet, storage, levels, image count, size
 *                   class) times candidate tile heights and CTAs per SM on itself -- running the
 *                   transform several times -- and appends the winner; later plans read it.
 *                   Without a path a default schedule is used.
 * The plan allocates its own small device buffers (descriptors, tensor maps, counters) at
 * creation and captures [counter reset, kernel] in a graph; buffers are bound at creation.
 * Results are identical to the single-image entry points (bit for bit for the integer wavelet).
 * The Deslauriers-Dubuc wavelets take the forward and inverse directions (their adjoint
 * directions return DWT2_EUNSUPPORTED). */
typedef struct {
    void* img;
    int64_t img_pitch_bytes;
    int H, W;
    void* coeffs;
} dwt2_image_desc;

typedef enum {
    DWT2_DIR_FORWARD = 0,
    DWT2_DIR_INVERSE = 1,
    DWT2_DIR_FORWARD_ADJOINT = 2, /* W^T: band gradients (coeffs) -> image gradient (img) */
    DWT2_DIR_INVERSE_ADJOINT = 3  /* W^-T: image gradient (img) -> band gradients (coeffs) */
} dwt2_direction;

typedef struct dwt2_plan dwt2_plan;

size_t dwt2_plan_workspace_bytes(const dwt2_image_desc* imgs, int n, int wavelet, int levels,
                                 int band_dtype);
int dwt2_plan_create(const dwt2_image_desc* imgs, int n, int wavelet, int levels, int img_dtype,
                     int band_dtype, int direction, void* workspace, size_t ws_bytes,
                     const char* tune_cache, dwt2_plan** plan);
/* Enqueue the plan's graph on stream (asynchronous). */
int dwt2_plan_execute(dwt2_plan* plan, void* stream);
/* The schedule in use: quad rows per tile at level 1 (level j uses max(4, rows >> (j - 1))), CTAs
 * per SM, number of tiles. */
int dwt2_plan_info(const dwt2_plan* plan, int* rows_per_tile, int* ctas_per_sm, int* n_tiles);
int dwt2_plan_destroy(dwt2_plan* plan);

/* ---------------------------------------------------------------------------------------------
 * Self-test of the bounded device waits (no counterpart in the paper; failure detection for the
 * library).  Every wait inside the kernels -- on a stage barrier, or in the persistent kernels on
 * another tile's completion counter -- gives up after a time limit of 2 s: the kernel raises its
 * abort flag, records DWT2_ETIMEOUT in the workspace status word and returns.  This call launches
 * one warp that waits on a barrier phase nothing completes (which = 0) or on a counter in the
 * workspace header that nothing increments (which = 1).
 *   workspace  at least 256 bytes, prepared by dwt2_workspace_init (which zeroes the counter).
 * Returns DWT2_OK once launched; about 2 s later dwt2_check_status(workspace, stream) reports
 * DWT2_ETIMEOUT.  The context stays usable. */
int dwt2_selftest_wait_timeout(int which, void* workspace, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Forward transform without a caller-provided workspace.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory (for example code whose host
 * application owns all device memory and passes in only the input and output buffers, or a
 * real-time loop that must never call the allocator).  Instead of a workspace it uses a scratch
 * array of DWT2_STATIC_SCRATCH_BYTES built into the library, which every GPU that loads this part
 * of the library keeps until the process exits.
 *   - Arguments are those of dwt2_forward without workspace / ws_bytes.
 *   - Returns DWT2_ENOMEM (with a message in dwt2_last_error) when the transform needs more
 *     scratch than DWT2_STATIC_SCRATCH_BYTES, i.e. dwt2_workspace_bytes(...) of these arguments
 *     exceeds it; 4096 x 4096 fp32 or int32 fits at any level count, and one level fits at any
 *     size.
 *   - It allocates nothing: no cudaMalloc, no cudaFree, no allocating library call.
 *   - Every call looks up the scratch's device address in the current device's current context
 *     (a host-side lookup, so a device reset or a switch of context is followed); the first
 *     call in a context also loads the library's device code there: make that first call
 *     before any stream capture.
 *   - Invalid arguments are rejected before anything is queued on the stream.  A valid call
 *     clears the status word at the start of the scratch on stream; the scratch keeps the
 *     previous call's contents otherwise.  All calls share the one scratch array: calls that may
 *     run at the same time on the GPU (other streams, other host threads) race and must be
 *     ordered by the caller.
 *   - Device-side wait timeouts (see dwt2_selftest_wait_timeout) are recorded only in that
 *     scratch, which the caller cannot read, and the next call clears them: this entry point
 *     does not report them.  A caller that must learn of a timeout uses dwt2_forward with a
 *     workspace and dwt2_check_status. */
#define DWT2_STATIC_SCRATCH_BYTES (24u << 20)
int dwt2_forward_static(const void* img, int64_t img_pitch_bytes, int H, int W, int img_dtype,
                        void* coeffs, int wavelet, int levels, int band_dtype, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DWT2_H */
