/*
 * pxst.h -- C ABI of the GB300 (sm_103a) PXST hot-path library, libpxst.so.
 *
 * The method is ptychographic X-ray speckle tracking as described in Morgan et al.,
 * "speckle-tracking: a software suite for ptychographic X-ray speckle tracking".
 * The library implements steps (i) and (ii) of the main loop (section "Main loop"):
 * make the reference image, then update the pixel map, on one GPU.
 *
 * Conventions for every entry point
 *   - Array pointers are DEVICE pointers into C-contiguous arrays owned by the caller.
 *     The library never allocates device memory: scratch space is the caller's
 *     `workspace` buffer, at least pxst_workspace_size() bytes, 256-byte aligned.
 *   - Layouts (discrete forward model of section "Initialisation"):
 *       frames  float32 [n_frames][ny][nx]   I[n, i, j]
 *       W       float32 [ny][nx]             whitefield
 *       mask    uint8   [ny][nx]             M: 1 = good pixel, 0 = excluded
 *       u       float64 [2][ny][nx]          pixel map; u[0] = row (slow scan, i),
 *                                            u[1] = column (fast scan, j), in units of
 *                                            reference-image pixels
 *       delta   float64 [n_frames][2]        (Delta_i[n], Delta_j[n]), same units
 *       I_ref   float32 [ref_ny][ref_nx]     reference image
 *       w       float32 [ref_ny][ref_nx]     accumulated weight sum_n sum_x b M W^2
 *                                            (0 = the reference pixel is not covered)
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream).
 *     Argument and shape errors are detected on the host and returned before anything
 *     is launched. Problems found on the device (a non-finite or out-of-range pixel-map
 *     entry, a wait that timed out) set bits in a status word inside the workspace;
 *     pxst_get_status() synchronises the stream and returns and clears them.
 *   - The workspace must not be shared by calls that may run concurrently.
 */
#ifndef PXST_H
#define PXST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t pxst_status;
#define PXST_OK            0
#define PXST_ERR_ARG      (-1)   /* null pointer, negative size, bad option value      */
#define PXST_ERR_SHAPE    (-2)   /* inconsistent or unsupported dimensions             */
#define PXST_ERR_RANGE    (-3)   /* device saw a non-finite / out-of-range map entry   */
#define PXST_ERR_CUDA     (-4)   /* a CUDA runtime call failed                         */
#define PXST_ERR_NOMEM    (-5)   /* workspace smaller than pxst_workspace_size()       */
#define PXST_ERR_TIMEOUT  (-6)   /* a device-side wait gave up                         */
#define PXST_ERR_INPUT    (-7)   /* device saw a non-finite frame value, or a whitefield
                                    value that is not finite and positive, at a pixel
                                    with M = 1                                          */

/* Device status bits (pxst_get_status reports the most severe as a pxst_status). */
#define PXST_DEV_NONFINITE_U  0x1
#define PXST_DEV_U_RANGE      0x2
#define PXST_DEV_TIMEOUT      0x4
#define PXST_DEV_BAD_INPUT    0x8   /* see PXST_ERR_INPUT. A pixel with a bad whitefield value
                                       is treated as masked (keeps its map, error NaN, adds
                                       nothing to the reference image); a non-finite frame value
                                       adds nothing to the reference image, and its pixel keeps
                                       its map with error +inf (no candidate has a finite error) */

typedef struct {
    int32_t n_frames;   /* N  >= 1 */
    int32_t ny, nx;     /* detector rows (slow scan) and columns (fast scan) */
    int32_t ref_ny, ref_nx;   /* reference-image grid */
} pxst_dims;

/* Arithmetic form of the candidate search. */
#define PXST_FORM_FP32  0   /* direct sum of (I - W R)^2 in FP32 on CUDA cores */
#define PXST_FORM_BF16  1   /* cross term on tensor cores, BF16 operands, FP32 accumulation
                               (pixels with candidates not valid in every frame ranked again
                               with each candidate's variance over its valid frames, a second
                               contraction); the best rescore_k candidates per pixel, the 3x3
                               about the minimum and the fit are then evaluated exactly as in
                               FP32 */
#define PXST_FORM_TF32  2   /* as PXST_FORM_BF16 with TF32 operands */

typedef struct {
    int32_t win_y, win_x;  /* search window half-widths S_y, S_x: candidates are the
                              integers c = round(u) + (a, b), |a| <= S_y, |b| <= S_x */
    int32_t quadratic;     /* 1: 3x3 paraboloid sub-pixel refinement, 0: integer argmin */
    int32_t form;          /* PXST_FORM_* */
    int32_t rescore_k;     /* tensor forms: candidates per pixel re-evaluated in FP32:
                              4 or 8 (0 = 8 below 128 frames, else 4) */
    int32_t tile;          /* tile shape (0 = automatic). FP32 form: bits 0-3 the tile height in
                              rows of 32 pixels, 0 (automatic), 1, 2, 4 or 8 (a height whose
                              staging does not fit falls back to the automatic choice); bits
                              4-5 the strip length, 0 (automatic), 1, 2, 3 = 7, 9, 11 window
                              columns per strip. Tensor forms: 0 = 8 x 16 pixels
                              against 8 x 32 candidates, 1 = 4 x 32 / 4 x 64, 2 = 2 x 64 /
                              2 x 128. Any other value is PXST_ERR_ARG. */
    int64_t timeout_ns;    /* limit of every device-side wait of the call, in ns (the
                              tensor forms' pipeline waits); 0 = 1 s. A wait that runs out
                              sets PXST_DEV_TIMEOUT and the kernel returns without hanging */
} pxst_options;

/* Bytes of workspace needed by every entry point below for these sizes. */
size_t pxst_workspace_size(const pxst_dims *dims, const pxst_options *opts);

/*
 * make_object_map -- "Make reference image" (section "Main loop", its first
 * pseudo-code block, with the bilinear assignment rule of section "Sub-pixel
 * interpolation"). For every frame n and pixel (i, j) with M = 1, the point
 * u[:, i, j] - Delta[n] distributes M W I[n,i,j] into a numerator and M W^2 into w over
 * the four surrounding reference pixels with bilinear weights; corners outside the grid
 * are dropped. Then I_ref = numerator / w where w > 0 and 0 elsewhere.
 * Outputs I_ref and w are overwritten. Accumulation: FP32 in shared memory per tile,
 * FP64 in global memory, FP64 division.
 */
pxst_status pxst_make_object_map(const pxst_dims *dims, const float *frames, const float *W,
                                 const uint8_t *mask, const double *u, const double *delta,
                                 float *I_ref, float *w, void *workspace, size_t ws_bytes,
                                 void *stream);

/*
 * make_object_map_noalloc -- the same computation as pxst_make_object_map, for callers
 * that cannot allocate device memory: for example an acquisition plug-in running inside a
 * host framework that owns all of the GPU's memory, or a real-time loop that cannot accept
 * the implicit synchronisation and latency of cudaMalloc. It takes no workspace and
 * allocates nothing (no cudaMalloc, cudaFree or allocating library call); its scratch is
 * one fixed device array inside libpxst.so, about 16.1 MiB, which every GPU that loads the
 * library holds until the process exits. The paper has no counterpart to this entry point.
 *   Limits: n_frames <= 8192 and ref_ny * ref_nx <= 1048576; larger sizes return
 *   PXST_ERR_NOMEM (with a message on stderr) before anything is launched.
 *   The first call on a device (and the first after the device's context was reset or
 *   re-created) looks up the array's device address (cudaGetSymbolAddress) with that device
 *   current; with lazy module loading (the CUDA default) that first call is also the one
 *   that loads the library's device code and reserves the array, so make it as a warm-up
 *   before the rest of the GPU's memory is taken and before any stream capture.
 *   All calls share the one array and it keeps the last call's contents (each call clears
 *   what it accumulates into): calls that may overlap on the GPU, on any stream, race.
 *   Device-side status bits of this call are not reported (there is no workspace to read).
 */
pxst_status pxst_make_object_map_noalloc(const pxst_dims *dims, const float *frames,
                                         const float *W, const uint8_t *mask, const double *u,
                                         const double *delta, float *I_ref, float *w,
                                         void *stream);

/*
 * update_pixel_map -- "Update pixel mapping" (section "Main loop", second pseudo-code
 * block, and the quadratic_refinement option described right after it). For every pixel
 * with M = 1 and each integer candidate c in the window centred on round(u) (halves
 * round up): error(c) = sum_n (I - W R_n(c))^2 and var(c) = sum_n (I - W)^2, where
 * R_n(c) reads I_ref at c - Delta[n] by the masked, renormalised bilinear rule of
 * section "Sub-pixel interpolation" (mask: inside the grid and w > 0); frames whose
 * read has no valid corner are left out of both sums. e = error / var (error if
 * var = 0, +inf if no frame is valid). u becomes the first minimum in row-major window
 * order, refined by a least-squares paraboloid through the 3x3 errors about it when
 * opts->quadratic is set (per-axis parabolas where the 3x3 is incomplete or not convex).
 * u_inout is updated in place; pixels with M = 0, or without any valid candidate, keep
 * their u. err_out (nullable) receives e at the chosen integer candidate (NaN where
 * M = 0, +inf where nothing was valid).
 */
pxst_status pxst_update_pixel_map(const pxst_dims *dims, const pxst_options *opts,
                                  const float *frames, const float *W, const uint8_t *mask,
                                  const float *I_ref, const float *w, const double *delta,
                                  double *u_inout, float *err_out, void *workspace,
                                  size_t ws_bytes, void *stream);

/*
 * iterate -- n_iter passes of the main loop's steps (i) and (ii): make_object_map from
 * the current u, then update_pixel_map with that reference (section "Main loop").
 * On return I_ref and w hold the reference built in the last pass, u_inout the map
 * after the last update and err_out (nullable) its errors.
 */
pxst_status pxst_iterate(const pxst_dims *dims, const pxst_options *opts, int32_t n_iter,
                         const float *frames, const float *W, const uint8_t *mask,
                         const double *delta, double *u_inout, float *I_ref, float *w,
                         float *err_out, void *workspace, size_t ws_bytes, void *stream);

/*
 * reference_terms -- the per-candidate sums that turn the error of the update step
 * into a cross term plus separable parts (expanding the square of the "Update pixel
 * mapping" error): T[c] = sum_n V_n(c) R_n(c)^2 and n_valid[c] = sum_n V_n(c) for every
 * reference pixel c, with R_n(c) and V_n(c) the masked bilinear read of I_ref at
 * c - Delta[n] and its validity, as in pxst_update_pixel_map.
 * T float32 [ref_ny][ref_nx], n_valid int32 [ref_ny][ref_nx], both overwritten.
 */
pxst_status pxst_reference_terms(const pxst_dims *dims, const float *I_ref, const float *w,
                                 const double *delta, float *T, int32_t *n_valid,
                                 void *workspace, size_t ws_bytes, void *stream);

/*
 * wait_flag -- a stream-ordered wait for an external producer, for reconstructions that
 * start while the scan is still being acquired: the kernels queued on `stream` after this
 * call run once the 32-bit value at `flag` is >= `target` (the producer -- a host thread
 * writing pinned host memory, which is device-accessible under unified addressing, or a
 * copy into device memory -- raises it, for instance to the number of frames it has
 * written). One GPU thread polls it, with back-off, for at most timeout_ns (> 0; 0 = 1 s);
 * if the value has not arrived by then it sets PXST_DEV_TIMEOUT in the workspace's status
 * word and returns, so the stream never hangs: pxst_get_status then reports
 * PXST_ERR_TIMEOUT (the work queued after the wait has run on whatever the inputs held).
 * The producer must not be a kernel that could be waiting for a slot on the GPU.
 * Not described in the paper: it serves the acquisition loop around the method.
 */
pxst_status pxst_wait_flag(const int32_t *flag, int32_t target, int64_t timeout_ns, void *workspace,
                           size_t ws_bytes, void *stream);

/* Synchronise `stream`, then return (and clear) the device status word in `workspace`:
 * PXST_OK, PXST_ERR_RANGE, PXST_ERR_INPUT or PXST_ERR_TIMEOUT (the most severe, in the
 * order timeout, range, input). `bits_out` (nullable) gets the raw bits. */
pxst_status pxst_get_status(void *workspace, void *stream, int32_t *bits_out);

/* Number of pixels of the last update on this workspace that needed the per-frame
 * validity rule (a candidate read an uncovered or off-grid reference pixel), plus those
 * handled by the global-memory path (tile window too large for shared memory, or too many
 * frames to stage). Synchronises `stream`. */
pxst_status pxst_last_exact_count(void *workspace, void *stream, int64_t *count_out);

/* Per-kernel timing with CUDA events recorded on the launching stream.
 * pxst_timing_enable(1) starts recording (and clears earlier records);
 * pxst_timing_read() synchronises the recorded events and returns, for kernel k,
 * the number of launches and their summed duration in ms. Kernel ids: */
#define PXST_K_PREPARE    0   /* per-frame shift table */
#define PXST_K_SCATTER    1   /* make_object_map scatter (includes the accumulator clear and the
                                 reference weights per fractional-shift class) */
#define PXST_K_NORMALISE  2   /* make_object_map normalisation */
#define PXST_K_SEARCH     3   /* update_pixel_map candidate search + refinement */
#define PXST_K_EXACT      4   /* update_pixel_map exact path */
#define PXST_K_REFTERMS   5   /* reference_terms */
#define PXST_K_TPREP      6   /* tensor forms: centred frames, once per call */
#define PXST_K_GTABLE     7   /* tensor forms: shifted reference per frame, T~ and n_valid */
#define PXST_K_TSEARCH    8   /* tensor forms: tensor-core ranking of every candidate (both passes) */
#define PXST_K_RESCORE    9   /* tensor forms: exact FP32 evaluation of the best candidates */
#define PXST_K_ERROR      10  /* calc_error (with the per-pixel variance) */
#define PXST_K_TRANS      11  /* update_translations (with the per-pixel variance) */
#define PXST_K_FILTER     12  /* filter_map */
#define PXST_K_FRAC       13  /* update_pixel_map_fractional: the fractional candidates */
#define PXST_K_DEFOCUS    14  /* defocus_sweep (includes its make_object_map launches) */
#define PXST_K_INTEGRATE  15  /* integrate_map (the stencil codes and the conjugate-gradient solve) */
#define PXST_K_COUNT      16
pxst_status pxst_timing_enable(int32_t enable);
pxst_status pxst_timing_read(int64_t *launches, double *total_ms, int32_t n_kernels);
const char *pxst_kernel_name(int32_t k);

/* Diagnostic of the tensor-core contraction used by the BF16 / TF32 forms: one CTA
 * computes D[128][256] = A[128][K] . B[256][K]^T (D float32 row-major) with the same TMA,
 * tcgen05.mma and TMEM path as the search. A and B are row-major device arrays of
 * bfloat16 (form PXST_FORM_BF16) or float32 read as TF32 (PXST_FORM_TF32); K * element
 * size must be a multiple of 16 bytes and the pointers 16-byte aligned. *status (device
 * int) gets PXST_DEV_TIMEOUT if a wait ran out. Not part of the method: a self-check. */
pxst_status pxst_tensor_check(int32_t form, int32_t K, const void *A, const void *B, float *D,
                              int32_t *status, void *stream);

/* ---- Figures of merit and the translation update ------------------------------------------
 * pxst_calc_error (section "Calculate figures of merit"): the error term of Eq. 1 at each pixel
 * x and frame n, eps[n,x] = (I_n(x) - W(x) R_n)^2 / var(x), with R_n the masked renormalised
 * bilinear read of I_ref at u(x) - Delta_n (u fractional), var(x) = sum over the frames valid
 * at x of (I_n(x) - W(x))^2, frames invalid at x left out, eps = the squared residual where
 * var = 0, pixels with M = 0 (or a non-finite map) left out. Outputs (device pointers, each
 * may be NULL): pixel_err float [ny][nx] = sum over n (NaN where left out); frame_err double
 * [N] = sum over x; total_err double [1] = sum over both; ref_err float [ref_ny][ref_nx] = eps
 * scattered to u(x) - Delta_n with make_object_map's bilinear weights (corners off the grid
 * dropped) divided by the weights that landed (0 where none). Sums are FP64 atomics:
 * equal to rounding, not bitwise, from run to run. */
pxst_status pxst_calc_error(const pxst_dims *dims, const float *frames, const float *W, const uint8_t *mask,
                            const float *I_ref, const float *w, const double *u, const double *delta,
                            float *pixel_err, double *frame_err, double *total_err, float *ref_err,
                            void *workspace, size_t ws_bytes, void *stream);

/* pxst_update_translations (section "Update translations"): for every frame n and integer
 * shift (a, b), |a| <= win_y, |b| <= win_x (each at most 8, else PXST_ERR_ARG), the mean over
 * the pixels with M = 1, var(x) > 0 (var as above, at the current translations) and a valid
 * read at u(x) - Delta_n - (a, b) of (I_n(x) - W(x) R)^2 / var(x); the first minimum in
 * row-major order; with quadratic = 1 the 3x3 paraboloid of update_pixel_map about it;
 * delta_inout[n] += (a*, b*) + fit. frame_err (double [N], may be NULL) receives each frame's
 * mean error at its minimum (+inf if no pixel was valid: the translation is kept). */
pxst_status pxst_update_translations(const pxst_dims *dims, int32_t win_y, int32_t win_x, int32_t quadratic,
                                     const float *frames, const float *W, const uint8_t *mask,
                                     const float *I_ref, const float *w, const double *u, double *delta_inout,
                                     double *frame_err, void *workspace, size_t ws_bytes, void *stream);

/* pxst_update_pixel_map_fractional: the non-integer option of section "Update pixel mapping"
 * instead of the paraboloid. update_pixel_map without the fit (any form) gives each pixel's
 * integer minimum c*; then the candidates c* + (a, b) / sub, a, b in [-sub, sub], are
 * evaluated by the same masked rule with bilinear reads at the fractional positions, and u
 * becomes the first minimum in row-major order (err_out, if given, its error). A pixel whose
 * c* has no valid frame keeps its map. sub in [1, 8], else PXST_ERR_ARG; opts->quadratic is
 * ignored. Work: (2 sub + 1)^2 x N evaluations per pixel on top of the integer search. */
pxst_status pxst_update_pixel_map_fractional(const pxst_dims *dims, const pxst_options *opts, int32_t sub,
                                             const float *frames, const float *W, const uint8_t *mask,
                                             const float *I_ref, const float *w, const double *delta,
                                             double *u_inout, float *err_out, void *workspace, size_t ws_bytes,
                                             void *stream);

/* pxst_defocus_sweep (fit_defocus_registration, section "Initialisation"): for every pair of
 * map scales (sy[ky], sx[kx]) (host arrays, each in (0, 100), at most 64 pairs), the map is
 * scaled about the detector's central pixel (ny/2, nx/2), u'_a = u_a(centre) + s_a (u_a -
 * u_a(centre)), with the translations unchanged, make_object_map builds the reference image
 * (left in I_ref, w: the last pair's), and contrast[ky * n_sx + kx] (device double) receives
 * its standard deviation over its mean over the reference pixels with w > 0 (0 if none). The
 * pair with the highest contrast is the magnification estimate. */
pxst_status pxst_defocus_sweep(const pxst_dims *dims, const float *frames, const float *W, const uint8_t *mask,
                               const double *u, const double *delta, int32_t n_sy, const double *sy, int32_t n_sx,
                               const double *sx, double *contrast, float *I_ref, float *w, void *workspace,
                               size_t ws_bytes, void *stream);

/* pxst_integrate_map: the "integrate" option named at the end of section "Update pixel
 * mapping". The map is the gradient of a scalar (u = x - lambda z / (2 pi) grad Phi), so it
 * is integrated by least squares and differentiated again, which makes it irrotational.
 * Equations, one per pixel with M = 1 and axis a: the derivative of Psi along a at the
 * pixel equals u_a there, by the first of these stencils whose pixels all have M = 1:
 * central, (Psi[p+e] - Psi[p-e]) / 2; second-order forward, (-3 Psi[p] + 4 Psi[p+e] -
 * Psi[p+2e]) / 2; second-order backward, (3 Psi[p] - 4 Psi[p-e] + Psi[p-2e]) / 2; forward,
 * Psi[p+e] - Psi[p]; backward, Psi[p] - Psi[p-e] (no equation where the pixel has no good
 * neighbour along a). Psi minimises the squared residuals, by conjugate gradients on the
 * normal equations from Psi = 0, stopping when the residual of the normal equations falls
 * to tol times its start or after max_iter steps; u_inout then becomes G Psi at every
 * equation (the pixels and axes without one, and every M = 0 pixel, keep u). FP64. The
 * result is the orthogonal projection of the map onto these discrete gradient fields: a
 * map that is one (the gradient of a quadratic Psi, for instance) is returned unchanged.
 * info_out (device double[2], nullable): the steps taken and the final relative residual.
 * One cooperative launch (every block resident) runs the solve; its grid barriers give up
 * after timeout_ns (0 = 10 s) and set PXST_DEV_TIMEOUT, and every block then leaves: u is
 * left unchanged, except where a block gave up at the solve's last barrier just as the
 * others passed it (they then write their pixels' G Psi); the status reports it either way. */
pxst_status pxst_integrate_map(const pxst_dims *dims, const uint8_t *mask, double *u_inout, int32_t max_iter,
                               double tol, int64_t timeout_ns, double *info_out, void *workspace, size_t ws_bytes,
                               void *stream);

/* pxst_filter_map: the "sigma" regularisation of the pixel map named at the end of section
 * "Update pixel mapping": u(x) <- sum_y g(x - y) M(y) u(y) / sum_y g(x - y) M(y) for pixels
 * with M = 1, g(d) = exp(-|d|^2 / (2 sigma^2)) on a square support of radius floor(4 sigma +
 * 1/2) pixels per axis, zero outside the detector; M = 0 pixels keep their map; sigma = 0
 * leaves u unchanged. FP64, two separable passes. sigma must be in [0, 1024]. */
pxst_status pxst_filter_map(const pxst_dims *dims, double sigma, const uint8_t *mask, double *u_inout,
                            void *workspace, size_t ws_bytes, void *stream);

/* ---- Batched form ------------------------------------------------------------------------
 * Many independent scans of uneven frame count, detector size and window, iterated by one
 * graph launch. A pxst_scan names one scan's device arrays exactly as pxst_iterate takes
 * them (all device pointers, owned by the caller, alive and unmoved for the batch's life;
 * err_out may be NULL) and its own workspace of pxst_workspace_size(&dims, &opts) bytes.
 * Scans in one batch must not share any output array or workspace. */
typedef struct {
    pxst_dims dims;
    pxst_options opts;
    const float *frames;      /* [N][ny][nx] */
    const float *W;           /* [ny][nx] */
    const uint8_t *mask;      /* [ny][nx] */
    const double *delta;      /* [N][2] */
    double *u;                /* [2][ny][nx], updated in place */
    float *I_ref, *w;         /* [ref_ny][ref_nx] */
    float *err_out;           /* [ny][nx] or NULL */
    void *workspace;
    size_t ws_bytes;
} pxst_scan;

typedef struct pxst_batch_s *pxst_batch;

/* Plan a batch: validate every scan, optionally pick each scan's tile shape by measurement
 * (autotune = 1: pxst_autotune per shape class, which runs update_pixel_map on the scan's own
 * data and restores its map), spread the scans over n_branches parallel graph branches
 * (1..64; largest estimated work first, each to the least loaded branch) and capture n_iter
 * iterations of every scan (the pxst_iterate sequence: make_object_map, update_pixel_map)
 * into one CUDA graph. Synchronises `stream` (plan-time work runs on it). *out receives the
 * batch, to be released with pxst_batch_destroy. Errors: those of pxst_iterate for the
 * first scan that fails, PXST_ERR_ARG for bad counts, PXST_ERR_CUDA if capture fails. */
pxst_status pxst_batch_plan(const pxst_scan *scans, int32_t n_scans, int32_t n_iter, int32_t n_branches,
                            int32_t autotune, void *stream, pxst_batch *out);
/* Run the planned iterations of every scan: one cudaGraphLaunch on `stream` (asynchronous).
 * Device-side status goes to each scan's workspace as for pxst_iterate. */
pxst_status pxst_batch_run(pxst_batch batch, void *stream);
/* The branch a scan was placed on (-1 for a bad index). */
int32_t pxst_batch_branch(pxst_batch batch, int32_t scan);
void pxst_batch_destroy(pxst_batch batch);

/* Autotuner: time update_pixel_map on this scan for every tile shape its form allows
 * (pxst_options.tile), `trials` timed runs each after one warm-up, and return the shape with
 * the smallest median time (and that time in ms if best_ms is not NULL). The scan's map u is
 * saved in its workspace and restored after every run; err_out receives the last run's
 * errors. Results are cached per shape class (dims, window, form, rescore_k) for the
 * process. Synchronises `stream`; PXST_ERR_ARG on a capturing stream. */
pxst_status pxst_autotune(const pxst_scan *scan, int32_t trials, void *stream, int32_t *best_tile,
                          float *best_ms);

/* Running total of the kernel launches this library has issued in this process (every
 * entry point; launches captured into a graph are counted once, at capture). A caller
 * reads it before and after a region to count the kernels that region launched. */
pxst_status pxst_launch_count(int64_t *count_out);

/* Human-readable text for a status code. */
const char *pxst_status_string(pxst_status s);

/* Library version string and the CUDA architecture it was compiled for. */
const char *pxst_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PXST_H */
