// pxst_common.cuh -- device helpers and the workspace layout shared by the kernels of
// libpxst.so (sm_103a). Nothing here is shared with the CPU oracle.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "pxst.h"

namespace pxst {

// -Delta[n] split per axis into an integer part and a fraction in [0, 1):
//   -Delta = k + f.  A reference read at integer candidate c then touches the corners
//   c + k and c + k + 1 with weights (1 - f) and f, and a scatter of u - Delta touches
//   floor(u) + k (+1) with the fraction frac(u) + f (carried into k when >= 1).
struct FrameShift {
    int ky, kx;
    float fy, fx;
};

// A pixel's map coordinates split once into integers and FP32 fractions in [0, 1), with its
// var(x) (-1: the pixel does not count) and whitefield, for the kernels that read them once
// per frame (FP64 is a small fraction of FP32 on this GPU); 32 bytes, read as two 16-byte loads.
struct __align__(16) PixSplit {
    int i0, i1;
    float f0, f1;
    float var, W;
    int pad0, pad1;
};

// Workspace header: the device status word and a few per-call scalars.
struct WsHeader {
    int status;        // PXST_DEV_* bits, sticky until pxst_get_status
    int n_exact;       // pixels appended to the global-path list by the last update
    int n_exact_cta;   // pixels of the last update with a strip evaluated by the per-frame rule
    int kmin_y, kmax_y, kmin_x, kmax_x;   // range of the integer shifts over all frames
    int n_edge_tiles;  // tensor forms: tiles listed for the masked ranking
    int n_rescore_pix;     // tensor forms: pixels listed for the general rescore
    int n_second;      // tensor forms: pixels listed for the rescore's second 3x3 (follows n_rescore_pix)
    // frames grouped by their fractional shift (fy, fx): the reference weights of make_object_map
    // are formed per class (n_classes > kMaxClasses: too many classes, the scatter forms them)
    int n_classes;
    float cls_fy[8], cls_fx[8];
    int pad[37];
};
static_assert(sizeof(WsHeader) == 256, "header is one 256-byte line");

constexpr int kMaxClasses = 8;          // fractional-shift classes of the weight image
constexpr int kClassFramesMax = 2048;   // frames the class assignment handles (more: no classes)

// Candidates per pixel kept by the tensor-core ranking (the rescore evaluates the first
// 4 or all 8 of them exactly).
constexpr int kTopK = 8;
constexpr int kTransMax = 17 * 17;     // translation update: shifts within +-8 on each axis

constexpr int kIntegMaxBlocks = 4096;  // integrate: blocks of the cooperative launch (partial sums)

// Byte offsets of each region inside the caller's workspace (all 256-byte aligned).
struct WsLayout {
    size_t header, shifts, exact_list, num, den, u_save, var_px, usplit, tacc_sum, tacc_cnt, delta_tmp, filt_den;
    size_t integ_buf, integ_type, integ_bar;   // integrate: CG vectors, equation types, barrier
    size_t fclass, dcls;     // class of each frame; one zero-shift weight image per class
    // precision forms only (zero size otherwise)
    size_t At, G, A2, V, Tt, nvalid, Rm, cand, edge, wlist, second;
    int Npad;
    size_t total;
};

inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// frames padded to whole 128-byte operand rows of the tensor-core form
inline int tensor_npad(int n_frames, int form) {
    const int kb = form == PXST_FORM_TF32 ? 32 : 64;
    return (n_frames + kb - 1) / kb * kb;
}

inline WsLayout ws_layout(const pxst_dims &d, int form = PXST_FORM_FP32) {
    WsLayout L;
    const size_t P = (size_t)d.ny * d.nx, R = (size_t)d.ref_ny * d.ref_nx;
    size_t off = 0;
    L.header = off;     off += align256(sizeof(WsHeader));
    L.shifts = off;     off += align256(sizeof(FrameShift) * (size_t)d.n_frames);
    L.exact_list = off; off += align256(sizeof(int) * P);
    L.num = off;        off += align256(sizeof(double) * R);
    L.den = off;        off += align256(sizeof(double) * R);
    L.u_save = off;     off += align256(sizeof(double) * 2 * P);   // the autotuner's copy of u
    L.var_px = off;     off += align256(sizeof(float) * P);        // figures of merit: var(x)
    L.usplit = off;     off += align256(sizeof(PixSplit) * P);     // translation update: split map
    L.tacc_sum = off;   off += align256(sizeof(double) * kTransMax * (size_t)d.n_frames);
    L.tacc_cnt = off;   off += align256(sizeof(unsigned long long) * kTransMax * (size_t)d.n_frames);
    L.delta_tmp = off;  off += align256(sizeof(double) * 2 * (size_t)d.n_frames);
    L.filt_den = off;   off += align256(sizeof(double) * P);        // the map filter's row pass
    L.fclass = off;     off += align256(sizeof(int) * (size_t)d.n_frames);
    L.dcls = off;       off += align256(sizeof(float) * kMaxClasses * R);
    // integrate: psi, r, the search direction d, q = A d, per-block partial sums
    L.integ_buf = off;  off += align256(sizeof(double) * (4 * P + 2 * (size_t)kIntegMaxBlocks));
    L.integ_type = off; off += align256(2 * P);
    L.integ_bar = off;  off += align256(2 * sizeof(unsigned));
    L.Npad = 0;
    L.At = L.G = L.A2 = L.V = L.Tt = L.nvalid = L.Rm = L.cand = L.edge = L.wlist = L.second = off;
    if (form == PXST_FORM_BF16 || form == PXST_FORM_TF32) {
        const size_t es = form == PXST_FORM_TF32 ? 4 : 2;
        L.Npad = tensor_npad(d.n_frames, form);
        L.At = off;     off += align256(es * P * L.Npad);
        L.G = off;      off += align256(es * R * L.Npad);
        L.A2 = off;     off += align256(es * P * L.Npad);     // A~^2 and V: the masked ranking
        L.V = off;      off += align256(es * R * L.Npad);
        L.Tt = off;     off += align256(sizeof(float) * R);
        L.nvalid = off; off += align256(sizeof(int) * R);
        L.Rm = off;     off += align256(sizeof(float) * R);
        L.cand = off;   off += align256(sizeof(int) * kTopK * P);
        L.edge = off;   off += align256(P);
        // pixels left to the general rescore (those with a candidate not valid in every frame)
        L.wlist = off;  off += align256(sizeof(int) * (P + 1));
        // pixels whose minimum left the first 3x3: (pixel, window index, error, 0) each
        L.second = off; off += align256(4 * sizeof(int) * P);
    }
    L.total = off;
    return L;
}

__device__ __forceinline__ void split_neg_delta(double delta, int &k, float &f) {
    const double nd = -delta;
    double fl = floor(nd);
    float fr = (float)(nd - fl);
    if (fr >= 1.0f) {          // a fraction just below 1 rounded up in float32
        fr = 0.0f;
        fl += 1.0;
    }
    k = (int)fl;
    f = fr;
}

// |u| beyond this is rejected (status bit) so integer window arithmetic cannot overflow.
constexpr double kMaxCoord = 1.0e8;

// Launch-time configuration of the search kernel.
constexpr int kSearchSmemBudget = 200 * 1024;   // dynamic shared memory per CTA (bytes)

// Streaming multiprocessors of the current device (queried once per device and cached):
// grids that stride over their work are sized in multiples of it.
int device_sms();
// Count kernel launches made by this library (pxst_launch_count reports the running total).
void note_launch(int n = 1);

// Launch helpers implemented in the .cu files (all asynchronous on `stream`).
// fclass: the class of each frame (NULL: no classes; the scatter then forms the weights)
cudaError_t launch_prepare(const pxst_dims &d, const double *delta, WsHeader *hdr,
                           FrameShift *shifts, int *fclass, int reset_exact, cudaStream_t stream);
// dcls, fclass: the per-class weight images and the frames' classes (NULL: the scatter
// forms the reference weights itself, as the no-allocation entry point does)
cudaError_t launch_scatter(const pxst_dims &d, const float *frames, const float *W,
                           const uint8_t *mask, const double *u, const FrameShift *shifts,
                           WsHeader *hdr, double *num, double *den, float *dcls, const int *fclass,
                           cudaStream_t stream);
cudaError_t launch_normalise(const pxst_dims &d, const double *num, const double *den,
                             float *I_ref, float *w, cudaStream_t stream);
// span_y / span_x: range of the integer frame shifts (for sizing the shared-memory
// window; a smaller guess costs speed, never correctness). Negative = unknown.
cudaError_t launch_search(const pxst_dims &d, const pxst_options &o, const float *frames,
                          const float *W, const uint8_t *mask, const float *I_ref,
                          const float *w, const FrameShift *shifts, WsHeader *hdr,
                          int *exact_list, double *u, float *err_out, int span_y, int span_x,
                          cudaStream_t stream);
cudaError_t launch_rescore(const pxst_dims &d, const pxst_options &o, int ncand, const float *frames,
                           const float *W, const uint8_t *mask, const float *Rm, const int *nvalid,
                           const FrameShift *shifts, const int *cand, WsHeader *hdr, int *wlist, int *second,
                           double *u, float *err_out, cudaStream_t stream);
// precision forms (tensor.cu)
cudaError_t launch_tprep(const pxst_dims &d, int form, int Npad, const float *frames, const float *W,
                         const uint8_t *mask, void *At, WsHeader *hdr, cudaStream_t stream);
// A tiled TMA descriptor (rank 2-5, strides in bytes for dimensions 1..rank-1) through the
// driver entry point; 128-byte swizzle (the tensor-core operands) or none.
cudaError_t tmap_encode(CUtensorMap *map, CUtensorMapDataType dt, uint32_t rank, void *base,
                        const uint64_t *dims, const uint64_t *strides_bytes, const uint32_t *box,
                        bool swizzle128 = true);
cudaError_t launch_gtable(const pxst_dims &d, int form, int Npad, const float *I_ref, const float *w,
                          const FrameShift *shifts, const WsHeader *hdr, void *G, void *V, float *Tt, int *nvalid,
                          float *Rm, cudaStream_t stream);
cudaError_t launch_tsearch(const pxst_dims &d, const pxst_options &o, int Npad, const void *At, void *A2,
                           const void *G, const void *V, const uint8_t *mask, const float *W, const double *u,
                           const float *Tt, const int *nvalid, WsHeader *hdr, int *cand, uint8_t *edge,
                           int *tile_list, cudaStream_t stream);
cudaError_t launch_exact(const pxst_dims &d, const pxst_options &o, const float *frames,
                         const float *W, const uint8_t *mask, const float *I_ref,
                         const float *w, const FrameShift *shifts, WsHeader *hdr,
                         const int *exact_list, double *u, float *err_out, cudaStream_t stream);
int search_max_frames();
// figures of merit and the translation update (frames.cu)
cudaError_t launch_pixvar(const pxst_dims &d, const float *frames, const float *W, const uint8_t *mask,
                          const float *I_ref, const float *w, const double *u, const double *delta,
                          const FrameShift *shifts, float *var, PixSplit *split, WsHeader *hdr, cudaStream_t s);
cudaError_t launch_calc_error(const pxst_dims &d, const float *frames, const float *W, const uint8_t *mask,
                              const float *I_ref, const float *w, const double *u, const double *delta,
                              const FrameShift *shifts, const float *var, WsHeader *hdr, float *pixel_err,
                              double *frame_err, double *total, float *ref_err, double *num, double *den,
                              cudaStream_t s);
cudaError_t launch_update_translations(const pxst_dims &d, int Ty, int Tx, int quadratic, const float *frames,
                                       const float *W, const uint8_t *mask, const float *I_ref, const float *w,
                                       const double *u, const double *delta_in, const FrameShift *shifts,
                                       const float *var, const PixSplit *split, float *Rm, WsHeader *hdr,
                                       double *acc_sum, unsigned long long *acc_cnt, double *delta_out,
                                       double *err_out,
                                       cudaStream_t s);
cudaError_t launch_filter_map(const pxst_dims &d, double sigma, const uint8_t *mask, double *u, double *num,
                              double *den, cudaStream_t s);
cudaError_t launch_scale_map(const pxst_dims &d, double sy, double sx, const double *u, double *us, cudaStream_t s);
cudaError_t launch_contrast_sums(const pxst_dims &d, const float *I_ref, const float *w, double *acc, cudaStream_t s);
cudaError_t launch_contrast_final(int npairs, const double *acc, double *contrast, cudaStream_t s);
cudaError_t launch_frac_refine(const pxst_dims &d, int sub, const float *frames, const float *W, const uint8_t *mask,
                               const float *I_ref, const float *w, const FrameShift *shifts, double *u,
                               float *err_out, cudaStream_t s);
// integrate (integrate.cu): one cooperative launch of the whole conjugate-gradient solve
cudaError_t launch_integrate(const pxst_dims &d, const uint8_t *mask, double *u, int max_iter, double tol,
                             double *info, uint8_t *type, double *buf, unsigned *bar, WsHeader *hdr,
                             long long limit_ns, cudaStream_t s);
// learn (and cache) the integer shift span of a translation array outside any capture
void prime_shift_span(const pxst_dims &d, const double *delta, cudaStream_t s);
cudaError_t launch_refterms(const pxst_dims &d, const float *I_ref, const float *w,
                            const FrameShift *shifts, float *T, int32_t *n_valid,
                            cudaStream_t stream);

}  // namespace pxst

namespace pxst {

// Masked, renormalised bilinear read of I_ref (section "Sub-pixel interpolation"):
// corners (i0, j0), (i0, j0+1), (i0+1, j0), (i0+1, j0+1) with weights
// (1-fy)(1-fx), (1-fy)fx, fy(1-fx), fy fx; a corner counts if its weight is nonzero,
// it lies inside the grid and its coverage w is > 0. Returns false if none counts.
__device__ __forceinline__ bool gather_masked(const float *__restrict__ Iref,
                                              const float *__restrict__ w, int Ry, int Rx,
                                              int i0, int j0, float fy, float fx, float &R) {
    const float wt[4] = {(1.0f - fy) * (1.0f - fx), (1.0f - fy) * fx, fy * (1.0f - fx), fy * fx};
    float num = 0.0f, den = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int ii = i0 + (k >> 1), jj = j0 + (k & 1);
        if (wt[k] == 0.0f || ii < 0 || ii >= Ry || jj < 0 || jj >= Rx) continue;
        const size_t c = (size_t)ii * Rx + jj;
        if (!(__ldg(w + c) > 0.0f)) continue;
        num = fmaf(wt[k], __ldg(Iref + c), num);
        den += wt[k];
    }
    if (!(den > 0.0f)) return false;
    R = num / den;
    return true;
}

// R_n at (i0 + fy, j0 + fx) by the masked renormalised bilinear gather, read from the
// NaN-masked reference (the same arithmetic as gather_masked); false: frame not valid.
__device__ __forceinline__ bool gather_rm(const float *__restrict__ Rm, int Ry, int Rx, int i0, int j0,
                                          float fy, float fx, float &R) {
    if (fy == 0.0f && fx == 0.0f) {
        if (i0 < 0 || i0 >= Ry || j0 < 0 || j0 >= Rx) return false;
        R = __ldg(Rm + (size_t)i0 * Rx + j0);
        return R == R;
    }
    const float wt[4] = {(1.0f - fy) * (1.0f - fx), (1.0f - fy) * fx, fy * (1.0f - fx), fy * fx};
    float num = 0.0f, den = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int ii = i0 + (k >> 1), jj = j0 + (k & 1);
        if (wt[k] == 0.0f || ii < 0 || ii >= Ry || jj < 0 || jj >= Rx) continue;
        const float r = __ldg(Rm + (size_t)ii * Rx + jj);
        if (r != r) continue;
        num = fmaf(wt[k], r, num);
        den += wt[k];
    }
    if (!(den > 0.0f)) return false;
    R = num / den;
    return true;
}

// ------------------------------------------------------------------------------------
// 3x3 paraboloid refinement (end of section "Update pixel mapping"): least-squares fit
// of c0 + c1 a + c2 b + c3 a^2 + c4 ab + c5 b^2 at a, b in {-1, 0, 1}; stationary point
// of the fit if it is a convex bowl, otherwise a parabola per axis; shifts beyond one
// pixel are discarded per axis. f[3*(da+1) + (db+1)]; +inf marks a missing point.
__device__ inline void refine3x3(const float *f, double &da_out, double &db_out) {
    double v[9];
    bool complete = true;
    for (int k = 0; k < 9; ++k) {
        v[k] = (double)f[k];
        complete = complete && isfinite(v[k]);
    }
    double da = 0.0, db = 0.0;
    bool done = false;
    if (complete) {
        double s = 0, sa = 0, sb = 0, sab = 0, ra = 0, rb = 0;
        for (int ia = -1; ia <= 1; ++ia)
            for (int ib = -1; ib <= 1; ++ib) {
                const double t = v[(ia + 1) * 3 + (ib + 1)];
                s += t;
                sa += ia * t;
                sb += ib * t;
                sab += ia * ib * t;
                if (ia) ra += t;
                if (ib) rb += t;
            }
        const double g1 = sa / 6.0, g2 = sb / 6.0, h12 = sab / 4.0;
        const double h11 = (ra - 2.0 * (s - ra)) / 6.0, h22 = (rb - 2.0 * (s - rb)) / 6.0;
        const double det = 4.0 * h11 * h22 - h12 * h12;
        if (h11 > 0.0 && det > 0.0) {
            da = (h12 * g2 - 2.0 * h22 * g1) / det;
            db = (h12 * g1 - 2.0 * h11 * g2) / det;
            done = true;
        }
    }
    if (!done) {
        const double c = v[4];
        da = 0.0;
        if (isfinite(v[1]) && isfinite(v[7]) && isfinite(c)) {
            const double k = v[1] - 2.0 * c + v[7];
            if (k > 0.0) da = (v[1] - v[7]) / (2.0 * k);
        }
        db = 0.0;
        if (isfinite(v[3]) && isfinite(v[5]) && isfinite(c)) {
            const double k = v[3] - 2.0 * c + v[5];
            if (k > 0.0) db = (v[3] - v[5]) / (2.0 * k);
        }
    }
    if (!(fabs(da) <= 1.0)) da = 0.0;
    if (!(fabs(db) <= 1.0)) db = 0.0;
    da_out = da;
    db_out = db;
}

}  // namespace pxst
