// api.cu -- the extern "C" boundary of libpxst.so: argument checks, workspace carving,
// launch sequencing, device status, and per-kernel event timing.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "pxst_common.cuh"

using namespace pxst;

namespace {

bool dims_ok(const pxst_dims *d) {
    if (!d) return false;
    if (d->n_frames < 1 || d->ny < 1 || d->nx < 1 || d->ref_ny < 1 || d->ref_nx < 1) return false;
    if ((long long)d->ny * d->nx >= (1LL << 31)) return false;           // int pixel indices
    if ((long long)d->ref_ny * d->ref_nx >= (1LL << 31)) return false;   // int window math
    return true;
}

bool opts_ok(const pxst_options *o) {
    if (!o) return false;
    if (o->win_y < 0 || o->win_x < 0 || o->win_y > 4096 || o->win_x > 4096) return false;
    if ((long long)(2 * o->win_y + 1) * (2 * o->win_x + 1) >= (1LL << 30)) return false;
    if (o->quadratic != 0 && o->quadratic != 1) return false;
    if (o->form != PXST_FORM_FP32 && o->form != PXST_FORM_BF16 && o->form != PXST_FORM_TF32) return false;
    if (o->rescore_k != 0 && o->rescore_k != 4 && o->rescore_k != 8) return false;
    if (o->timeout_ns < 0) return false;
    const int ty = o->tile & 15, ls = o->tile >> 4;
    if (o->form == PXST_FORM_FP32 ? (o->tile < 0 || ls > 3 || (ty != 0 && ty != 1 && ty != 2 && ty != 4 && ty != 8))
                                  : (o->tile < 0 || o->tile > 2))
        return false;
    return true;
}

struct Ws {
    WsHeader *hdr;
    float *var_px;
    PixSplit *usplit;
    double *u_save, *filt_den;
    double *tacc_sum, *delta_tmp;
    unsigned long long *tacc_cnt;
    FrameShift *shifts;
    int *exact_list;
    double *num, *den;
    int *fclass;
    float *dcls;
    void *At, *G, *A2, *V;
    float *Tt, *Rm;
    int *nvalid, *cand, *wlist, *second;
    uint8_t *edge;
    int Npad;
};

pxst_status carve(const pxst_dims &d, int form, void *workspace, size_t ws_bytes, Ws &w) {
    if (!workspace) return PXST_ERR_ARG;
    if (((uintptr_t)workspace & 255) != 0) return PXST_ERR_ARG;
    const WsLayout L = ws_layout(d, form);
    if (ws_bytes < L.total) return PXST_ERR_NOMEM;
    char *b = static_cast<char *>(workspace);
    w.hdr = reinterpret_cast<WsHeader *>(b + L.header);
    w.var_px = reinterpret_cast<float *>(b + L.var_px);
    w.usplit = reinterpret_cast<PixSplit *>(b + L.usplit);
    w.u_save = reinterpret_cast<double *>(b + L.u_save);
    w.filt_den = reinterpret_cast<double *>(b + L.filt_den);
    w.tacc_sum = reinterpret_cast<double *>(b + L.tacc_sum);
    w.tacc_cnt = reinterpret_cast<unsigned long long *>(b + L.tacc_cnt);
    w.delta_tmp = reinterpret_cast<double *>(b + L.delta_tmp);
    w.shifts = reinterpret_cast<FrameShift *>(b + L.shifts);
    w.exact_list = reinterpret_cast<int *>(b + L.exact_list);
    w.num = reinterpret_cast<double *>(b + L.num);
    w.den = reinterpret_cast<double *>(b + L.den);
    w.fclass = reinterpret_cast<int *>(b + L.fclass);
    w.dcls = reinterpret_cast<float *>(b + L.dcls);
    w.At = b + L.At;
    w.G = b + L.G;
    w.A2 = b + L.A2;
    w.V = b + L.V;
    w.Tt = reinterpret_cast<float *>(b + L.Tt);
    w.nvalid = reinterpret_cast<int *>(b + L.nvalid);
    w.Rm = reinterpret_cast<float *>(b + L.Rm);
    w.cand = reinterpret_cast<int *>(b + L.cand);
    w.edge = reinterpret_cast<uint8_t *>(b + L.edge);
    w.wlist = reinterpret_cast<int *>(b + L.wlist);
    w.second = reinterpret_cast<int *>(b + L.second);
    w.Npad = L.Npad;
    return PXST_OK;
}

// ---- per-kernel timing -------------------------------------------------------------
struct Rec {
    int k;
    cudaEvent_t a, b;
};
std::mutex g_tmu;
bool g_timing = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
constexpr size_t kMaxRecs = 1 << 16;

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct Timed {
    cudaEvent_t a = nullptr, b = nullptr;
    int k;
    cudaStream_t s;
    Timed(int kernel, cudaStream_t st) : k(kernel), s(st) {
        std::lock_guard<std::mutex> g(g_tmu);
        if (g_timing && g_recs.size() < kMaxRecs) {
            // a stream being captured into a graph records no timing events
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
            a = take_event();
            b = take_event();
            cudaEventRecord(a, s);
        }
    }
    ~Timed() {
        if (!a) return;
        std::lock_guard<std::mutex> g(g_tmu);
        cudaEventRecord(b, s);
        g_recs.push_back({k, a, b});
    }
};

// ---- integer frame-shift span per translation array -----------------------------------
// The search kernel's shared-memory window spans the range of the integer parts of
// -Delta; the host learns it once per (device, translation pointer, frame count) with a
// synchronous read of Delta, and plans the launch with it. During stream capture no read
// is possible: an unknown span plans for the largest window.
struct SpanKey {
    int dev;
    const double *delta;
    int n;
    bool operator==(const SpanKey &o) const { return dev == o.dev && delta == o.delta && n == o.n; }
};
std::mutex g_smu;
std::vector<std::pair<SpanKey, std::pair<int, int>>> g_spans;

void shift_span(const pxst_dims &d, const double *delta, cudaStream_t s, int &sy, int &sx) {
    sy = sx = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    const SpanKey key{dev, delta, d.n_frames};
    {
        std::lock_guard<std::mutex> g(g_smu);
        for (auto &e : g_spans)
            if (e.first == key) {
                sy = e.second.first;
                sx = e.second.second;
                return;
            }
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    std::vector<double> h((size_t)2 * d.n_frames);
    if (cudaMemcpyAsync(h.data(), delta, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return;
    double mn[2] = {1e300, 1e300}, mx[2] = {-1e300, -1e300};
    for (int n = 0; n < d.n_frames; ++n)
        for (int a = 0; a < 2; ++a) {
            const double k = std::floor(-h[2 * n + a]);
            mn[a] = std::min(mn[a], k);
            mx[a] = std::max(mx[a], k);
        }
    sy = (int)std::min(mx[0] - mn[0] + 1, 1e6);     // +1: a fraction rounding up to 1
    sx = (int)std::min(mx[1] - mn[1] + 1, 1e6);
    std::lock_guard<std::mutex> g(g_smu);
    if (g_spans.size() > 256) g_spans.clear();
    g_spans.push_back({key, {sy, sx}});
}

pxst_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return PXST_OK;
    std::fprintf(stderr, "pxst: CUDA error %s\n", cudaGetErrorString(e));
    return PXST_ERR_CUDA;
}

#define PXST_TRY(expr)                                   \
    do {                                                 \
        cudaError_t _e = (expr);                         \
        if (_e != cudaSuccess) return cuda_status(_e);   \
    } while (0)

pxst_status run_prepare(const pxst_dims &d, const double *delta, Ws &w, cudaStream_t s) {
    Timed t(PXST_K_PREPARE, s);
    PXST_TRY(launch_prepare(d, delta, w.hdr, w.shifts, w.fclass, 1, s));
    return PXST_OK;
}

pxst_status run_omap(const pxst_dims &d, const float *frames, const float *W,
                     const uint8_t *mask, const double *u, float *I_ref, float *wout, Ws &w,
                     cudaStream_t s) {
    {
        Timed t(PXST_K_SCATTER, s);
        PXST_TRY(launch_scatter(d, frames, W, mask, u, w.shifts, w.hdr, w.num, w.den, w.dcls, w.fclass, s));
    }
    {
        Timed t(PXST_K_NORMALISE, s);
        PXST_TRY(launch_normalise(d, w.num, w.den, I_ref, wout, s));
    }
    return PXST_OK;
}

pxst_status run_update(const pxst_dims &d, const pxst_options &o, const float *frames,
                       const float *W, const uint8_t *mask, const float *I_ref, const float *wref,
                       const double *delta, double *u, float *err_out, Ws &w, cudaStream_t s,
                       bool operands_ready = false) {
    PXST_TRY(cudaMemsetAsync(&w.hdr->n_exact, 0, 2 * sizeof(int), s));   // n_exact, n_exact_cta
    if (o.form != PXST_FORM_FP32) {
        // tensor-core ranking of every candidate that is valid in every frame, the masked
        // ranking of the pixels with candidates that are not, then exact FP32 errors of the
        // best few per pixel and of the 3x3 about the minimum
        if (!operands_ready) {
            Timed t(PXST_K_TPREP, s);
            PXST_TRY(launch_tprep(d, o.form, w.Npad, frames, W, mask, w.At, w.hdr, s));
        }
        {
            Timed t(PXST_K_GTABLE, s);
            PXST_TRY(launch_gtable(d, o.form, w.Npad, I_ref, wref, w.shifts, w.hdr, w.G, w.V, w.Tt, w.nvalid, w.Rm, s));
        }
        {
            Timed t(PXST_K_TSEARCH, s);
            PXST_TRY(cudaMemsetAsync(&w.hdr->n_edge_tiles, 0, sizeof(int), s));
            PXST_TRY(launch_tsearch(d, o, w.Npad, w.At, w.A2, w.G, w.V, mask, W, u, w.Tt, w.nvalid, w.hdr,
                                    w.cand, w.edge, w.exact_list, s));
        }
        // few frames make the reduced-precision ranking noisier: rescore more of it
        const int rk = o.rescore_k ? o.rescore_k : (d.n_frames < 128 ? 8 : 4);
        Timed t(PXST_K_RESCORE, s);
        PXST_TRY(launch_rescore(d, o, rk, frames, W, mask, w.Rm, w.nvalid, w.shifts, w.cand, w.hdr, w.wlist, w.second, u, err_out, s));
    } else if (d.n_frames <= search_max_frames()) {
        int sy, sx;
        shift_span(d, delta, s, sy, sx);
        {
            Timed t(PXST_K_SEARCH, s);
            PXST_TRY(launch_search(d, o, frames, W, mask, I_ref, wref, w.shifts, w.hdr,
                                   w.exact_list, u, err_out, sy, sx, s));
        }
        Timed t(PXST_K_EXACT, s);
        PXST_TRY(launch_exact(d, o, frames, W, mask, I_ref, wref, w.shifts, w.hdr, w.exact_list,
                              u, err_out, s));
    } else {
        // too many frames to stage a tile on chip: every pixel takes the exact path
        Timed t(PXST_K_EXACT, s);
        PXST_TRY(launch_exact(d, o, frames, W, mask, I_ref, wref, w.shifts, w.hdr, nullptr, u,
                              err_out, s));
    }
    return PXST_OK;
}

// ---- device properties and the launch counter -------------------------------------------
constexpr int kMaxDev = 64;
std::atomic<int> g_sms[kMaxDev];
std::atomic<long long> g_launches{0};

}  // namespace

int pxst::device_sms() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 148;
    int n = g_sms[dev].load(std::memory_order_relaxed);
    if (n > 0) return n;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 148;
    g_sms[dev].store(n, std::memory_order_relaxed);
    return n;
}

void pxst::note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void pxst::prime_shift_span(const pxst_dims &d, const double *delta, cudaStream_t s) {
    int sy, sx;
    shift_span(d, delta, s, sy, sx);
}

extern "C" {

size_t pxst_workspace_size(const pxst_dims *dims, const pxst_options *opts) {
    if (!dims_ok(dims)) return 0;
    return ws_layout(*dims, opts ? opts->form : PXST_FORM_FP32).total;
}

pxst_status pxst_make_object_map(const pxst_dims *dims, const float *frames, const float *W,
                                 const uint8_t *mask, const double *u, const double *delta,
                                 float *I_ref, float *w, void *workspace, size_t ws_bytes,
                                 void *stream) {
    if (!dims_ok(dims)) return PXST_ERR_SHAPE;
    if (!frames || !W || !mask || !u || !delta || !I_ref || !w) return PXST_ERR_ARG;
    Ws ws;
    pxst_status st = carve(*dims, PXST_FORM_FP32, workspace, ws_bytes, ws);
    if (st != PXST_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = run_prepare(*dims, delta, ws, s);
    if (st != PXST_OK) return st;
    return run_omap(*dims, frames, W, mask, u, I_ref, w, ws, s);
}

pxst_status pxst_update_pixel_map(const pxst_dims *dims, const pxst_options *opts,
                                  const float *frames, const float *W, const uint8_t *mask,
                                  const float *I_ref, const float *w, const double *delta,
                                  double *u_inout, float *err_out, void *workspace,
                                  size_t ws_bytes, void *stream) {
    if (!dims_ok(dims)) return PXST_ERR_SHAPE;
    if (!opts_ok(opts)) return PXST_ERR_ARG;
    if (!frames || !W || !mask || !I_ref || !w || !delta || !u_inout) return PXST_ERR_ARG;
    Ws ws;
    pxst_status st = carve(*dims, opts->form, workspace, ws_bytes, ws);
    if (st != PXST_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = run_prepare(*dims, delta, ws, s);
    if (st != PXST_OK) return st;
    return run_update(*dims, *opts, frames, W, mask, I_ref, w, delta, u_inout, err_out, ws, s);
}

pxst_status pxst_iterate(const pxst_dims *dims, const pxst_options *opts, int32_t n_iter,
                         const float *frames, const float *W, const uint8_t *mask,
                         const double *delta, double *u_inout, float *I_ref, float *w,
                         float *err_out, void *workspace, size_t ws_bytes, void *stream) {
    if (!dims_ok(dims)) return PXST_ERR_SHAPE;
    if (!opts_ok(opts) || n_iter < 0) return PXST_ERR_ARG;
    if (!frames || !W || !mask || !delta || !u_inout || !I_ref || !w) return PXST_ERR_ARG;
    Ws ws;
    pxst_status st = carve(*dims, opts->form, workspace, ws_bytes, ws);
    if (st != PXST_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = run_prepare(*dims, delta, ws, s);
    if (st != PXST_OK) return st;
    if (opts->form != PXST_FORM_FP32 && n_iter > 0) {
        Timed t(PXST_K_TPREP, s);
        PXST_TRY(launch_tprep(*dims, opts->form, ws.Npad, frames, W, mask, ws.At, ws.hdr, s));
    }
    for (int it = 0; it < n_iter; ++it) {
        st = run_omap(*dims, frames, W, mask, u_inout, I_ref, w, ws, s);
        if (st != PXST_OK) return st;
        st = run_update(*dims, *opts, frames, W, mask, I_ref, w, delta, u_inout, err_out, ws, s, true);
        if (st != PXST_OK) return st;
    }
    return PXST_OK;
}

pxst_status pxst_calc_error(const pxst_dims *dims, const float *frames, const float *W, const uint8_t *mask,
                            const float *I_ref, const float *w, const double *u, const double *delta,
                            float *pixel_err, double *frame_err, double *total_err, float *ref_err,
                            void *workspace, size_t ws_bytes, void *stream) {
    if (!dims_ok(dims)) return PXST_ERR_SHAPE;
    if (!frames || !W || !mask || !I_ref || !w || !u || !delta) return PXST_ERR_ARG;
    Ws ws;
    pxst_status st = carve(*dims, PXST_FORM_FP32, workspace, ws_bytes, ws);
    if (st != PXST_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = run_prepare(*dims, delta, ws, s);
    if (st != PXST_OK) return st;
    Timed t(PXST_K_ERROR, s);
    PXST_TRY(launch_pixvar(*dims, frames, W, mask, I_ref, w, u, delta, ws.shifts, ws.var_px, nullptr, ws.hdr, s));
    PXST_TRY(launch_calc_error(*dims, frames, W, mask, I_ref, w, u, delta, ws.shifts, ws.var_px, ws.hdr, pixel_err,
                               frame_err, total_err, ref_err, ws.num, ws.den, s));
    return PXST_OK;
}

pxst_status pxst_update_translations(const pxst_dims *dims, int32_t win_y, int32_t win_x, int32_t quadratic,
                                     const float *frames, const float *W, const uint8_t *mask,
                                     const float *I_ref, const float *w, const double *u, double *delta_inout,
                                     double *frame_err, void *workspace, size_t ws_bytes, void *stream) {
    if (!dims_ok(dims)) return PXST_ERR_SHAPE;
    if (win_y < 0 || win_x < 0 || win_y > 8 || win_x > 8 || (quadratic != 0 && quadratic != 1)) return PXST_ERR_ARG;
    if (!frames || !W || !mask || !I_ref || !w || !u || !delta_inout) return PXST_ERR_ARG;
    Ws ws;
    pxst_status st = carve(*dims, PXST_FORM_FP32, workspace, ws_bytes, ws);
    if (st != PXST_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = run_prepare(*dims, delta_inout, ws, s);
    if (st != PXST_OK) return st;
    Timed t(PXST_K_TRANS, s);
    PXST_TRY(launch_pixvar(*dims, frames, W, mask, I_ref, w, u, delta_inout, ws.shifts, ws.var_px, ws.usplit, ws.hdr,
                           s));
    // every frame's shifts are scored against the translations as they were on entry; the
    // NaN-marked reference goes to the make_object_map accumulators, unused by this call
    PXST_TRY(launch_update_translations(*dims, win_y, win_x, quadratic, frames, W, mask, I_ref, w, u, delta_inout,
                                        ws.shifts, ws.var_px, ws.usplit, reinterpret_cast<float *>(ws.num), ws.hdr,
                                        ws.tacc_sum, ws.tacc_cnt, ws.delta_tmp,
                                        frame_err, s));
    PXST_TRY(cudaMemcpyAsync(delta_inout, ws.delta_tmp, sizeof(double) * 2 * dims->n_frames,
                             cudaMemcpyDeviceToDevice, s));
    return PXST_OK;
}

pxst_status pxst_update_pixel_map_fractional(const pxst_dims *dims, const pxst_options *opts, int32_t sub,
                                             const float *frames, const float *W, const uint8_t *mask,
                                             const float *I_ref, const float *w, const double *delta,
                                             double *u_inout, float *err_out, void *workspace, size_t ws_bytes,
                                             void *stream) {
    if (!dims_ok(dims)) return PXST_ERR_SHAPE;
    if (!opts_ok(opts) || sub < 1 || sub > 8) return PXST_ERR_ARG;
    if (!frames || !W || !mask || !I_ref || !w || !delta || !u_inout) return PXST_ERR_ARG;
    Ws ws;
    pxst_status st = carve(*dims, opts->form, workspace, ws_bytes, ws);
    if (st != PXST_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = run_prepare(*dims, delta, ws, s);
    if (st != PXST_OK) return st;
    pxst_options o = *opts;
    o.quadratic = 0;                          // the integer minimum, then the fractional grid about it
    st = run_update(*dims, o, frames, W, mask, I_ref, w, delta, u_inout, err_out, ws, s);
    if (st != PXST_OK) return st;
    Timed t(PXST_K_FRAC, s);
    PXST_TRY(launch_frac_refine(*dims, sub, frames, W, mask, I_ref, w, ws.shifts, u_inout, err_out, s));
    return PXST_OK;
}

pxst_status pxst_defocus_sweep(const pxst_dims *dims, const float *frames, const float *W, const uint8_t *mask,
                               const double *u, const double *delta, int32_t n_sy, const double *sy, int32_t n_sx,
                               const double *sx, double *contrast, float *I_ref, float *w, void *workspace,
                               size_t ws_bytes, void *stream) {
    if (!dims_ok(dims)) return PXST_ERR_SHAPE;
    if (!frames || !W || !mask || !u || !delta || !sy || !sx || !contrast || !I_ref || !w) return PXST_ERR_ARG;
    if (n_sy < 1 || n_sx < 1 || n_sy * n_sx > 64) return PXST_ERR_ARG;
    for (int k = 0; k < n_sy; ++k)
        if (!(sy[k] > 0.0 && sy[k] < 100.0)) return PXST_ERR_ARG;
    for (int k = 0; k < n_sx; ++k)
        if (!(sx[k] > 0.0 && sx[k] < 100.0)) return PXST_ERR_ARG;
    Ws ws;
    pxst_status st = carve(*dims, PXST_FORM_FP32, workspace, ws_bytes, ws);
    if (st != PXST_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = run_prepare(*dims, delta, ws, s);
    if (st != PXST_OK) return st;
    const int npairs = n_sy * n_sx;
    double *acc = ws.tacc_sum;                        // 3 sums per pair (>= kTransMax doubles)
    PXST_TRY(cudaMemsetAsync(acc, 0, sizeof(double) * 3 * npairs, s));
    Timed t(PXST_K_DEFOCUS, s);
    for (int ky = 0; ky < n_sy; ++ky)
        for (int kx = 0; kx < n_sx; ++kx) {
            PXST_TRY(launch_scale_map(*dims, sy[ky], sx[kx], u, ws.u_save, s));
            st = run_omap(*dims, frames, W, mask, ws.u_save, I_ref, w, ws, s);
            if (st != PXST_OK) return st;
            PXST_TRY(launch_contrast_sums(*dims, I_ref, w, acc + 3 * (ky * n_sx + kx), s));
        }
    PXST_TRY(launch_contrast_final(npairs, acc, contrast, s));
    return PXST_OK;
}

pxst_status pxst_integrate_map(const pxst_dims *dims, const uint8_t *mask, double *u_inout, int32_t max_iter,
                               double tol, int64_t timeout_ns, double *info_out, void *workspace, size_t ws_bytes,
                               void *stream) {
    if (!dims_ok(dims)) return PXST_ERR_SHAPE;
    if (!mask || !u_inout || max_iter < 0 || !(tol >= 0.0) || timeout_ns < 0) return PXST_ERR_ARG;
    if (!workspace || ((uintptr_t)workspace & 255) != 0) return PXST_ERR_ARG;
    const WsLayout L = ws_layout(*dims, PXST_FORM_FP32);
    if (ws_bytes < L.total) return PXST_ERR_NOMEM;
    char *b = static_cast<char *>(workspace);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Timed t(PXST_K_INTEGRATE, s);
    PXST_TRY(launch_integrate(*dims, mask, u_inout, max_iter, tol, info_out, reinterpret_cast<uint8_t *>(b + L.integ_type),
                              reinterpret_cast<double *>(b + L.integ_buf), reinterpret_cast<unsigned *>(b + L.integ_bar),
                              reinterpret_cast<WsHeader *>(b + L.header), timeout_ns, s));
    return PXST_OK;
}

pxst_status pxst_filter_map(const pxst_dims *dims, double sigma, const uint8_t *mask, double *u_inout,
                            void *workspace, size_t ws_bytes, void *stream) {
    if (!dims_ok(dims)) return PXST_ERR_SHAPE;
    if (!mask || !u_inout || !(sigma >= 0.0) || sigma > 1024.0) return PXST_ERR_ARG;
    Ws ws;
    pxst_status st = carve(*dims, PXST_FORM_FP32, workspace, ws_bytes, ws);
    if (st != PXST_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Timed t(PXST_K_FILTER, s);
    PXST_TRY(launch_filter_map(*dims, sigma, mask, u_inout, ws.u_save, ws.filt_den, s));
    return PXST_OK;
}

pxst_status pxst_reference_terms(const pxst_dims *dims, const float *I_ref, const float *w,
                                 const double *delta, float *T, int32_t *n_valid,
                                 void *workspace, size_t ws_bytes, void *stream) {
    if (!dims_ok(dims)) return PXST_ERR_SHAPE;
    if (!I_ref || !w || !delta || !T || !n_valid) return PXST_ERR_ARG;
    Ws ws;
    pxst_status st = carve(*dims, PXST_FORM_FP32, workspace, ws_bytes, ws);
    if (st != PXST_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = run_prepare(*dims, delta, ws, s);
    if (st != PXST_OK) return st;
    Timed t(PXST_K_REFTERMS, s);
    PXST_TRY(launch_refterms(*dims, I_ref, w, ws.shifts, T, n_valid, s));
    return PXST_OK;
}

pxst_status pxst_get_status(void *workspace, void *stream, int32_t *bits_out) {
    if (!workspace) return PXST_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    WsHeader *hdr = static_cast<WsHeader *>(workspace);
    int bits = 0;
    PXST_TRY(cudaStreamSynchronize(s));
    PXST_TRY(cudaMemcpy(&bits, &hdr->status, sizeof(int), cudaMemcpyDeviceToHost));
    PXST_TRY(cudaMemset(&hdr->status, 0, sizeof(int)));
    if (bits_out) *bits_out = bits;
    if (bits & PXST_DEV_TIMEOUT) return PXST_ERR_TIMEOUT;
    if (bits & (PXST_DEV_NONFINITE_U | PXST_DEV_U_RANGE)) return PXST_ERR_RANGE;
    if (bits & PXST_DEV_BAD_INPUT) return PXST_ERR_INPUT;
    return PXST_OK;
}

pxst_status pxst_last_exact_count(void *workspace, void *stream, int64_t *count_out) {
    if (!workspace || !count_out) return PXST_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    WsHeader *hdr = static_cast<WsHeader *>(workspace);
    int n[2] = {0, 0};
    PXST_TRY(cudaStreamSynchronize(s));
    PXST_TRY(cudaMemcpy(n, &hdr->n_exact, 2 * sizeof(int), cudaMemcpyDeviceToHost));
    *count_out = (int64_t)n[0] + n[1];
    return PXST_OK;
}

pxst_status pxst_timing_enable(int32_t enable) {
    std::lock_guard<std::mutex> g(g_tmu);
    for (auto &r : g_recs) {
        cudaEventSynchronize(r.b);
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    g_timing = enable != 0;
    return PXST_OK;
}

pxst_status pxst_timing_read(int64_t *launches, double *total_ms, int32_t n_kernels) {
    if (!launches || !total_ms || n_kernels < 0) return PXST_ERR_ARG;
    std::lock_guard<std::mutex> g(g_tmu);
    for (int k = 0; k < n_kernels; ++k) {
        launches[k] = 0;
        total_ms[k] = 0.0;
    }
    for (auto &r : g_recs) {
        if (r.k >= n_kernels) continue;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) return cuda_status(e);
        float ms = 0.0f;
        e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) return cuda_status(e);
        launches[r.k] += 1;
        total_ms[r.k] += ms;
    }
    return PXST_OK;
}

const char *pxst_kernel_name(int32_t k) {
    switch (k) {
        case PXST_K_PREPARE: return "prepare";
        case PXST_K_SCATTER: return "omap_scatter";
        case PXST_K_NORMALISE: return "omap_normalise";
        case PXST_K_SEARCH: return "upm_search";
        case PXST_K_EXACT: return "upm_exact";
        case PXST_K_REFTERMS: return "reference_terms";
        case PXST_K_TPREP: return "tensor_prep";
        case PXST_K_GTABLE: return "tensor_gtable";
        case PXST_K_TSEARCH: return "tensor_search";
        case PXST_K_RESCORE: return "upm_rescore";
        case PXST_K_ERROR: return "calc_error";
        case PXST_K_TRANS: return "update_translations";
        case PXST_K_FILTER: return "filter_map";
        case PXST_K_FRAC: return "upm_fractional";
        case PXST_K_DEFOCUS: return "defocus_sweep";
        case PXST_K_INTEGRATE: return "integrate";
        default: return "?";
    }
}

const char *pxst_status_string(pxst_status s) {
    switch (s) {
        case PXST_OK: return "ok";
        case PXST_ERR_ARG: return "invalid argument";
        case PXST_ERR_SHAPE: return "invalid or unsupported dimensions";
        case PXST_ERR_RANGE: return "non-finite or out-of-range pixel map on the device";
        case PXST_ERR_CUDA: return "CUDA runtime error";
        case PXST_ERR_NOMEM: return "workspace too small";
        case PXST_ERR_TIMEOUT: return "device-side wait timed out";
        case PXST_ERR_INPUT: return "non-finite frame value or non-positive whitefield at a good pixel";
        default: return "unknown status";
    }
}

pxst_status pxst_launch_count(int64_t *count_out) {
    if (!count_out) return PXST_ERR_ARG;
    *count_out = g_launches.load(std::memory_order_relaxed);
    return PXST_OK;
}

const char *pxst_version(void) { return "pxst 0.1 (sm_103a)"; }

}  // extern "C"
