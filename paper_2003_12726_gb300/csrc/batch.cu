// batch.cu -- the batched form: many scans of uneven size iterated by one graph launch,
// and the autotuner that picks each scan's tile shape by measurement.
//
// pxst_batch_plan captures every scan's main loop (pxst_iterate) into one CUDA graph:
// the scans are spread over parallel branches (largest estimated work first, each to the
// least loaded branch), so that small scans fill the GPU side by side; pxst_batch_run
// replays the graph with one cudaGraphLaunch. Everything a capture cannot do (reading the
// translations back for the shift span, timing tile shapes) happens at plan time.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "pxst_common.cuh"

struct pxst_batch_s {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<int> branch_of;      // branch each scan runs on
    int n_branches = 0;
};

namespace pxst {
namespace {

// tile shapes a form can take (0: automatic / the default shape)
std::vector<int> tile_candidates(int form) {
    if (form == PXST_FORM_FP32) {
        // tile heights (automatic, 1, 2, 4, 8 rows of 32 pixels) x strip lengths (automatic, 7, 9, 11)
        std::vector<int> v;
        for (int l : {0, 1, 2, 3})
            for (int ty : {0, 1, 2, 4, 8}) v.push_back(ty | (l << 4));
        return v;
    }
    return {0, 1, 2};
}

// one shape class: what a tile choice depends on
using TuneKey = std::tuple<int, int, int, int, int, int, int, int, int>;
TuneKey tune_key(const pxst_scan &s) {
    return TuneKey{s.dims.n_frames, s.dims.ny, s.dims.nx, s.dims.ref_ny, s.dims.ref_nx,
                   s.opts.win_y, s.opts.win_x, s.opts.form, s.opts.rescore_k};
}
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, float>> g_tuned;   // best tile, its time (ms)

double est_work(const pxst_scan &s) {
    const double cand = (2.0 * s.opts.win_y + 1) * (2.0 * s.opts.win_x + 1);
    const double evals = (double)s.dims.ny * s.dims.nx * cand * s.dims.n_frames;
    return s.opts.form == PXST_FORM_FP32 ? evals : 0.25 * evals;
}

}  // namespace
}  // namespace pxst

using namespace pxst;

extern "C" {

pxst_status pxst_autotune(const pxst_scan *scan, int32_t trials, void *stream, int32_t *best_tile,
                          float *best_ms) {
    if (!scan || !best_tile || trials < 1) return PXST_ERR_ARG;
    const pxst_scan &sc = *scan;
    if (!sc.u || !sc.I_ref || !sc.w || !sc.workspace) return PXST_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return PXST_ERR_ARG;
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tuned.find(tune_key(sc));
        if (it != g_tuned.end()) {
            *best_tile = it->second.first;
            if (best_ms) *best_ms = it->second.second;
            return PXST_OK;
        }
    }
    // the map is updated in place by every trial: keep the caller's and restore it after each
    const size_t P = (size_t)sc.dims.ny * sc.dims.nx, ubytes = 2 * P * sizeof(double);
    const WsLayout L = ws_layout(sc.dims, sc.opts.form);
    if (sc.ws_bytes < L.total) return PXST_ERR_NOMEM;
    double *u_save = reinterpret_cast<double *>(static_cast<char *>(sc.workspace) + L.u_save);
    if (cudaMemcpyAsync(u_save, sc.u, ubytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return PXST_ERR_CUDA;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return PXST_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return PXST_ERR_CUDA;
    }
    int best = 0;
    float best_t = INFINITY;
    pxst_status st = PXST_OK;
    for (int tile : tile_candidates(sc.opts.form)) {
        pxst_options o = sc.opts;
        o.tile = tile;
        std::vector<float> ts;
        for (int r = 0; r <= trials && st == PXST_OK; ++r) {        // r = 0: warm-up
            cudaMemcpyAsync(sc.u, u_save, ubytes, cudaMemcpyDeviceToDevice, s);
            cudaEventRecord(e0, s);
            st = pxst_update_pixel_map(&sc.dims, &o, sc.frames, sc.W, sc.mask, sc.I_ref, sc.w, sc.delta, sc.u,
                                       sc.err_out, sc.workspace, sc.ws_bytes, s);
            cudaEventRecord(e1, s);
            if (st != PXST_OK) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                st = PXST_ERR_CUDA;
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0) ts.push_back(ms);
        }
        if (st != PXST_OK) break;
        std::sort(ts.begin(), ts.end());
        const float med = ts[ts.size() / 2];
        if (med < best_t) {
            best_t = med;
            best = tile;
        }
    }
    cudaMemcpyAsync(sc.u, u_save, ubytes, cudaMemcpyDeviceToDevice, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && st == PXST_OK) st = PXST_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != PXST_OK) return st;
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tuned[tune_key(sc)] = {best, best_t};
    }
    *best_tile = best;
    if (best_ms) *best_ms = best_t;
    return PXST_OK;
}

pxst_status pxst_batch_plan(const pxst_scan *scans, int32_t n_scans, int32_t n_iter, int32_t n_branches,
                            int32_t autotune, void *stream, pxst_batch *out) {
    if (!scans || n_scans < 1 || n_iter < 0 || n_branches < 1 || n_branches > 64 || !out) return PXST_ERR_ARG;
    *out = nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<pxst_scan> sc(scans, scans + n_scans);
    // validate every scan up front (a zero-iteration pass checks the arguments and the
    // workspace, and primes the per-translation-array shift span outside the capture)
    for (auto &x : sc) {
        pxst_status st = pxst_iterate(&x.dims, &x.opts, 0, x.frames, x.W, x.mask, x.delta, x.u, x.I_ref, x.w,
                                      x.err_out, x.workspace, x.ws_bytes, s);
        if (st != PXST_OK) return st;
        // the FP32 search plans its window from the shift span: learn it now
        if (x.opts.form == PXST_FORM_FP32) prime_shift_span(x.dims, x.delta, s);
    }
    if (autotune) {
        for (auto &x : sc) {
            int32_t tile = 0;
            pxst_status st = pxst_autotune(&x, 3, s, &tile, nullptr);
            if (st != PXST_OK) return st;
            x.opts.tile = tile;
        }
    }
    auto *b = new (std::nothrow) pxst_batch_s();
    if (!b) return PXST_ERR_NOMEM;
    const int nb = std::min<int>(n_branches, n_scans);
    b->n_branches = nb;
    b->branch_of.assign(n_scans, 0);
    // largest work first, each to the least loaded branch
    std::vector<int> order(n_scans);
    for (int i = 0; i < n_scans; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return est_work(sc[a]) > est_work(sc[c]); });
    std::vector<double> load(nb, 0.0);
    for (int i : order) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        b->branch_of[i] = k;
        load[k] += est_work(sc[i]);
    }
    // capture: origin stream -> nb branch streams -> origin
    std::vector<cudaStream_t> br(nb, nullptr);
    std::vector<cudaEvent_t> done(nb, nullptr);
    cudaStream_t origin = nullptr;
    cudaEvent_t fork = nullptr;
    pxst_status st = PXST_OK;
    auto fail = [&](pxst_status e) {
        if (st == PXST_OK) st = e;
    };
    if (cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking) != cudaSuccess) fail(PXST_ERR_CUDA);
    for (int k = 0; k < nb && st == PXST_OK; ++k) {
        if (cudaStreamCreateWithFlags(&br[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&done[k], cudaEventDisableTiming) != cudaSuccess)
            fail(PXST_ERR_CUDA);
    }
    if (st == PXST_OK && cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess) fail(PXST_ERR_CUDA);
    // the plan's own work (validation, tuning) is ordered before the capture
    if (st == PXST_OK && cudaStreamSynchronize(s) != cudaSuccess) fail(PXST_ERR_CUDA);
    if (st == PXST_OK) {
        if (cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            fail(PXST_ERR_CUDA);
        } else {
            cudaEventRecord(fork, origin);
            for (int k = 0; k < nb; ++k) cudaStreamWaitEvent(br[k], fork, 0);
            for (int i : order) {
                const pxst_scan &x = sc[i];
                const pxst_status e = pxst_iterate(&x.dims, &x.opts, n_iter, x.frames, x.W, x.mask, x.delta, x.u,
                                                   x.I_ref, x.w, x.err_out, x.workspace, x.ws_bytes,
                                                   br[b->branch_of[i]]);
                if (e != PXST_OK) fail(e);
            }
            for (int k = 0; k < nb; ++k) {
                cudaEventRecord(done[k], br[k]);
                cudaStreamWaitEvent(origin, done[k], 0);
            }
            if (cudaStreamEndCapture(origin, &b->graph) != cudaSuccess) fail(PXST_ERR_CUDA);
            if (st == PXST_OK && cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) fail(PXST_ERR_CUDA);
        }
    }
    for (int k = 0; k < nb; ++k) {
        if (done[k]) cudaEventDestroy(done[k]);
        if (br[k]) cudaStreamDestroy(br[k]);
    }
    if (fork) cudaEventDestroy(fork);
    if (origin) cudaStreamDestroy(origin);
    if (st != PXST_OK) {
        cudaGetLastError();
        pxst_batch_destroy(b);
        return st;
    }
    *out = b;
    return PXST_OK;
}

pxst_status pxst_batch_run(pxst_batch batch, void *stream) {
    if (!batch || !batch->exec) return PXST_ERR_ARG;
    return cudaGraphLaunch(batch->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? PXST_OK
                                                                                            : PXST_ERR_CUDA;
}

int32_t pxst_batch_branch(pxst_batch batch, int32_t scan) {
    if (!batch || scan < 0 || scan >= (int32_t)batch->branch_of.size()) return -1;
    return batch->branch_of[scan];
}

void pxst_batch_destroy(pxst_batch batch) {
    if (!batch) return;
    if (batch->exec) cudaGraphExecDestroy(batch->exec);
    if (batch->graph) cudaGraphDestroy(batch->graph);
    delete batch;
}

}  // extern "C"
