// upm.cu -- update_pixel_map ("Update pixel mapping", section "Main loop") on sm_103a.
//
// Fast path (k_search): one CTA per tile of TY x 32 pixels. Each pixel has TPP threads
// that share its candidate strips (one candidate row, L consecutive columns per strip).
//   * the tile's frames, all N of them, are staged once in shared memory;
//   * the tile's reference window (every candidate of every pixel of the tile, widened
//     by the range of integer frame shifts and one bilinear corner) is staged once, with
//     uncovered or off-grid reference pixels stored as NaN;
//   * per candidate and frame: R = bilinear read of the window at the frame's shift
//     (a plain load for integer translations, a lerp for fractional ones, selected per
//     frame), d = I - W R, err += d^2: two FP32 FMAs per evaluation;
//   * a NaN error means some frame read an invalid reference pixel, where the paper's
//     rule drops that corner (or the whole frame) instead; only such strips are evaluated
//     again with the rule applied per frame. Valid strips need no per-frame check, so the
//     check costs nothing in the inner loop;
//   * the argmin (first minimum in row-major order) is reduced in registers, then over
//     the TPP threads; the 3x3 about it is re-evaluated and fitted in FP64.
// Global path (k_exact): one warp per listed pixel, candidates over lanes, per-frame
// masked renormalised reads from global memory, lexicographic warp argmin, FP64 fit.
// It serves tiles whose reference window does not fit in shared memory and scans with
// too many frames to stage.
#include <climits>
#include <cmath>

#include "pxst_common.cuh"

namespace pxst {
namespace {

struct SearchArgs {
    int N, ny, nx, Ry, Rx, Sy, Sx, quadratic, nstrips, nitems, win_cap;
    const float *frames, *W;
    const uint8_t *mask;
    const float *Iref, *w;
    const FrameShift *shifts;
    WsHeader *hdr;
    int *exact_list;
    double *u;
    float *err_out;
};

// ------------------------------------------------------------------------------------
// 3x3 paraboloid refinement (end of section "Update pixel mapping"): least-squares fit
// of c0 + c1 a + c2 b + c3 a^2 + c4 ab + c5 b^2 at a, b in {-1, 0, 1}; stationary point
// of the fit if it is a convex bowl, otherwise a parabola per axis; shifts beyond one
// pixel are discarded per axis. f[3*(da+1) + (db+1)]; +inf marks a missing point.
__device__ void refine3x3(const float *f, double &da_out, double &db_out) {
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

// ------------------------------------------------------------------------------------
// One strip of L candidates (same row, consecutive columns) over all frames.
// win points at the window row/column of the strip's first candidate for a zero shift.
template <int L>
__device__ __forceinline__ void eval_strip(const float *__restrict__ fr, int TP, int p,
                                           const FrameShift *__restrict__ sh, int N,
                                           const float *__restrict__ win, int WS, float Wv,
                                           float (&acc)[L]) {
#pragma unroll
    for (int k = 0; k < L; ++k) acc[k] = 0.0f;
    for (int n = 0; n < N; ++n) {
        const FrameShift s = sh[n];
        const float I = fr[n * TP + p];
        const float *wp = win + s.ky * WS + s.kx;
        float G[L];
        if (s.fy == 0.0f) {
            if (s.fx == 0.0f) {
#pragma unroll
                for (int k = 0; k < L; ++k) G[k] = wp[k];
            } else {
                float a0 = wp[0];
#pragma unroll
                for (int k = 0; k < L; ++k) {
                    const float b0 = wp[k + 1];
                    G[k] = fmaf(s.fx, b0 - a0, a0);
                    a0 = b0;
                }
            }
        } else {
            const float *wq = wp + WS;
            if (s.fx == 0.0f) {
#pragma unroll
                for (int k = 0; k < L; ++k) G[k] = fmaf(s.fy, wq[k] - wp[k], wp[k]);
            } else {
                float a0 = wp[0], a1 = wq[0];
#pragma unroll
                for (int k = 0; k < L; ++k) {
                    const float b0 = wp[k + 1], b1 = wq[k + 1];
                    const float t0 = fmaf(s.fx, b0 - a0, a0);
                    const float t1 = fmaf(s.fx, b1 - a1, a1);
                    G[k] = fmaf(s.fy, t1 - t0, t0);
                    a0 = b0;
                    a1 = b1;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < L; ++k) {
            const float d = fmaf(-Wv, G[k], I);
            acc[k] = fmaf(d, d, acc[k]);
        }
    }
}

// The same strip with the validity rule applied per frame: a window value that is NaN
// (off the grid or uncovered) drops its corner, the remaining corners are renormalised,
// and a frame with no valid corner is left out of both the error and var. Used only for
// strips in which the fast evaluation produced a NaN. e[k] = err / var (err if var = 0,
// +inf if no frame is valid).
template <int L>
__device__ __noinline__ void eval_strip_exact(const float *__restrict__ fr, int TP, int p,
                                              const FrameShift *__restrict__ sh, int N,
                                              const float *__restrict__ win, int WS, float Wv,
                                              float (&e)[L]) {
    float err[L], var[L];
    int nv[L];
#pragma unroll
    for (int k = 0; k < L; ++k) {
        err[k] = 0.0f;
        var[k] = 0.0f;
        nv[k] = 0;
    }
    for (int n = 0; n < N; ++n) {
        const FrameShift s = sh[n];
        const float I = fr[n * TP + p];
        const float t = I - Wv;
        const float *wp = win + s.ky * WS + s.kx;
        const float wt[4] = {(1.0f - s.fy) * (1.0f - s.fx), (1.0f - s.fy) * s.fx,
                             s.fy * (1.0f - s.fx), s.fy * s.fx};
#pragma unroll
        for (int k = 0; k < L; ++k) {
            const float v[4] = {wp[k], wp[k + 1], wp[WS + k], wp[WS + k + 1]};
            float num = 0.0f, den = 0.0f;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (wt[c] == 0.0f || isnan(v[c])) continue;
                num = fmaf(wt[c], v[c], num);
                den += wt[c];
            }
            if (den > 0.0f) {
                const float d = fmaf(-Wv, num / den, I);
                err[k] = fmaf(d, d, err[k]);
                var[k] = fmaf(t, t, var[k]);
                nv[k] += 1;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < L; ++k)
        e[k] = nv[k] == 0 ? INFINITY : (var[k] > 0.0f ? err[k] / var[k] : err[k]);
}

__device__ __forceinline__ bool lex_less(float e, int i, float e2, int i2) {
    return e < e2 || (e == e2 && i < i2);
}

template <int L, int TY, int TPP>
__global__ void __launch_bounds__(32 * TY * TPP) k_search(SearchArgs a) {
    constexpr int TP = 32 * TY;
    constexpr int NT = TP * TPP;
    extern __shared__ __align__(16) unsigned char smraw[];
    FrameShift *sh = reinterpret_cast<FrameShift *>(smraw);
    float *fr = reinterpret_cast<float *>(sh + a.N);
    float *win = fr + (size_t)a.N * TP;

    __shared__ int s_box[4];
    __shared__ int s_ci[TP], s_cj[TP], s_state[TP];
    __shared__ float s_W[TP], s_var[TP];
    __shared__ float s_be[TPP][TP];
    __shared__ int s_bi[TPP][TP];
    __shared__ float s_nb[9][TP];
    __shared__ int s_slow[TP];

    const int tid = threadIdx.x, p = tid % TP, sub = tid / TP;
    const int x = blockIdx.x * 32 + (p & 31), y = blockIdx.y * TY + (p >> 5);
    const size_t P = (size_t)a.ny * a.nx;
    const size_t pix = (size_t)y * a.nx + x;
    const bool inb = x < a.nx && y < a.ny;

    if (tid < 4) s_box[tid] = (tid & 1) ? INT_MIN : INT_MAX;
    for (int n = tid; n < a.N; n += NT) sh[n] = a.shifts[n];
    __syncthreads();
    if (sub == 0) {
        int st = 0, ci = 0, cj = 0;
        float Wv = 0.0f;
        if (inb && !a.mask[pix] && a.err_out) a.err_out[pix] = __int_as_float(0x7fc00000);
        if (inb && a.mask[pix]) {
            const double u0 = a.u[pix], u1 = a.u[P + pix];
            if (!isfinite(u0) || !isfinite(u1)) {
                atomicOr(&a.hdr->status, PXST_DEV_NONFINITE_U);
            } else if (fabs(u0) > kMaxCoord || fabs(u1) > kMaxCoord) {
                atomicOr(&a.hdr->status, PXST_DEV_U_RANGE);
            } else {
                ci = (int)floor(u0 + 0.5);
                cj = (int)floor(u1 + 0.5);
                Wv = a.W[pix];
                st = 1;
                atomicMin(&s_box[0], ci); atomicMax(&s_box[1], ci);
                atomicMin(&s_box[2], cj); atomicMax(&s_box[3], cj);
            }
        }
        s_state[p] = st;
        s_slow[p] = 0;
        s_ci[p] = ci;
        s_cj[p] = cj;
        s_W[p] = Wv;
    }
    // the tile's frames: [n][TP], coalesced 128-byte rows
    for (int idx = tid; idx < a.N * TP; idx += NT) {
        const int n = idx / TP, q = idx % TP;
        const int xx = blockIdx.x * 32 + (q & 31), yy = blockIdx.y * TY + (q >> 5);
        fr[idx] = (xx < a.nx && yy < a.ny) ? __ldg(a.frames + (size_t)n * P + (size_t)yy * a.nx + xx) : 0.0f;
    }
    __syncthreads();
    if (s_box[0] == INT_MAX) return;                 // no active pixel in this tile

    const int wy0 = s_box[0] - a.Sy + a.hdr->kmin_y;
    const int wy1 = s_box[1] + a.Sy + a.hdr->kmax_y + 1;
    const int wx0 = s_box[2] - a.Sx + a.hdr->kmin_x;
    const int wx1 = s_box[3] - a.Sx + a.nstrips * L - 1 + a.hdr->kmax_x + 1;
    const long long WHl = (long long)wy1 - wy0 + 1, WSl = (long long)wx1 - wx0 + 1;
    if (WHl * WSl > a.win_cap) {
        // the window does not fit: every active pixel of the tile takes the exact path
        if (sub == 0 && s_state[p] == 1) {
            const int k = atomicAdd(&a.hdr->n_exact, 1);
            a.exact_list[k] = (int)pix;
        }
        return;
    }
    const int WS = (int)WSl, WN = (int)(WHl * WSl);
    const float qnan = __int_as_float(0x7fc00000);
    for (int idx = tid; idx < WN; idx += NT) {
        const int gy = wy0 + idx / WS, gx = wx0 + idx % WS;
        float v = qnan;
        if (gy >= 0 && gy < a.Ry && gx >= 0 && gx < a.Rx) {
            const size_t g = (size_t)gy * a.Rx + gx;
            if (__ldg(a.w + g) > 0.0f) v = __ldg(a.Iref + g);
        }
        win[idx] = v;
    }
    if (sub == 0 && s_state[p] == 1) {
        const float Wv = s_W[p];
        float v = 0.0f;
        for (int n = 0; n < a.N; ++n) {
            const float t = fr[n * TP + p] - Wv;
            v = fmaf(t, t, v);
        }
        s_var[p] = v;
    }
    __syncthreads();

    const int wxn = 2 * a.Sx + 1;
    float best_e = INFINITY;
    int best_i = INT_MAX;
    const int st0 = s_state[p];
    if (st0 == 1) {
        const int ci = s_ci[p], cj = s_cj[p];
        const float Wv = s_W[p], var = s_var[p];
        for (int item = sub; item < a.nitems; item += TPP) {
            const int aa = item / a.nstrips - a.Sy;
            const int b0 = (item % a.nstrips) * L - a.Sx;
            const float *wstrip = win + (ci + aa - wy0) * WS + (cj + b0 - wx0);
            float acc[L];
            eval_strip<L>(fr, TP, p, sh, a.N, wstrip, WS, Wv, acc);
            bool nan_seen = false;
#pragma unroll
            for (int k = 0; k < L; ++k) {
                acc[k] = var > 0.0f ? acc[k] / var : acc[k];
                nan_seen = nan_seen || (isnan(acc[k]) && b0 + k <= a.Sx);
            }
            if (nan_seen) {
                eval_strip_exact<L>(fr, TP, p, sh, a.N, wstrip, WS, Wv, acc);
                s_slow[p] = 1;
            }
#pragma unroll
            for (int k = 0; k < L; ++k) {
                const int b = b0 + k;
                if (b > a.Sx) break;
                const int idx = (aa + a.Sy) * wxn + (b + a.Sx);
                if (acc[k] < best_e) { best_e = acc[k]; best_i = idx; }
            }
        }
    }
    s_be[sub][p] = best_e;
    s_bi[sub][p] = best_i;
    __syncthreads();
    if (sub == 0 && s_state[p] >= 1) {
        float be = s_be[0][p];
        int bi = s_bi[0][p];
#pragma unroll
        for (int t = 1; t < TPP; ++t)
            if (lex_less(s_be[t][p], s_bi[t][p], be, bi)) { be = s_be[t][p]; bi = s_bi[t][p]; }
        s_be[0][p] = be;
        s_bi[0][p] = bi;
    }
    __syncthreads();

    if (a.quadratic) {
        const int st = s_state[p];
        const float be = s_be[0][p];
        if (st == 1 && be < INFINITY) {
            const int bi = s_bi[0][p];
            const int ia = bi / wxn, ib = bi % wxn;
            const int ci = s_ci[p], cj = s_cj[p];
            const float Wv = s_W[p], var = s_var[p];
            for (int j = sub; j < 9; j += TPP) {
                const int na = ia + j / 3 - 1, nb = ib + j % 3 - 1;
                float e;
                if (na < 0 || na > 2 * a.Sy || nb < 0 || nb >= wxn) {
                    e = INFINITY;
                } else if (j == 4) {
                    e = be;
                } else {
                    const float *wn = win + (ci + na - a.Sy - wy0) * WS + (cj + nb - a.Sx - wx0);
                    float acc[1];
                    eval_strip<1>(fr, TP, p, sh, a.N, wn, WS, Wv, acc);
                    e = var > 0.0f ? acc[0] / var : acc[0];
                    if (isnan(e)) {
                        eval_strip_exact<1>(fr, TP, p, sh, a.N, wn, WS, Wv, acc);
                        e = acc[0];
                        s_slow[p] = 1;
                    }
                }
                s_nb[j][p] = e;
            }
        }
        __syncthreads();
    }

    if (sub == 0 && inb) {
        const int st = s_state[p];
        if (s_slow[p]) atomicAdd(&a.hdr->n_exact_cta, 1);
        if (st == 1) {
            const float be = s_be[0][p];
            if (!(be < INFINITY)) {
                if (a.err_out) a.err_out[pix] = INFINITY;
            } else {
                const int bi = s_bi[0][p];
                const int ia = bi / wxn, ib = bi % wxn;
                double da = 0.0, db = 0.0;
                if (a.quadratic) {
                    float f[9];
#pragma unroll
                    for (int j = 0; j < 9; ++j) f[j] = s_nb[j][p];
                    refine3x3(f, da, db);
                }
                a.u[pix] = (double)(s_ci[p] + ia - a.Sy) + da;
                a.u[P + pix] = (double)(s_cj[p] + ib - a.Sx) + db;
                if (a.err_out) a.err_out[pix] = be;
            }
        }
    }
}

// ------------------------------------------------------------------------------------
struct ExactArgs {
    int N, ny, nx, Ry, Rx, Sy, Sx, quadratic;
    const float *frames, *W;
    const uint8_t *mask;
    const float *Iref, *w;
    const FrameShift *shifts;
    WsHeader *hdr;
    const int *list;   // pixels to process; NULL = every pixel of the detector
    double *u;
    float *err_out;
};

__device__ float eval_exact(const ExactArgs &a, size_t pix, float Wv, int c0, int c1) {
    const size_t P = (size_t)a.ny * a.nx;
    float err = 0.0f, var = 0.0f;
    int nv = 0;
    for (int n = 0; n < a.N; ++n) {
        const FrameShift s = a.shifts[n];
        float R;
        if (!gather_masked(a.Iref, a.w, a.Ry, a.Rx, c0 + s.ky, c1 + s.kx, s.fy, s.fx, R)) continue;
        const float I = __ldg(a.frames + (size_t)n * P + pix);
        const float d = fmaf(-Wv, R, I);
        err = fmaf(d, d, err);
        const float t = I - Wv;
        var = fmaf(t, t, var);
        ++nv;
    }
    if (nv == 0) return INFINITY;
    return var > 0.0f ? err / var : err;
}

__global__ void __launch_bounds__(256) k_exact(ExactArgs a) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const size_t P = (size_t)a.ny * a.nx;
    const long long count = a.list ? (long long)a.hdr->n_exact : (long long)P;
    const int wyn = 2 * a.Sy + 1, wxn = 2 * a.Sx + 1, nwin = wyn * wxn;
    for (long long k = warp; k < count; k += nwarps) {
        const size_t pix = a.list ? (size_t)a.list[k] : (size_t)k;
        if (!a.list) {
            // every pixel: apply the same admission rules as the fast path
            if (!a.mask[pix]) {
                if (lane == 0 && a.err_out) a.err_out[pix] = __int_as_float(0x7fc00000);
                continue;
            }
            const double v0 = a.u[pix], v1 = a.u[P + pix];
            if (!isfinite(v0) || !isfinite(v1) || fabs(v0) > kMaxCoord || fabs(v1) > kMaxCoord) {
                if (lane == 0)
                    atomicOr(&a.hdr->status, (!isfinite(v0) || !isfinite(v1)) ? PXST_DEV_NONFINITE_U
                                                                             : PXST_DEV_U_RANGE);
                continue;
            }
        }
        const double u0 = a.u[pix], u1 = a.u[P + pix];
        const int ci = (int)floor(u0 + 0.5), cj = (int)floor(u1 + 0.5);
        const float Wv = a.W[pix];
        float be = INFINITY;
        int bi = INT_MAX;
        for (int idx = lane; idx < nwin; idx += 32) {
            const float e = eval_exact(a, pix, Wv, ci + idx / wxn - a.Sy, cj + idx % wxn - a.Sx);
            if (e < be) { be = e; bi = idx; }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float oe = __shfl_xor_sync(0xffffffffu, be, off);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
            if (lex_less(oe, oi, be, bi)) { be = oe; bi = oi; }
        }
        if (!(be < INFINITY)) {
            if (lane == 0 && a.err_out) a.err_out[pix] = INFINITY;
            continue;
        }
        const int ia = bi / wxn, ib = bi % wxn;
        float mine = INFINITY;
        if (a.quadratic && lane < 9) {
            const int na = ia + lane / 3 - 1, nb = ib + lane % 3 - 1;
            if (lane == 4) mine = be;
            else if (na >= 0 && na < wyn && nb >= 0 && nb < wxn)
                mine = eval_exact(a, pix, Wv, ci + na - a.Sy, cj + nb - a.Sx);
        }
        float f[9];
#pragma unroll
        for (int j = 0; j < 9; ++j) f[j] = __shfl_sync(0xffffffffu, mine, j);
        if (lane == 0) {
            double da = 0.0, db = 0.0;
            if (a.quadratic) refine3x3(f, da, db);
            a.u[pix] = (double)(ci + ia - a.Sy) + da;
            a.u[P + pix] = (double)(cj + ib - a.Sx) + db;
            if (a.err_out) a.err_out[pix] = be;
        }
    }
}

// ------------------------------------------------------------------------------------
// host-side planning

struct Plan {
    int L, TY, TPP, nstrips, nitems;
    size_t smem;
    int win_cap;
};

int pick_strip(int wxn) {
    const int cand[5] = {11, 9, 8, 7, 4};
    int best = 4, waste = INT_MAX;
    for (int L : cand) {
        const int ns = (wxn + L - 1) / L;
        const int wst = ns * L - wxn;
        if (wst < waste) { waste = wst; best = L; }
    }
    return best;
}

template <int L, int TY, int TPP>
cudaError_t launch_one(const SearchArgs &a, const Plan &pl, cudaStream_t stream) {
    auto kern = k_search<L, TY, TPP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.nx + 31) / 32, (a.ny + TY - 1) / TY);
    kern<<<grid, 32 * TY * TPP, pl.smem, stream>>>(a);
    return cudaGetLastError();
}

template <int L>
cudaError_t launch_L(const SearchArgs &a, const Plan &pl, cudaStream_t stream) {
    switch (pl.TY) {
        case 8: return launch_one<L, 8, 1>(a, pl, stream);
        case 4: return launch_one<L, 4, 2>(a, pl, stream);
        case 2: return launch_one<L, 2, 4>(a, pl, stream);
        default: return launch_one<L, 1, 8>(a, pl, stream);
    }
}

}  // namespace

// Largest frame count the fast path can stage (a 1 x 32 tile in shared memory).
int search_max_frames() { return (kSearchSmemBudget - 16 * 1024) / (32 * 4 + 16); }

cudaError_t launch_search(const pxst_dims &d, const pxst_options &o, const float *frames,
                          const float *W, const uint8_t *mask, const float *I_ref,
                          const float *w, const FrameShift *shifts, WsHeader *hdr,
                          int *exact_list, double *u, float *err_out, cudaStream_t stream) {
    Plan pl;
    const int wxn = 2 * o.win_x + 1, wyn = 2 * o.win_y + 1;
    pl.L = pick_strip(wxn);
    pl.nstrips = (wxn + pl.L - 1) / pl.L;
    pl.nitems = wyn * pl.nstrips;
    const size_t per_frame = 16;                 // FrameShift
    // largest tile whose frames take at most ~110 KB of shared memory
    pl.TY = 1;
    for (int ty = 8; ty >= 1; ty >>= 1)
        if ((size_t)d.n_frames * 32 * ty * 4 <= 110 * 1024) { pl.TY = ty; break; }
    pl.TPP = 8 / pl.TY;
    const size_t fixed = (size_t)d.n_frames * (per_frame + 32 * pl.TY * 4);
    // two CTAs per SM when the frames leave room for a useful window, else one
    size_t total = fixed + 24 * 1024 <= 100 * 1024 ? 100 * 1024 : (size_t)kSearchSmemBudget;
    if (fixed + 4096 > total) total = fixed + 4096;
    pl.smem = total;
    pl.win_cap = (int)((total - fixed) / 4);

    SearchArgs a;
    a.N = d.n_frames; a.ny = d.ny; a.nx = d.nx; a.Ry = d.ref_ny; a.Rx = d.ref_nx;
    a.Sy = o.win_y; a.Sx = o.win_x; a.quadratic = o.quadratic ? 1 : 0;
    a.nstrips = pl.nstrips; a.nitems = pl.nitems; a.win_cap = pl.win_cap;
    a.frames = frames; a.W = W; a.mask = mask; a.Iref = I_ref; a.w = w; a.shifts = shifts;
    a.hdr = hdr; a.exact_list = exact_list; a.u = u; a.err_out = err_out;
    switch (pl.L) {
        case 11: return launch_L<11>(a, pl, stream);
        case 9: return launch_L<9>(a, pl, stream);
        case 8: return launch_L<8>(a, pl, stream);
        case 7: return launch_L<7>(a, pl, stream);
        default: return launch_L<4>(a, pl, stream);
    }
}

cudaError_t launch_exact(const pxst_dims &d, const pxst_options &o, const float *frames,
                         const float *W, const uint8_t *mask, const float *I_ref,
                         const float *w, const FrameShift *shifts, WsHeader *hdr,
                         const int *exact_list, double *u, float *err_out, cudaStream_t stream) {
    // exact_list == NULL: every pixel (used when the frames cannot be staged on chip)
    ExactArgs a;
    a.N = d.n_frames; a.ny = d.ny; a.nx = d.nx; a.Ry = d.ref_ny; a.Rx = d.ref_nx;
    a.Sy = o.win_y; a.Sx = o.win_x; a.quadratic = o.quadratic ? 1 : 0;
    a.frames = frames; a.W = W; a.mask = mask; a.Iref = I_ref; a.w = w; a.shifts = shifts;
    a.hdr = hdr; a.list = exact_list; a.u = u; a.err_out = err_out;
    k_exact<<<152 * 4, 256, 0, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace pxst
