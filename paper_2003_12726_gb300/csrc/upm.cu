// upm.cu -- update_pixel_map ("Update pixel mapping", section "Main loop") on sm_103a.
//
// Fast path (k_search): one CTA of 256 threads per tile of TY x 32 pixels.
//   * the tile's frames, all N of them, are staged once in shared memory;
//   * the tile's reference window (every candidate of every pixel of the tile, widened
//     by the range of integer frame shifts and one bilinear corner) is staged once, with
//     uncovered or off-grid reference pixels stored as NaN;
//   * groups of 4 neighbouring pixels of a row share strips of L absolute reference
//     columns on one reference row: per frame one window read and, for fractional
//     translations, one lerp per column serve the 4 pixels, then d = I - W R and
//     err += d^2 are two FP32 FMAs per evaluation;
//   * a NaN error means some frame read an invalid reference pixel, where the paper's
//     rule drops that corner (or the whole frame) instead; only such strips are evaluated
//     again with the rule applied per frame. Valid strips need no per-frame check, so the
//     check costs nothing in the inner loop;
//   * per-pixel argmins (first minimum in row-major window order) are combined with a
//     packed 64-bit atomicMin in shared memory; the 3x3 about the minimum is re-evaluated
//     and fitted in FP64.
// Global path (k_exact): one warp per listed pixel, candidates over lanes, per-frame
// masked renormalised reads from global memory, lexicographic warp argmin, FP64 fit.
// It serves tiles whose reference window does not fit in shared memory and scans with
// too many frames to stage.
// Rescore (k_rescore_tile, k_rescore_general): the exact stage of the tensor-core forms,
// one thread per pixel.
#include <algorithm>
#include <climits>
#include <cmath>

#include "pxst_common.cuh"

namespace pxst {
namespace {

struct SearchArgs {
    int N, ny, nx, Ry, Rx, Sy, Sx, quadratic, ebuf, win_cap;
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
// One strip of L candidates (same row, consecutive columns) over all frames.
// win points at the window row/column of the strip's first candidate for a zero shift.
template <int L>
__device__ __forceinline__ void eval_strip(const float *__restrict__ fr, int pitch, int p,
                                           const FrameShift *__restrict__ sh, int N,
                                           const float *__restrict__ win, int WS, float Wv,
                                           float (&acc)[L]) {
#pragma unroll
    for (int k = 0; k < L; ++k) acc[k] = 0.0f;
    for (int n = 0; n < N; ++n) {
        const FrameShift s = sh[n];
        const float I = fr[n * pitch + p];
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
// strips in which the fast evaluation produced a NaN. Accumulates frames
// n = n0, n0 + step, ... into err/var/nv (which the caller zeroes and later reduces).
template <int L>
__device__ __forceinline__ void accum_strip_exact(const float *__restrict__ fr, int pitch, int p,
                                                  const FrameShift *__restrict__ sh, int n0,
                                                  int step, int N, const float *__restrict__ win,
                                                  int WS, float Wv, float (&err)[L],
                                                  float (&var)[L], float (&nv)[L],
                                                  unsigned cm = 0xffffffffu) {
    for (int n = n0; n < N; n += step) {
        const FrameShift s = sh[n];
        const float I = fr[n * pitch + p];
        const float t = I - Wv, t2 = t * t;
        const float *wp = win + s.ky * WS + s.kx;
        const float w00 = (1.0f - s.fy) * (1.0f - s.fx), w01 = (1.0f - s.fy) * s.fx;
        const float w10 = s.fy * (1.0f - s.fx), w11 = s.fy * s.fx;
#pragma unroll
        for (int k = 0; k < L; ++k) {
            if (!((cm >> k) & 1u)) continue;          // a column the fast path evaluated
            const float v00 = wp[k];
            const float v01 = s.fx != 0.0f ? wp[k + 1] : 0.0f;
            const float v10 = s.fy != 0.0f ? wp[WS + k] : 0.0f;
            const float v11 = (s.fx != 0.0f && s.fy != 0.0f) ? wp[WS + k + 1] : 0.0f;
            float R;
            bool valid;
            if (!isnan(v00) && !isnan(v01) && !isnan(v10) && !isnan(v11)) {
                // every corner counts: the read the fast path makes, bit for bit
                if (s.fy == 0.0f) R = s.fx == 0.0f ? v00 : fmaf(s.fx, v01 - v00, v00);
                else if (s.fx == 0.0f) R = fmaf(s.fy, v10 - v00, v00);
                else {
                    const float t0 = fmaf(s.fx, v01 - v00, v00), t1 = fmaf(s.fx, v11 - v10, v10);
                    R = fmaf(s.fy, t1 - t0, t0);
                }
                valid = true;
            } else {
                float num = 0.0f, den = 0.0f;
                if (!isnan(v00)) { num = w00 * v00; den = w00; }
                if (s.fx != 0.0f && !isnan(v01)) { num = fmaf(w01, v01, num); den += w01; }
                if (s.fy != 0.0f && !isnan(v10)) { num = fmaf(w10, v10, num); den += w10; }
                if (s.fx != 0.0f && s.fy != 0.0f && !isnan(v11)) { num = fmaf(w11, v11, num); den += w11; }
                valid = den > 0.0f;
                R = valid ? num / den : 0.0f;
            }
            if (valid) {
                const float d = fmaf(-Wv, R, I);
                err[k] = fmaf(d, d, err[k]);
                var[k] += t2;
                nv[k] += 1.0f;
            }
        }
    }
}

// e = err / var, with the pixel's own all-frame var (the fast path's value) wherever every
// frame counted, so that a candidate gets the same value whichever path evaluated it.
template <int L>
__device__ __forceinline__ void finish_exact(const float (&err)[L], const float (&var)[L],
                                             const float (&nv)[L], int N, float var_all,
                                             float (&e)[L]) {
#pragma unroll
    for (int k = 0; k < L; ++k) {
        const float vk = nv[k] == (float)N ? var_all : var[k];
        e[k] = nv[k] == 0.0f ? INFINITY : (vk > 0.0f ? err[k] / vk : err[k]);
    }
}

// Whole-strip exact evaluation by one thread, with the same frame partition (n mod 4) and
// the same combination of the four partial sums as the strips evaluated by four lanes.
template <int L>
__device__ __noinline__ void eval_strip_exact(const float *__restrict__ fr, int pitch, int p,
                                              const FrameShift *__restrict__ sh, int N,
                                              const float *__restrict__ win, int WS, float Wv,
                                              float var_all, float (&e)[L]) {
    float err[4][L], var[4][L], nv[4][L];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int k = 0; k < L; ++k) err[j][k] = var[j][k] = nv[j][k] = 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) accum_strip_exact<L>(fr, pitch, p, sh, j, 4, N, win, WS, Wv, err[j], var[j], nv[j]);
    float E[L], V[L], C[L];
#pragma unroll
    for (int k = 0; k < L; ++k) {
        E[k] = (err[0][k] + err[1][k]) + (err[2][k] + err[3][k]);
        V[k] = (var[0][k] + var[1][k]) + (var[2][k] + var[3][k]);
        C[k] = (nv[0][k] + nv[1][k]) + (nv[2][k] + nv[3][k]);
    }
    finish_exact<L>(E, V, C, N, var_all, e);
}

__device__ __forceinline__ bool lex_less(float e, int i, float e2, int i2) {
    return e < e2 || (e == e2 && i < i2);
}

constexpr int kGroup = 4;            // pixels per group: consecutive columns of one row
constexpr int kSplit = 4;            // lanes that share one strip, each taking every 4th frame
constexpr int kSearchThreads = 256;
constexpr int kExactList = 4096;     // (strip, pixel, NaN columns) entries for the exact phase
constexpr int kWinRowsMax = 512;     // window rows with a coverage flag (taller windows: no flag)
static_assert(kSplit == kGroup, "the reduce-scatter hands lane j the sums of pixel j");

// One strip of L consecutive absolute reference columns on one reference row, for the
// kGroup pixels of a group, over the frames n = n0, n0 + kSplit, ...:
// acc[p][k] = sum_n (I_p - W_p R_n(col_k))^2. `win` points at the window position of the
// strip's first column for a zero shift; frame rows of `fr` are FP floats apart. One
// window read (and one lerp for fractional translations) serves all kGroup pixels.
template <int L>
__device__ __forceinline__ void eval_group(const float *__restrict__ fr, int FP, int g0,
                                           const FrameShift *__restrict__ sh, int n0, int N,
                                           const float *__restrict__ win, int WS,
                                           const float (&Wv)[kGroup], float (&acc)[kGroup][L]) {
    // pixels (0,1) and (2,3) are packed in float2 lanes: one FFMA2 advances two pixels
    const float2 nW[2] = {make_float2(-Wv[0], -Wv[1]), make_float2(-Wv[2], -Wv[3])};
    float2 acc2[2][L];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int k = 0; k < L; ++k) acc2[h][k] = make_float2(0.0f, 0.0f);
    for (int n = n0; n < N; n += kSplit) {
        const FrameShift s = sh[n];
        const float4 I4 = *reinterpret_cast<const float4 *>(fr + n * FP + g0);
        const float2 I2[2] = {make_float2(I4.x, I4.y), make_float2(I4.z, I4.w)};
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
            const float2 GG = make_float2(G[k], G[k]);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float2 d = __ffma2_rn(nW[h], GG, I2[h]);      // I - W R, two pixels
                acc2[h][k] = __ffma2_rn(d, d, acc2[h][k]);          // += d^2
            }
        }
    }
#pragma unroll
    for (int k = 0; k < L; ++k) {
        acc[0][k] = acc2[0][k].x;
        acc[1][k] = acc2[0][k].y;
        acc[2][k] = acc2[1][k].x;
        acc[3][k] = acc2[1][k].y;
    }
}

// Reduce-scatter over the kSplit = 4 lanes of a strip: afterwards lane j (j = lane & 3)
// holds in out[k] the sum over the 4 lanes of acc[j][k]. Every lane of the warp calls it.
template <int L>
__device__ __forceinline__ void reduce_scatter4(const float (&acc)[kGroup][L], int j, float (&out)[L]) {
    const bool b0 = j & 1, b1 = (j >> 1) & 1;
    float h[2][L];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int k = 0; k < L; ++k) {
            const float send = b0 ? acc[2 * q][k] : acc[2 * q + 1][k];
            const float keep = b0 ? acc[2 * q + 1][k] : acc[2 * q][k];
            h[q][k] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
        }
#pragma unroll
    for (int k = 0; k < L; ++k) {
        const float send = b1 ? h[0][k] : h[1][k];
        const float keep = b1 ? h[1][k] : h[0][k];
        out[k] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
}

__device__ __forceinline__ unsigned long long pack_key(float e, int idx) {
    // e >= 0 (or +inf): its bit pattern orders like the value, so (e, idx) compares
    // lexicographically as one unsigned 64-bit key
    return ((unsigned long long)__float_as_uint(e) << 32) | (unsigned int)idx;
}

// Fast path. One CTA per tile of TY rows x 32 columns of pixels, 256 threads.
// Groups of kGroup neighbouring pixels share the strips of the union of their windows
// (absolute reference rows and columns); each strip is evaluated by kSplit lanes that
// split the frames, then reduce-scatter so that lane j finishes pixel j of the group.
// Each candidate of each pixel is evaluated exactly once; per-pixel argmins are combined
// with a packed (error, window index) 64-bit atomicMin in shared memory, which keeps the
// first minimum in row-major window order. With a.ebuf every error is also kept in
// shared memory, so the 3x3 about the minimum is read back instead of re-evaluated.
template <int L, int TY>
__global__ void __launch_bounds__(kSearchThreads, (L <= 9 ? 3 : 2)) k_search(SearchArgs a) {
    constexpr int TP = 32 * TY;
    constexpr int FP = TP + 4;            // frame pitch: the 4 lanes of a strip hit 4 banks
    constexpr int NG = TP / kGroup;
    constexpr int NT = kSearchThreads;
    extern __shared__ __align__(16) unsigned char smraw[];
    FrameShift *sh = reinterpret_cast<FrameShift *>(smraw);
    float *fr = reinterpret_cast<float *>(sh + a.N);
    const int wxn = 2 * a.Sx + 1, nwin = (2 * a.Sy + 1) * wxn;
    float *ebuf = fr + (size_t)a.N * FP;
    float *win = ebuf + (a.ebuf ? (size_t)TP * nwin : 0);

    __shared__ int s_box[4];
    __shared__ int s_ci[TP], s_cj[TP], s_act[TP], s_slow[TP];
    __shared__ float s_W[TP], s_var[TP];
    __shared__ unsigned long long s_key[TP];
    __shared__ float s_nb[9][TP];
    __shared__ int s_gr0[NG], s_gc0[NG], s_gns[NG], s_goff[NG + 1];
    // exact phase: entries (item << 13) | (j << 11) | mask of the columns that read an
    // invalid reference pixel in some frame; s_rowany: the window row holds a valid cell
    __shared__ unsigned int s_xlist[kExactList];
    __shared__ int s_xn;
    __shared__ unsigned char s_rowany[kWinRowsMax];
    __shared__ int s_glob[TP];                       // 1: the pixel is left to the global path

    const int tid = threadIdx.x;
    const size_t P = (size_t)a.ny * a.nx;

    if (tid < 4) s_box[tid] = (tid & 1) ? INT_MIN : INT_MAX;
    if (tid == 0) s_xn = 0;
    for (int q = tid; q < kWinRowsMax; q += NT) s_rowany[q] = 0;
    int fy_local = 0;
    for (int n = tid; n < a.N; n += NT) {
        const FrameShift f = a.shifts[n];
        sh[n] = f;
        fy_local |= f.fy != 0.0f;
    }
    // some frame reads the row below its integer shift (a fractional ss translation)
    const int any_fy = __syncthreads_or(fy_local);
    for (int p = tid; p < TP; p += NT) {
        const int x = blockIdx.x * 32 + (p & 31), y = blockIdx.y * TY + (p >> 5);
        int act = 0, ci = 0, cj = 0;
        float Wv = 0.0f;
        if (x < a.nx && y < a.ny) {
            const size_t pix = (size_t)y * a.nx + x;
            if (!a.mask[pix]) {
                if (a.err_out) a.err_out[pix] = __int_as_float(0x7fc00000);
            } else {
                const double u0 = a.u[pix], u1 = a.u[P + pix];
                if (!isfinite(u0) || !isfinite(u1)) {
                    atomicOr(&a.hdr->status, PXST_DEV_NONFINITE_U);
                } else if (fabs(u0) > kMaxCoord || fabs(u1) > kMaxCoord) {
                    atomicOr(&a.hdr->status, PXST_DEV_U_RANGE);
                } else if (!(a.W[pix] > 0.0f) || !isfinite(a.W[pix])) {
                    // not a usable whitefield value: the pixel is left as a masked one
                    atomicOr(&a.hdr->status, PXST_DEV_BAD_INPUT);
                    if (a.err_out) a.err_out[pix] = __int_as_float(0x7fc00000);
                } else {
                    ci = (int)floor(u0 + 0.5);
                    cj = (int)floor(u1 + 0.5);
                    Wv = a.W[pix];
                    act = 1;
                }
            }
        }
        s_act[p] = act;
        s_ci[p] = ci;
        s_cj[p] = cj;
        s_W[p] = Wv;
        s_slow[p] = 0;
        s_glob[p] = 0;
        s_key[p] = ~0ull;
    }
    // the tile's frames: [n][FP], coalesced 128-byte rows
    for (int idx = tid; idx < a.N * TP; idx += NT) {
        const int n = idx / TP, q = idx % TP;
        const int xx = blockIdx.x * 32 + (q & 31), yy = blockIdx.y * TY + (q >> 5);
        fr[n * FP + q] = (xx < a.nx && yy < a.ny) ? __ldg(a.frames + (size_t)n * P + (size_t)yy * a.nx + xx) : 0.0f;
    }
    __syncthreads();
    for (int p = tid; p < TP; p += NT) {
        if (!s_act[p]) continue;
        const float Wv = s_W[p];
        float v = 0.0f;
        for (int n = 0; n < a.N; ++n) {
            const float t = fr[n * FP + p] - Wv;
            v = fmaf(t, t, v);
        }
        s_var[p] = v;
        // a non-finite frame value: every candidate's error is NaN, so the pixel keeps its map
        if (!isfinite(v)) atomicOr(&a.hdr->status, PXST_DEV_BAD_INPUT);
    }
    for (int g = tid; g < NG; g += NT) {
        int mn_i = INT_MAX, mx_i = INT_MIN, mn_j = INT_MAX, mx_j = INT_MIN;
        for (int q = 0; q < kGroup; ++q) {
            const int p = g * kGroup + q;
            if (!s_act[p]) continue;
            mn_i = min(mn_i, s_ci[p]); mx_i = max(mx_i, s_ci[p]);
            mn_j = min(mn_j, s_cj[p]); mx_j = max(mx_j, s_cj[p]);
        }
        int cnt = 0;
        if (mn_i != INT_MAX) {
            const int uy = mx_i - mn_i + 2 * a.Sy + 1, ux = mx_j - mn_j + wxn;
            const int ns = (ux + L - 1) / L;
            s_gr0[g] = mn_i - a.Sy;
            s_gc0[g] = mn_j - a.Sx;
            s_gns[g] = ns;
            cnt = uy * ns;
            atomicMin(&s_box[0], mn_i);
            atomicMax(&s_box[1], mx_i);
            atomicMin(&s_box[2], mn_j);
            atomicMax(&s_box[3], mn_j - a.Sx + ns * L - 1);
        }
        s_goff[g + 1] = cnt;
    }
    __syncthreads();
    if (s_box[0] == INT_MAX) return;                 // no active pixel in this tile
    if (tid == 0) {
        s_goff[0] = 0;
        for (int g = 0; g < NG; ++g) s_goff[g + 1] += s_goff[g];
    }

    const int wy0 = s_box[0] - a.Sy + a.hdr->kmin_y;
    const int wy1 = s_box[1] + a.Sy + a.hdr->kmax_y + 1;
    const int wx0 = s_box[2] - a.Sx + a.hdr->kmin_x;
    const int wx1 = s_box[3] + a.hdr->kmax_x + 1;
    long long WSl = (long long)wx1 - wx0 + 1;
    WSl += (WSl & 1) ? 0 : 1;                        // odd row pitch: fewer bank conflicts
    const long long WHl = (long long)wy1 - wy0 + 1;
    if (WHl * WSl > a.win_cap) {
        // the window does not fit: every active pixel of the tile takes the global path
        for (int p = tid; p < TP; p += NT) {
            if (!s_act[p]) continue;
            const int x = blockIdx.x * 32 + (p & 31), y = blockIdx.y * TY + (p >> 5);
            const int k = atomicAdd(&a.hdr->n_exact, 1);
            a.exact_list[k] = y * a.nx + x;
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
        if (v == v && idx / WS < kWinRowsMax) s_rowany[idx / WS] = 1;
    }
    __syncthreads();
    const int WH = (int)WHl;
    const int kmin_y = a.hdr->kmin_y, kmax_y = a.hdr->kmax_y;

    // ---- search: strips of the groups' window unions, 4 lanes per strip ----------------
    const int j = tid & (kSplit - 1);
    const int units = s_goff[NG] * kSplit;
    for (int u0 = 0; u0 < units; u0 += NT) {
        const int t = u0 + tid;
        const bool valid = t < units;               // uniform over each strip's 4 lanes
        const int item = t / kSplit;
        int g = 0, r = 0, c = 0;
        float acc[kGroup][L];
        if (valid) {
            int lo = 0, hi = NG - 1;                 // group g with s_goff[g] <= item < s_goff[g+1]
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_goff[mid] <= item) lo = mid; else hi = mid - 1;
            }
            g = lo;
            const int loc = item - s_goff[g], ns = s_gns[g];
            r = s_gr0[g] + loc / ns;
            c = s_gc0[g] + (loc % ns) * L;
            float Wv[kGroup];
#pragma unroll
            for (int q = 0; q < kGroup; ++q) Wv[q] = s_W[g * kGroup + q];
            eval_group<L>(fr, FP, g * kGroup, sh, j, a.N, win + (r - wy0) * WS + (c - wx0), WS, Wv, acc);
        } else {
#pragma unroll
            for (int q = 0; q < kGroup; ++q)
#pragma unroll
                for (int k = 0; k < L; ++k) acc[q][k] = 0.0f;
        }
        float e[L];
        reduce_scatter4<L>(acc, j, e);
        const int p = g * kGroup + j;
        if (!valid || !s_act[p]) continue;
        const int aa = r - s_ci[p];
        if (aa < -a.Sy || aa > a.Sy) continue;
        const int bofs = c - s_cj[p];
        const float var = s_var[p];
        unsigned cm = 0u;                            // window columns whose error is NaN
#pragma unroll
        for (int k = 0; k < L; ++k) {
            e[k] = var > 0.0f ? e[k] / var : e[k];
            const int b = bofs + k;
            if (isnan(e[k]) && b >= -a.Sx && b <= a.Sx) cm |= 1u << k;
        }
        if (cm) {
            // every frame reads window rows r + ky (+1 for a fractional ss shift); if none of
            // them holds a valid cell, no frame is valid for any column: the error is +inf
            const int q0 = r - wy0 + kmin_y, q1 = r - wy0 + kmax_y + any_fy;
            bool none = WH <= kWinRowsMax;
            for (int q = q0; none && q <= q1; ++q) none = s_rowany[q] == 0;
            if (none) {
#pragma unroll
                for (int k = 0; k < L; ++k)
                    if ((cm >> k) & 1u) e[k] = INFINITY;
                cm = 0u;
            } else {
                s_slow[p] = 1;
                const int slot = item < (1 << 19) ? atomicAdd(&s_xn, 1) : kExactList;
                if (slot < kExactList)               // evaluated by the whole CTA below
                    s_xlist[slot] = ((unsigned)item << 13) | ((unsigned)j << 11) | cm;
                else
                    s_glob[p] = 1;                   // beyond the list: the global path
            }
        }
        // the columns every frame of which was valid: the fast path's value is the exact one
        float be = INFINITY;
        int bi = -1;
#pragma unroll
        for (int k = 0; k < L; ++k) {
            const int b = bofs + k;
            if (b < -a.Sx || b > a.Sx || ((cm >> k) & 1u)) continue;
            const int idx = (aa + a.Sy) * wxn + (b + a.Sx);
            if (a.ebuf) ebuf[p * nwin + idx] = e[k];
            if (bi < 0 || e[k] < be) {
                be = e[k];
                bi = idx;
            }
        }
        if (bi >= 0) atomicMin(&s_key[p], pack_key(be, bi));
    }
    __syncthreads();

    // ---- columns that read invalid reference pixels: per-frame rule, 4 lanes per entry ----
    // Each warp takes 8 list entries at a time; every exact error is formed by the same
    // frame split and reduction whichever warp takes its entry, so results do not depend
    // on scheduling.
    {
        const int lane = tid & 31, warp = tid >> 5, slot = lane >> 2;
        const int nent = min(s_xn, kExactList);
        for (int e0 = warp * 8; e0 < nent; e0 += NT / 4) {
            const int ent = e0 + slot;
            const bool valid = ent < nent;
            float err[L], var[L], nv[L];
#pragma unroll
            for (int k = 0; k < L; ++k) err[k] = var[k] = nv[k] = 0.0f;
            int p = 0, r = 0, c = 0;
            unsigned cm = 0u;
            if (valid) {
                const unsigned x = s_xlist[ent];
                const int item = (int)(x >> 13);
                cm = x & 0x7ffu;
                int lo = 0, hi = NG - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_goff[mid] <= item) lo = mid; else hi = mid - 1;
                }
                const int loc = item - s_goff[lo], ns = s_gns[lo];
                r = s_gr0[lo] + loc / ns;
                c = s_gc0[lo] + (loc % ns) * L;
                p = lo * kGroup + (int)((x >> 11) & 3u);
                accum_strip_exact<L>(fr, FP, p, sh, j, kSplit, a.N, win + (r - wy0) * WS + (c - wx0), WS, s_W[p],
                                     err, var, nv, cm);
            }
#pragma unroll
            for (int k = 0; k < L; ++k)
#pragma unroll
                for (int off = 1; off < kSplit; off <<= 1) {
                    err[k] += __shfl_xor_sync(0xffffffffu, err[k], off);
                    var[k] += __shfl_xor_sync(0xffffffffu, var[k], off);
                    nv[k] += __shfl_xor_sync(0xffffffffu, nv[k], off);
                }
            if (!valid || j != 0) continue;
            const int aa = r - s_ci[p], bofs = c - s_cj[p];
            float e[L];
            finish_exact<L>(err, var, nv, a.N, s_var[p], e);
            float be = INFINITY;
            int bi = -1;
#pragma unroll
            for (int k = 0; k < L; ++k) {
                const int b = bofs + k;
                if (!((cm >> k) & 1u)) continue;
                const int idx = (aa + a.Sy) * wxn + (b + a.Sx);
                if (a.ebuf) ebuf[p * nwin + idx] = e[k];
                if (bi < 0 || e[k] < be) {
                    be = e[k];
                    bi = idx;
                }
            }
            if (bi >= 0) atomicMin(&s_key[p], pack_key(be, bi));
        }
    }
    __syncthreads();

    // ---- 3x3 about each pixel's minimum ---------------------------------------------------
    if (a.quadratic) {
        for (int q = tid; q < TP * 9; q += NT) {
            const int p = q / 9, jn = q % 9;
            if (!s_act[p]) continue;
            const unsigned long long key = s_key[p];
            const float be = __uint_as_float((unsigned int)(key >> 32));
            if (!(be < INFINITY)) continue;
            const int bi = (int)(key & 0xffffffffu);
            const int na = bi / wxn + jn / 3 - 1, nb = bi % wxn + jn % 3 - 1;
            float ev;
            if (na < 0 || na > 2 * a.Sy || nb < 0 || nb >= wxn) {
                ev = INFINITY;
            } else if (jn == 4) {
                ev = be;
            } else if (a.ebuf) {
                ev = ebuf[p * nwin + na * wxn + nb];
            } else {
                const float *wn = win + (s_ci[p] + na - a.Sy - wy0) * WS + (s_cj[p] + nb - a.Sx - wx0);
                float acc1[1];
                eval_strip<1>(fr, FP, p, sh, a.N, wn, WS, s_W[p], acc1);
                const float var = s_var[p];
                ev = var > 0.0f ? acc1[0] / var : acc1[0];
                if (isnan(ev)) {
                    eval_strip_exact<1>(fr, FP, p, sh, a.N, wn, WS, s_W[p], var, acc1);
                    ev = acc1[0];
                    s_slow[p] = 1;
                }
            }
            s_nb[jn][p] = ev;
        }
        __syncthreads();
    }

    for (int p = tid; p < TP; p += NT) {
        if (!s_act[p]) continue;
        const int x = blockIdx.x * 32 + (p & 31), y = blockIdx.y * TY + (p >> 5);
        const size_t pix = (size_t)y * a.nx + x;
        if (s_glob[p]) {
            a.exact_list[atomicAdd(&a.hdr->n_exact, 1)] = (int)pix;
            continue;
        }
        if (s_slow[p]) atomicAdd(&a.hdr->n_exact_cta, 1);
        const unsigned long long key = s_key[p];
        const float be = __uint_as_float((unsigned int)(key >> 32));
        if (!(be < INFINITY)) {
            if (a.err_out) a.err_out[pix] = INFINITY;
            continue;
        }
        const int bi = (int)(key & 0xffffffffu);
        const int ia = bi / wxn, ib = bi % wxn;
        double da = 0.0, db = 0.0;
        if (a.quadratic) {
            float f[9];
#pragma unroll
            for (int jn = 0; jn < 9; ++jn) f[jn] = s_nb[jn][p];
            refine3x3(f, da, db);
        }
        a.u[pix] = (double)(s_ci[p] + ia - a.Sy) + da;
        a.u[P + pix] = (double)(s_cj[p] + ib - a.Sx) + db;
        if (a.err_out) a.err_out[pix] = be;
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
            if (!(a.W[pix] > 0.0f) || !isfinite(a.W[pix])) {
                if (lane == 0) {
                    atomicOr(&a.hdr->status, PXST_DEV_BAD_INPUT);
                    if (a.err_out) a.err_out[pix] = __int_as_float(0x7fc00000);
                }
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
    int L, TY, nstrips;
    size_t smem;
    int win_cap;
};

// Strip length: odd (bank-friendly), chosen to waste the fewest columns on the union of
// a group's windows (window width plus the few columns its kGroup centres spread over).
int pick_strip(int wxn) {
    const int cand[3] = {11, 9, 7};
    const int ux = wxn + kGroup;
    int best = 7, waste = INT_MAX;
    for (int L : cand) {
        const int wst = ((ux + L - 1) / L) * L - ux;
        if (wst < waste) { waste = wst; best = L; }
    }
    return best;
}

template <int L, int TY>
cudaError_t launch_one(const SearchArgs &a, const Plan &pl, cudaStream_t stream) {
    auto kern = k_search<L, TY>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.nx + 31) / 32, (a.ny + TY - 1) / TY);
    kern<<<grid, kSearchThreads, pl.smem, stream>>>(a); note_launch();
    return cudaGetLastError();
}

// Static shared memory and the register-limited number of resident CTAs of one variant.
template <int L, int TY>
cudaError_t variant_info(size_t &static_smem, int &ctas_by_regs) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_search<L, TY>);
    if (e != cudaSuccess) return e;
    static_smem = fa.sharedSizeBytes;
    const int regs = (fa.numRegs + 7) & ~7;          // allocated per thread in units of 8
    ctas_by_regs = 65536 / (regs * kSearchThreads);
    return cudaSuccess;
}

template <int L>
cudaError_t variant_info_L(int TY, size_t &st, int &cr) {
    switch (TY) {
        case 8: return variant_info<L, 8>(st, cr);
        case 4: return variant_info<L, 4>(st, cr);
        case 2: return variant_info<L, 2>(st, cr);
        default: return variant_info<L, 1>(st, cr);
    }
}

cudaError_t variant_info_any(int L, int TY, size_t &st, int &cr) {
    switch (L) {
        case 11: return variant_info_L<11>(TY, st, cr);
        case 9: return variant_info_L<9>(TY, st, cr);
        default: return variant_info_L<7>(TY, st, cr);
    }
}

template <int L>
cudaError_t launch_L(const SearchArgs &a, const Plan &pl, cudaStream_t stream) {
    switch (pl.TY) {
        case 8: return launch_one<L, 8>(a, pl, stream);
        case 4: return launch_one<L, 4>(a, pl, stream);
        case 2: return launch_one<L, 2>(a, pl, stream);
        default: return launch_one<L, 1>(a, pl, stream);
    }
}


// ------------------------------------------------------------------------------------
// Rescore of the tensor-core forms: exact FP32 errors of the candidates the reduced-
// precision ranking kept (for pixels with candidates not valid in every frame, the masked
// ranking's), and of the 3x3 about the best, then the FP64 fit. k_rescore: one block per
// 128 consecutive pixels, one thread per pixel; each thread streams its own pixel's frames
// through a 3-stage cp.async pipeline in shared memory (no block barrier in the loop, so
// warps run at their own pace) while it evaluates the 3x3 about its first candidate and the
// other kept candidates; the reference is read through the cache.
struct RescoreArgs {
    int N, ny, nx, Ry, Rx, Sy, Sx, quadratic, ncand;
    const float *frames, *W;
    const uint8_t *mask;
    const float *Rm;          // I_ref where w > 0, NaN elsewhere
    const int *nvalid;        // frames in which each reference pixel is a valid candidate
    const FrameShift *shifts;
    const int *cand;          // [P][kTopK] window indices, -1 = none
    WsHeader *hdr;
    int *wlist;               // warps (pixel index / 32) left to the general kernel
    int *second;              // [4 x n_second]: pixel, window index of its minimum, error bits, 0
    double *u;
    float *err_out;
};

// The frames stream through once: their loads are marked streaming (evict first), so that
// they do not displace the masked reference and the validity counts, which every pixel
// re-reads.

// Running sums of one candidate over the frames where it is valid.
struct CandSums {
    float err, var;
    int nv;
    __device__ __forceinline__ void zero() { err = var = 0.0f; nv = 0; }
    // frame value I, t = I - W; R read for this frame (ok: valid)
    __device__ __forceinline__ void add(bool ok, float R, float I, float t, float Wv) {
        if (ok) {
            const float d = fmaf(-Wv, R, I);
            err = fmaf(d, d, err);
            var = fmaf(t, t, var);
            ++nv;
        }
    }
    __device__ __forceinline__ float e() const { return nv == 0 ? INFINITY : (var > 0.0f ? err / var : err); }
};

// R for a whole-pixel shift (ky, kx) of candidate (cy, cx) with flat index base = cy Rx + cx
// and off = ky Rx + kx: NaN when the read is off the grid (or uncovered). `safe`: every
// shift keeps this candidate's reads on the grid, so no bounds test is needed.
__device__ __forceinline__ float read_int(const RescoreArgs &a, int cy, int cx, int base, bool safe, int ky, int kx,
                                          int off) {
    const bool inb = safe || ((unsigned)(cy + ky) < (unsigned)a.Ry && (unsigned)(cx + kx) < (unsigned)a.Rx);
    return inb ? __ldg(a.Rm + (base + off)) : __int_as_float(0x7fc00000);
}

// R_n of candidate (cy, cx) for any shift: whole shifts by one load, else the general gather
__device__ __forceinline__ bool read_any(const RescoreArgs &a, int cy, int cx, int base, bool safe,
                                         const FrameShift &s, float &R) {
    if (s.fy == 0.0f && s.fx == 0.0f) {
        R = read_int(a, cy, cx, base, safe, s.ky, s.kx, s.ky * a.Rx + s.kx);
        return R == R;
    }
    return gather_rm(a.Rm, a.Ry, a.Rx, cy + s.ky, cx + s.kx, s.fy, s.fx, R);
}

// every shift's reads of candidate rows [y0, y1] and columns [x0, x1] stay on the grid
__device__ __forceinline__ bool span_safe(const RescoreArgs &a, int y0, int y1, int x0, int x1) {
    const WsHeader &h = *a.hdr;
    return y0 + h.kmin_y >= 0 && y1 + h.kmax_y + 1 < a.Ry && x0 + h.kmin_x >= 0 && x1 + h.kmax_x + 1 < a.Rx;
}

constexpr int RS_F = 16;      // frames per pipeline stage
constexpr int RS_S = 3;       // pipeline stages

__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory"); }

// The candidates one thread rescores: the 3x3 about the first kept candidate c0 (a window
// index) and up to XK other kept candidates that lie outside that 3x3.
template <int XK>
struct PixCands {
    static constexpr int NX = XK > 0 ? XK : 1;
    bool act;                 // a good pixel with a usable map value
    bool run;                 // ... and the ranking kept a candidate
    int ci, cj;               // the rounded map: the window centre
    float Wv;
    int c0, y0, x0, base0;    // c0, its reference pixel and flat index
    bool safe9;               // every shift's reads of the 3x3 stay on the grid
    bool in9[9];              // 3x3 point inside the window
    int nxk;
    int xid[NX], xy[NX], xx[NX], xbase[NX];
    bool xsafe[NX];
};

template <int XK>
__device__ __forceinline__ void pix_setup(const RescoreArgs &a, size_t pix, bool inb, PixCands<XK> &pc) {
    const size_t P = (size_t)a.ny * a.nx;
    const int wxn = 2 * a.Sx + 1;
    pc.act = false;
    pc.ci = pc.cj = 0;
    pc.Wv = 0.0f;
    if (inb) {
        if (!a.mask[pix]) {
            if (a.err_out) a.err_out[pix] = __int_as_float(0x7fc00000);
        } else {
            const double u0 = a.u[pix], u1 = a.u[P + pix];
            if (!isfinite(u0) || !isfinite(u1)) {
                atomicOr(&a.hdr->status, PXST_DEV_NONFINITE_U);
            } else if (fabs(u0) > kMaxCoord || fabs(u1) > kMaxCoord) {
                atomicOr(&a.hdr->status, PXST_DEV_U_RANGE);
            } else if (!(a.W[pix] > 0.0f) || !isfinite(a.W[pix])) {
                // not a usable whitefield value: the pixel is left as a masked one
                atomicOr(&a.hdr->status, PXST_DEV_BAD_INPUT);
                if (a.err_out) a.err_out[pix] = __int_as_float(0x7fc00000);
            } else {
                pc.ci = (int)floor(u0 + 0.5);
                pc.cj = (int)floor(u1 + 0.5);
                pc.Wv = a.W[pix];
                pc.act = true;
            }
        }
    }
    pc.c0 = -1;
    pc.nxk = 0;
    if (pc.act) {
        pc.c0 = a.cand[pix * kTopK];
#pragma unroll
        for (int m = 1; m <= XK; ++m) {
            const int idx = m < a.ncand ? a.cand[pix * kTopK + m] : -1;
            const bool far =
                idx >= 0 && pc.c0 >= 0 && (abs(idx / wxn - pc.c0 / wxn) > 1 || abs(idx % wxn - pc.c0 % wxn) > 1);
#pragma unroll
            for (int q = 0; q < XK; ++q)
                if (q == pc.nxk && far) pc.xid[q] = idx;
            pc.nxk += far ? 1 : 0;
        }
    }
    pc.run = pc.act && pc.c0 >= 0;
    const int a0 = pc.run ? pc.c0 / wxn : 0, b0 = pc.run ? pc.c0 % wxn : 0;
    pc.y0 = pc.ci + a0 - a.Sy;
    pc.x0 = pc.cj + b0 - a.Sx;
    pc.base0 = pc.y0 * a.Rx + pc.x0;
    pc.safe9 = pc.run && span_safe(a, pc.y0 - 1, pc.y0 + 1, pc.x0 - 1, pc.x0 + 1);
#pragma unroll
    for (int jn = 0; jn < 9; ++jn) {
        const int na = a0 + jn / 3 - 1, nb = b0 + jn % 3 - 1;
        pc.in9[jn] = pc.run && na >= 0 && na <= 2 * a.Sy && nb >= 0 && nb < wxn;
    }
#pragma unroll
    for (int q = 0; q < XK; ++q) {
        const bool on = pc.run && q < pc.nxk;
        pc.xy[q] = on ? pc.ci + pc.xid[q] / wxn - a.Sy : pc.y0;      // unused: c0 (a harmless read)
        pc.xx[q] = on ? pc.cj + pc.xid[q] % wxn - a.Sx : pc.x0;
        pc.xbase[q] = pc.xy[q] * a.Rx + pc.xx[q];
        pc.xsafe[q] = on ? span_safe(a, pc.xy[q], pc.xy[q], pc.xx[q], pc.xx[q]) : pc.safe9;
    }
}

// Every candidate the pixel evaluates (the whole 3x3 and the other kept ones) lies on the
// reference grid, is valid in every frame (its validity count is N) and reads on the grid
// for every shift: the lean kernel may skip the per-frame rule.
template <int XK>
__device__ __forceinline__ bool pix_lean(const RescoreArgs &a, const PixCands<XK> &pc) {
    if (!pc.run) return true;
    bool ok = pc.safe9 && pc.y0 >= 1 && pc.y0 + 1 < a.Ry && pc.x0 >= 1 && pc.x0 + 1 < a.Rx;
    if (!ok) return false;
#pragma unroll
    for (int jn = 0; jn < 9; ++jn)
        ok = ok && __ldg(a.nvalid + pc.base0 + (jn / 3 - 1) * a.Rx + (jn % 3 - 1)) == a.N;
#pragma unroll
    for (int q = 0; q < XK; ++q)
        if (q < pc.nxk)
            ok = ok && pc.xsafe[q] && (unsigned)pc.xy[q] < (unsigned)a.Ry && (unsigned)pc.xx[q] < (unsigned)a.Rx &&
                 __ldg(a.nvalid + pc.xbase[q]) == a.N;
    return ok;
}

// The lexicographic minimum over the evaluated candidates (f9: the 3x3 about c0, +inf
// outside the window; fx: the other kept ones), the 3x3 about it when it is not c0
// (evaluated here, frames from global memory), the FP64 fit and the outputs.
template <int XK>
__device__ __forceinline__ void pix_finish(const RescoreArgs &a, size_t pix, const PixCands<XK> &pc, float (&f9)[9],
                                           const float (&fx)[PixCands<XK>::NX]) {
    const size_t P = (size_t)a.ny * a.nx;
    const int wxn = 2 * a.Sx + 1;
    unsigned long long key = ~0ull;
    if (pc.run) {
#pragma unroll
        for (int jn = 0; jn < 9; ++jn)
            if (pc.in9[jn]) key = min(key, pack_key(f9[jn], pc.c0 + (jn / 3 - 1) * wxn + (jn % 3 - 1)));
#pragma unroll
        for (int q = 0; q < XK; ++q)
            if (q < pc.nxk) key = min(key, pack_key(fx[q], pc.xid[q]));
    }
    const float be = __uint_as_float((unsigned int)(key >> 32));
    if (!(be < INFINITY)) {
        // NaN errors of evaluated candidates come only from a non-finite frame value
        if (pc.run && be != be) atomicOr(&a.hdr->status, PXST_DEV_BAD_INPUT);
        if (a.err_out) a.err_out[pix] = INFINITY;
        return;
    }
    const int bi = (int)(key & 0xffffffffu);
    const int ia = bi / wxn, ib = bi % wxn;
    double da = 0.0, db = 0.0;
    if (a.quadratic) {
        if (bi != pc.c0) {
            // the minimum moved off the evaluated 3x3: the second pass (k_rescore_second)
            // evaluates the 3x3 about it, fits and writes the map
            const int k = atomicAdd(&a.hdr->n_second, 1);
            reinterpret_cast<int4 *>(a.second)[k] = make_int4((int)pix, bi, __float_as_int(be), 0);
            if (a.err_out) a.err_out[pix] = be;
            return;
        }
        refine3x3(f9, da, db);
    }
    a.u[pix] = (double)(pc.ci + ia - a.Sy) + da;
    a.u[P + pix] = (double)(pc.cj + ib - a.Sx) + db;
    if (a.err_out) a.err_out[pix] = be;
}

// Lean rescore: one CTA per tile of RT_TY detector rows x 32 columns, one thread per pixel,
// for the pixels that pass pix_lean; a pixel that does not is appended to the list of
// k_rescore_general. The reference the 3x3s of the tile's pixels read (their bounding box,
// widened by the range of the integer frame shifts and one corner) is staged once in shared
// memory when it fits the CTA's share, so that each frame's reads of the 3x3 are
// shared-memory loads rather than L1 hits (the other kept candidates are read through the
// cache); otherwise the 3x3 is read from the masked reference too. Each thread streams its own
// pixel's frames through an 8-deep register double buffer. For a whole-pixel shift the 3x3
// is read as three rows of three about one index; every 3x3 point is summed (those outside
// the window are dropped at the end) and the variance is the pixel's own over all frames.
constexpr int RT_TY = 8;                      // detector rows per tile (one warp each)
constexpr int RT_THREADS = 32 * RT_TY;
constexpr int RT_PREFETCH = 8;                // frames in flight per thread
constexpr int RT_SMEM = 72 * 1024;            // dynamic shared memory per CTA: three CTAs per SM

// R at window index q for the shift's fraction (fy, fx), by the masked renormalised rule with
// the arithmetic of gather_rm (corners NaN where uncovered); false: no valid corner.
__device__ __forceinline__ bool gather_win(const float *__restrict__ src, int stride, int q, float fy, float fx,
                                           float &R) {
    const float wt[4] = {(1.0f - fy) * (1.0f - fx), (1.0f - fy) * fx, fy * (1.0f - fx), fy * fx};
    const int off[4] = {0, 1, stride, stride + 1};
    float num = 0.0f, den = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (wt[k] == 0.0f) continue;
        const float r = src[q + off[k]];
        if (r != r) continue;
        num = fmaf(wt[k], r, num);
        den += wt[k];
    }
    if (!(den > 0.0f)) return false;
    R = num / den;
    return true;
}

// The frame loop of k_rescore_tile: sums, over every frame, the errors of the 3x3 about c0
// (acc[0..3] in pairs, acc[4] = (ninth point, variance)) and of the other kept candidates
// (ex), reading the reference at window index base + the frame's shift from `src` (the
// staged window, pitch WS, or the masked reference, pitch Rx). Frames stream through a
// register double buffer RT_PREFETCH deep.
template <int XK>
__device__ __forceinline__ void rescore_frames(const RescoreArgs &a, const PixCands<XK> &pc,
                                               const float *__restrict__ src, int WS, int base0, int nxw,
                                               const FrameShift *__restrict__ sh, size_t pix, float2 (&acc)[5],
                                               float (&ex)[PixCands<XK>::NX]) {
    const size_t P = (size_t)a.ny * a.nx;
#pragma unroll
    for (int k = 0; k < 5; ++k) acc[k] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int q = 0; q < XK; ++q) ex[q] = 0.0f;
    const float Wv = pc.Wv;
    const float2 nW2 = make_float2(-Wv, -Wv);
    const bool run = pc.run;
    const float *fp = a.frames + pix;
    float In[RT_PREFETCH];
#pragma unroll
    for (int jf = 0; jf < RT_PREFETCH; ++jf) In[jf] = (run && jf < a.N) ? __ldcs(fp + (size_t)jf * P) : 0.0f;
    for (int n0 = 0; n0 < a.N; n0 += RT_PREFETCH) {
        float Iv[RT_PREFETCH];
#pragma unroll
        for (int jf = 0; jf < RT_PREFETCH; ++jf) {
            Iv[jf] = In[jf];
            const int m = n0 + RT_PREFETCH + jf;
            In[jf] = (run && m < a.N) ? __ldcs(fp + (size_t)m * P) : 0.0f;
        }
        if (!run) continue;
#pragma unroll
        for (int jf = 0; jf < RT_PREFETCH; ++jf) {
            if (n0 + jf >= a.N) break;                      // uniform over the CTA
            const FrameShift sft = sh[n0 + jf];
            const float I = Iv[jf];
            const float2 I2 = make_float2(I, I);
            const int off = sft.ky * WS + sft.kx;
            if (sft.fy == 0.0f && sft.fx == 0.0f) {         // the same for every lane
                const float *r0 = src + (base0 + off);
                const float *rm = r0 - WS, *rp = r0 + WS;
                const float R[9] = {rm[-1], rm[0], rm[1], r0[-1], r0[0], r0[1], rp[-1], rp[0], rp[1]};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float2 d = __ffma2_rn(nW2, make_float2(R[2 * k], R[2 * k + 1]), I2);
                    acc[k] = __ffma2_rn(d, d, acc[k]);
                }
                // (I - W R8, I - W): the last point and the variance term
                const float2 d8 = __ffma2_rn(nW2, make_float2(R[8], 1.0f), I2);
                acc[4] = __ffma2_rn(d8, d8, acc[4]);
#pragma unroll
                for (int q = 0; q < XK; ++q) {
                    if (q >= nxw) break;
                    const float d = fmaf(-Wv, __ldg(a.Rm + (pc.xbase[q] + sft.ky * a.Rx + sft.kx)), I);
                    ex[q] = fmaf(d, d, ex[q]);
                }
            } else {
                const float tt = I - Wv;
                acc[4].y = fmaf(tt, tt, acc[4].y);
                // a fractional shift: the masked bilinear read (valid: the counts are N)
#pragma unroll
                for (int jn = 0; jn < 9; ++jn) {
                    float R;
                    if (gather_win(src, WS, base0 + off + (jn / 3 - 1) * WS + (jn % 3 - 1), sft.fy, sft.fx, R)) {
                        const float d = fmaf(-Wv, R, I);
                        float &e = (jn & 1) ? acc[jn >> 1].y : acc[jn >> 1].x;
                        e = fmaf(d, d, e);
                    }
                }
#pragma unroll
                for (int q = 0; q < XK; ++q) {
                    if (q >= nxw) break;
                    float R;
                    if (gather_rm(a.Rm, a.Ry, a.Rx, pc.xy[q] + sft.ky, pc.xx[q] + sft.kx, sft.fy, sft.fx, R)) {
                        const float d = fmaf(-Wv, R, I);
                        ex[q] = fmaf(d, d, ex[q]);
                    }
                }
            }
        }
    }
}

// The frame loop for scans whose translations are all whole pixels, reading the staged
// window: per frame one shared-memory offset and the reads at c0's 3x3 and the other kept
// candidates, no per-frame test; 16 frames per chunk without a bound check inside it, so
// the compiler can overlap one frame's reads with the previous frame's arithmetic.
template <int XK>
__device__ __forceinline__ void rescore_frames_int(const RescoreArgs &a, const PixCands<XK> &pc,
                                                   const float *__restrict__ win, const int *__restrict__ offs,
                                                   const int *__restrict__ offg, int WS, int base0, int nxw,
                                                   size_t pix, float2 (&acc)[5], float (&ex)[PixCands<XK>::NX]) {
    const size_t P = (size_t)a.ny * a.nx;
#pragma unroll
    for (int k = 0; k < 5; ++k) acc[k] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int q = 0; q < XK; ++q) ex[q] = 0.0f;
    const float Wv = pc.Wv;
    const float2 nW2 = make_float2(-Wv, -Wv);
    const bool run = pc.run;
    const float *fp = a.frames + pix;
    const float *c0 = win + base0;
    auto one = [&](float I, int off, int og) {
        const float2 I2 = make_float2(I, I);
        const float *r0 = c0 + off;
        const float R[9] = {r0[-WS - 1], r0[-WS], r0[-WS + 1], r0[-1], r0[0], r0[1], r0[WS - 1], r0[WS], r0[WS + 1]};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 d = __ffma2_rn(nW2, make_float2(R[2 * k], R[2 * k + 1]), I2);
            acc[k] = __ffma2_rn(d, d, acc[k]);
        }
        const float2 d8 = __ffma2_rn(nW2, make_float2(R[8], 1.0f), I2);
        acc[4] = __ffma2_rn(d8, d8, acc[4]);
#pragma unroll
        for (int q = 0; q < XK; ++q) {
            if (q >= nxw) break;
            const float d = fmaf(-Wv, __ldg(a.Rm + (pc.xbase[q] + og)), I);
            ex[q] = fmaf(d, d, ex[q]);
        }
    };
    float In[RT_PREFETCH];
#pragma unroll
    for (int jf = 0; jf < RT_PREFETCH; ++jf) In[jf] = (run && jf < a.N) ? __ldcs(fp + (size_t)jf * P) : 0.0f;
    int n0 = 0;
    for (; n0 + RT_PREFETCH <= a.N; n0 += RT_PREFETCH) {
        float Iv[RT_PREFETCH];
#pragma unroll
        for (int jf = 0; jf < RT_PREFETCH; ++jf) {
            Iv[jf] = In[jf];
            const int m = n0 + RT_PREFETCH + jf;
            In[jf] = (run && m < a.N) ? __ldcs(fp + (size_t)m * P) : 0.0f;
        }
        if (!run) continue;
#pragma unroll
        for (int jf = 0; jf < RT_PREFETCH; ++jf) one(Iv[jf], offs[n0 + jf], offg[n0 + jf]);
    }
    if (run)
        for (int jf = 0; n0 + jf < a.N; ++jf) one(In[jf], offs[n0 + jf], offg[n0 + jf]);
}

template <int XK>
__global__ void __launch_bounds__(RT_THREADS, XK <= 3 ? 3 : 2) k_rescore_tile(RescoreArgs a, int win_cap, int sh_staged) {
    extern __shared__ __align__(16) unsigned char rt_raw[];
    FrameShift *s_sh = reinterpret_cast<FrameShift *>(rt_raw);
    int *s_off = reinterpret_cast<int *>(s_sh + (sh_staged ? a.N : 0));     // whole-pixel shifts: window offsets
    int *s_offg = s_off + (sh_staged ? a.N : 0);                             // ... and offsets in the reference
    float *s_win = reinterpret_cast<float *>(s_offg + (sh_staged ? a.N : 0));
    const FrameShift *sh = sh_staged ? s_sh : a.shifts;
    __shared__ int s_box[4];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int x = blockIdx.x * 32 + lane, y = blockIdx.y * RT_TY + wid;
    const bool inb = x < a.nx && y < a.ny;
    const size_t pix = inb ? (size_t)y * a.nx + x : 0;
    if (threadIdx.x < 4) s_box[threadIdx.x] = (threadIdx.x & 1) ? INT_MIN : INT_MAX;
    if (sh_staged)
        for (int n = threadIdx.x; n < a.N; n += RT_THREADS) s_sh[n] = a.shifts[n];
    PixCands<XK> pc;
    pix_setup<XK>(a, pix, inb, pc);
    // a pixel with an evaluated candidate that is not valid in every frame (near the edge of
    // the reference's coverage) is left to the general kernel's per-frame rule, so that every
    // warp here runs the lean loop and an edge tile takes no longer than any other
    if (pc.run && !pix_lean<XK>(a, pc)) {
        a.wlist[atomicAdd(&a.hdr->n_rescore_pix, 1)] = (int)pix;
        pc.act = pc.run = false;
    }
    __syncthreads();
    // the box of the 3x3s about the tile's first candidates (the other kept candidates, a
    // few per pixel anywhere in the window, are read through the cache)
    if (pc.run) {
        atomicMin(&s_box[0], pc.y0 - 1); atomicMax(&s_box[1], pc.y0 + 1);
        atomicMin(&s_box[2], pc.x0 - 1); atomicMax(&s_box[3], pc.x0 + 1);
    }
    __syncthreads();
    const bool any = s_box[0] != INT_MAX;
    // the window: the box widened by the shifts' integer range (+1 row and column for the
    // second corner of a fractional shift); cells off the grid are NaN (not valid)
    const int wy0 = any ? s_box[0] + a.hdr->kmin_y : 0, wy1 = any ? s_box[1] + a.hdr->kmax_y + 1 : 0;
    const int wx0 = any ? s_box[2] + a.hdr->kmin_x : 0, wx1 = any ? s_box[3] + a.hdr->kmax_x + 1 : 0;
    long long WSl = (long long)wx1 - wx0 + 1;
    WSl += (WSl & 1) ? 0 : 1;                       // odd row pitch: rows read by a warp spread over banks
    const long long WHl = (long long)wy1 - wy0 + 1;
    const bool staged = sh_staged && any && WSl * WHl <= win_cap;
    const int WS = staged ? (int)WSl : a.Rx;
    if (staged) {
        const int WN = (int)(WSl * WHl);
        const float qnan = __int_as_float(0x7fc00000);
        for (int idx = threadIdx.x; idx < WN; idx += RT_THREADS) {
            const int gy = wy0 + idx / WS, gx = wx0 + idx % WS;
            s_win[idx] = (gy >= 0 && gy < a.Ry && gx >= 0 && gx < a.Rx) ? __ldg(a.Rm + (size_t)gy * a.Rx + gx) : qnan;
        }
        for (int n = threadIdx.x; n < a.N; n += RT_THREADS) {
            s_off[n] = s_sh[n].ky * WS + s_sh[n].kx;
            s_offg[n] = s_sh[n].ky * a.Rx + s_sh[n].kx;
        }
    }
    __syncthreads();
    if (!pc.act) return;
    // window index of c0 for a zero shift
    const int base0 = staged ? (pc.y0 - wy0) * WS + (pc.x0 - wx0) : pc.base0;
    float f9[9], fxe[PixCands<XK>::NX];
    {
        const int nxw = __reduce_max_sync(__activemask(), pc.nxk);
        // the 3x3 errors in pairs, (e9[2k], e9[2k+1]) = acc[k], and acc[4] = (e9[8], var): one
        // packed FMA advances two sums
        float2 acc[5];
        float ex[PixCands<XK>::NX];
        // whole-pixel translations only (one fraction class, zero): the loop without tests
        const bool whole = a.hdr->n_classes == 1 && a.hdr->cls_fy[0] == 0.0f && a.hdr->cls_fx[0] == 0.0f;
        // staged: shared-memory loads from the window (a pointer the compiler knows is shared)
        if (staged && whole)
            rescore_frames_int<XK>(a, pc, s_win, s_off, s_offg, WS, base0, nxw, pix, acc, ex);
        else if (staged)
            rescore_frames<XK>(a, pc, s_win, WS, base0, nxw, sh, pix, acc, ex);
        else
            rescore_frames<XK>(a, pc, a.Rm, WS, base0, nxw, sh, pix, acc, ex);
        // every evaluated candidate was valid in all N frames: e = err / var (err if var = 0)
        const float var = acc[4].y;
#pragma unroll
        for (int jn = 0; jn < 9; ++jn) {
            const float e = (jn & 1) ? acc[jn >> 1].y : acc[jn >> 1].x;
            f9[jn] = pc.in9[jn] ? (var > 0.0f ? e / var : e) : INFINITY;
        }
#pragma unroll
        for (int q = 0; q < XK; ++q) fxe[q] = q < pc.nxk ? (var > 0.0f ? ex[q] / var : ex[q]) : INFINITY;
    }
    pix_finish<XK>(a, pix, pc, f9, fxe);
}

// General rescore: one block per 32 pixels listed by k_rescore_tile (blocks beyond the list's
// length return at once), with the per-frame rule of the masked renormalised reads: each
// candidate sums its error and variance over the frames where it is valid. The block's 4
// warps take the same 32 pixels and a quarter of the frames each (so that the few listed
// pixels still fill the GPU); their sums are added in warp order and warp 0 finishes.
constexpr int RG_W = 4;
template <int XK>
__global__ void __launch_bounds__(32 * RG_W) k_rescore_general(RescoreArgs a) {
    constexpr int NC = 9 + PixCands<XK>::NX;                      // candidates per pixel
    constexpr int STAGE_BYTES = RG_W * RS_S * RS_F * 32 * 4;       // frames, per warp
    constexpr int SUM_BYTES = (RG_W - 1) * NC * 32 * 12;           // partial sums, warps 1..
    __shared__ __align__(16) uint8_t sraw[STAGE_BYTES > SUM_BYTES ? STAGE_BYTES : SUM_BYTES];
    const int n_list = a.hdr->n_rescore_pix;
    if ((int)blockIdx.x * 32 >= n_list) return;
    const size_t P = (size_t)a.ny * a.nx;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int idx = blockIdx.x * 32 + lane;
    const bool inb = idx < n_list;
    const size_t pix = (size_t)a.wlist[inb ? idx : blockIdx.x * 32];
    PixCands<XK> pc;
    pix_setup<XK>(a, pix, inb, pc);
    CandSums s9[9], sx[PixCands<XK>::NX];
#pragma unroll
    for (int jn = 0; jn < 9; ++jn) s9[jn].zero();
#pragma unroll
    for (int q = 0; q < XK; ++q) sx[q].zero();
    const float Wv = pc.Wv;
    // this warp's frames [fb, fe), staged in its own part of the buffer, column = lane
    float(*sfr)[RS_F][32] = reinterpret_cast<float(*)[RS_F][32]>(sraw) + wid * RS_S;
    const int qn = (a.N + RG_W - 1) / RG_W;
    const int fb = min(a.N, wid * qn), fe = min(a.N, fb + qn);
    const int nst = (fe - fb + RS_F - 1) / RS_F;
    auto issue = [&](int st) {
        if (st < nst && pc.run) {
            const int buf = st % RS_S;
#pragma unroll
            for (int f = 0; f < RS_F; ++f) {
                const int n = fb + st * RS_F + f;
                if (n < fe) cp_async4(&sfr[buf][f][lane], a.frames + (size_t)n * P + pix);
            }
        }
        cp_async_commit();
    };
#pragma unroll
    for (int st = 0; st < RS_S - 1; ++st) issue(st);
    for (int st = 0; st < nst; ++st) {
        issue(st + RS_S - 1);
        cp_async_wait<RS_S - 1>();
        const int buf = st % RS_S;
        if (pc.run) {
            const int nf = min(RS_F, fe - fb - st * RS_F);
            for (int f = 0; f < nf; ++f) {
                const FrameShift s = a.shifts[fb + st * RS_F + f];
                const float I = sfr[buf][f][lane];
                const float tt = I - Wv;
#pragma unroll
                for (int jn = 0; jn < 9; ++jn) {
                    if (!pc.in9[jn]) continue;
                    const int dy = jn / 3 - 1, dx = jn % 3 - 1;
                    float R;
                    const bool ok = read_any(a, pc.y0 + dy, pc.x0 + dx, pc.base0 + dy * a.Rx + dx, pc.safe9, s, R);
                    s9[jn].add(ok, R, I, tt, Wv);
                }
#pragma unroll
                for (int q = 0; q < XK; ++q) {
                    if (q >= pc.nxk) continue;
                    float R;
                    const bool ok = read_any(a, pc.xy[q], pc.xx[q], pc.xbase[q], pc.xsafe[q], s, R);
                    sx[q].add(ok, R, I, tt, Wv);
                }
            }
        }
    }
    cp_async_wait<0>();
    __syncthreads();                                   // every warp is done with its frames
    // partial sums of warps 1.. : [warp - 1][candidate][lane] (err, var, nv)
    float *se = reinterpret_cast<float *>(sraw);
    float *sv = se + (RG_W - 1) * NC * 32;
    int *sn = reinterpret_cast<int *>(sv + (RG_W - 1) * NC * 32);
    if (wid > 0) {
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const CandSums &c = k < 9 ? s9[k] : sx[k < 9 + XK ? k - 9 : 0];
            const int o = ((wid - 1) * NC + k) * 32 + lane;
            se[o] = c.err;
            sv[o] = c.var;
            sn[o] = c.nv;
        }
    }
    __syncthreads();
    if (wid > 0 || !pc.act) return;
#pragma unroll
    for (int w = 1; w < RG_W; ++w) {
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            if (k >= 9 + XK) break;
            CandSums &c = k < 9 ? s9[k] : sx[k - 9];
            const int o = ((w - 1) * NC + k) * 32 + lane;
            c.err += se[o];
            c.var += sv[o];
            c.nv += sn[o];
        }
    }
    float f9[9], fxe[PixCands<XK>::NX];
#pragma unroll
    for (int jn = 0; jn < 9; ++jn) f9[jn] = pc.in9[jn] ? s9[jn].e() : INFINITY;
#pragma unroll
    for (int q = 0; q < XK; ++q) fxe[q] = q < pc.nxk ? sx[q].e() : INFINITY;
    pix_finish<XK>(a, pix, pc, f9, fxe);
}

// Second pass of the rescore: the pixels whose minimum left the first 3x3 (a few hundred in a
// megapixel), one warp per listed pixel. The lanes split the frames (n = lane, lane + 32, ...)
// and sum, by the per-frame rule, the 8 points of the 3x3 about the minimum; the warp adds
// the lanes' sums in a fixed butterfly order; lane 0 fits and writes the map. (Evaluated
// inside the tile kernels instead, one thread running 8 candidates through every frame held
// its whole CTA for about ten times a typical CTA's duration.)
__global__ void __launch_bounds__(256) k_rescore_second(RescoreArgs a) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    const size_t P = (size_t)a.ny * a.nx;
    const int wxn = 2 * a.Sx + 1;
    const int n_list = a.hdr->n_second;
    for (int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); e < n_list; e += nw) {
        const int4 ent = reinterpret_cast<const int4 *>(a.second)[e];
        const size_t pix = (size_t)ent.x;
        const int bi = ent.y;
        const float be = __int_as_float(ent.z);
        // the window centre of the map before this update (the map is written below only)
        const int ci = (int)floor(a.u[pix] + 0.5), cj = (int)floor(a.u[P + pix] + 0.5);
        const float Wv = a.W[pix];
        const int ia = bi / wxn, ib = bi % wxn;
        int cy[8], cx[8], base[8];
        bool in[8], safe[8];
        CandSums cs[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int jn = k < 4 ? k : k + 1;
            const int na = ia + jn / 3 - 1, nb = ib + jn % 3 - 1;
            in[k] = na >= 0 && na <= 2 * a.Sy && nb >= 0 && nb < wxn;
            cy[k] = ci + na - a.Sy;
            cx[k] = cj + nb - a.Sx;
            base[k] = cy[k] * a.Rx + cx[k];
            safe[k] = span_safe(a, cy[k], cy[k], cx[k], cx[k]);
            cs[k].zero();
        }
        for (int n = lane; n < a.N; n += 32) {
            const FrameShift sft = a.shifts[n];
            const float I = __ldcs(a.frames + (size_t)n * P + pix);
            const float t = I - Wv;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (!in[k]) continue;
                float R = 0.0f;
                const bool ok = read_any(a, cy[k], cx[k], base[k], safe[k], sft, R);
                cs[k].add(ok, R, I, t, Wv);
            }
        }
        float f9[9];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float er = cs[k].err, va = cs[k].var;
            int nv = cs[k].nv;
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) {
                er += __shfl_xor_sync(0xffffffffu, er, m);
                va += __shfl_xor_sync(0xffffffffu, va, m);
                nv += __shfl_xor_sync(0xffffffffu, nv, m);
            }
            const int jn = k < 4 ? k : k + 1;
            f9[jn] = !in[k] ? INFINITY : (nv == 0 ? INFINITY : (va > 0.0f ? er / va : er));
        }
        f9[4] = be;
        if (lane == 0) {
            double da = 0.0, db = 0.0;
            refine3x3(f9, da, db);
            a.u[pix] = (double)(ci + ia - a.Sy) + da;
            a.u[P + pix] = (double)(cj + ib - a.Sx) + db;
        }
    }
}

}  // namespace

// Largest frame count the fast path can stage (a 1 x 32 tile in shared memory).
int search_max_frames() { return (kSearchSmemBudget - 16 * 1024) / (36 * 4 + 16); }

cudaError_t launch_search(const pxst_dims &d, const pxst_options &o, const float *frames,
                          const float *W, const uint8_t *mask, const float *I_ref,
                          const float *w, const FrameShift *shifts, WsHeader *hdr,
                          int *exact_list, double *u, float *err_out, int span_y, int span_x,
                          cudaStream_t stream) {
    Plan pl;
    const int wxn = 2 * o.win_x + 1;
    const size_t nwin = (size_t)(2 * o.win_y + 1) * wxn;
    // strip length: requested (tile bits 4-5: 1, 2, 3 = 7, 9, 11 columns) or the least waste
    const int ty_req = o.tile & 15, l_req = o.tile >> 4;
    pl.L = l_req == 1 ? 7 : l_req == 2 ? 9 : l_req == 3 ? 11 : pick_strip(wxn);
    const size_t N = (size_t)d.n_frames, shifts_b = N * sizeof(FrameShift);
    const size_t sm_per_sm = 228 * 1024;
    // window estimate for a local magnification up to 2 (unknown span: the largest window)
    auto window_est = [&](int ty) -> size_t {
        if (span_y < 0 || span_x < 0) return (size_t)kSearchSmemBudget;
        const size_t rows = 2 * ty + 2 * o.win_y + span_y + 4;
        const size_t cols = 64 + wxn + pl.L + span_x + 6;
        return rows * cols * 4;
    };
    // Choose (tile height, error buffer) for the most resident CTAs per SM, then prefer
    // keeping the errors (no 3x3 re-evaluation), then taller tiles; the window gets the
    // rest of the CTA's share of shared memory.
    int best_score = -1;
    pl.TY = 1;
    pl.smem = 0;
    int best_ebuf = 0;
    for (int ebuf = 1; ebuf >= 0; --ebuf)
        for (int ty = 8; ty >= 1; ty >>= 1) {
            if (ty_req > 0 && ty != ty_req) continue;          // a requested tile height
            size_t st = 0;
            int cr = 1;
            cudaError_t e = variant_info_any(pl.L, ty, st, cr);
            if (e != cudaSuccess) return e;
            const size_t fixed = shifts_b + N * (32 * ty + 4) * 4 + (ebuf ? (size_t)32 * ty * nwin * 4 : 0);
            for (int k = 3; k >= 1; --k) {
                if (k > cr) continue;
                size_t per_cta = sm_per_sm / k - 1024 - st;
                if (per_cta > (size_t)kSearchSmemBudget) per_cta = kSearchSmemBudget;
                const size_t need = fixed + window_est(ty);
                if (need > per_cta && !(k == 1 && fixed + 4096 <= per_cta && window_est(ty) >= (size_t)kSearchSmemBudget))
                    continue;
                const int score = k * 100 + ebuf * 10 + ty;
                if (score > best_score) {
                    best_score = score;
                    pl.TY = ty;
                    best_ebuf = ebuf;
                    pl.smem = per_cta;
                }
                break;
            }
        }
    if (best_score < 0 && ty_req > 0) {
        // the requested height does not fit: the automatic height (the strip length kept)
        pxst_options o2 = o;
        o2.tile = o.tile & ~15;
        return launch_search(d, o2, frames, W, mask, I_ref, w, shifts, hdr, exact_list, u, err_out, span_y, span_x,
                             stream);
    }
    if (best_score < 0) return cudaErrorInvalidConfiguration;   // callers check frame count first
    const size_t fixed = shifts_b + N * (32 * pl.TY + 4) * 4 + (best_ebuf ? (size_t)32 * pl.TY * nwin * 4 : 0);
    pl.win_cap = (int)((pl.smem - fixed) / 4);

    SearchArgs a;
    a.N = d.n_frames; a.ny = d.ny; a.nx = d.nx; a.Ry = d.ref_ny; a.Rx = d.ref_nx;
    a.Sy = o.win_y; a.Sx = o.win_x; a.quadratic = o.quadratic ? 1 : 0;
    a.ebuf = best_ebuf; a.win_cap = pl.win_cap;
    a.frames = frames; a.W = W; a.mask = mask; a.Iref = I_ref; a.w = w; a.shifts = shifts;
    a.hdr = hdr; a.exact_list = exact_list; a.u = u; a.err_out = err_out;
    switch (pl.L) {
        case 11: return launch_L<11>(a, pl, stream);
        case 9: return launch_L<9>(a, pl, stream);
        default: return launch_L<7>(a, pl, stream);
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
    k_exact<<<device_sms() * 4, 256, 0, stream>>>(a); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_rescore(const pxst_dims &d, const pxst_options &o, int ncand, const float *frames,
                           const float *W, const uint8_t *mask, const float *Rm, const int *nvalid,
                           const FrameShift *shifts, const int *cand, WsHeader *hdr, int *wlist, int *second,
                           double *u, float *err_out, cudaStream_t stream) {
    RescoreArgs a;
    a.N = d.n_frames; a.ny = d.ny; a.nx = d.nx; a.Ry = d.ref_ny; a.Rx = d.ref_nx;
    a.Sy = o.win_y; a.Sx = o.win_x; a.quadratic = o.quadratic ? 1 : 0; a.ncand = ncand;
    a.frames = frames; a.W = W; a.mask = mask; a.Rm = Rm; a.nvalid = nvalid; a.shifts = shifts;
    a.cand = cand; a.hdr = hdr; a.wlist = wlist; a.second = second; a.u = u; a.err_out = err_out;
    const dim3 tgrid((unsigned)((d.nx + 31) / 32), (unsigned)((d.ny + RT_TY - 1) / RT_TY));
    const unsigned gblocks = (unsigned)(((size_t)d.ny * d.nx + 31) / 32);   // at most one per 32 listed pixels
    // the shift table (when it leaves room) and the window share the CTA's part of shared
    // memory; a window that does not fit is read through the cache
    const long long shifts_b = (long long)(sizeof(FrameShift) + 2 * sizeof(int)) * d.n_frames;
    const int sh_staged = shifts_b <= RT_SMEM / 2 ? 1 : 0;
    const int smem = RT_SMEM;
    const int win_cap = (int)((smem - (sh_staged ? shifts_b : 0)) / 4);
    // n_rescore_pix and n_second
    cudaError_t e = cudaMemsetAsync(&hdr->n_rescore_pix, 0, 2 * sizeof(int), stream);
    if (e != cudaSuccess) return e;
    auto go = [&](auto tile_kernel, auto general_kernel) {
        cudaError_t r = cudaFuncSetAttribute(tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (r != cudaSuccess) return r;
        tile_kernel<<<tgrid, RT_THREADS, smem, stream>>>(a, win_cap, sh_staged); note_launch();
        general_kernel<<<gblocks, 32 * RG_W, 0, stream>>>(a); note_launch();
        if ((r = cudaGetLastError()) != cudaSuccess) return r;
        if (a.quadratic) {
            k_rescore_second<<<device_sms() * 2, 256, 0, stream>>>(a); note_launch();
        }
        return cudaGetLastError();
    };
    return ncand <= 4 ? go(k_rescore_tile<3>, k_rescore_general<3>) : go(k_rescore_tile<7>, k_rescore_general<7>);
}

}  // namespace pxst
