// frames.cu -- figures of merit (section "Calculate figures of merit") and the
// translation update (section "Update translations") on sm_103a.
//
//   k_pixvar      var(x) = sum over the frames valid at u(x) - Delta_n of (I_n - W)^2
//   k_calc_error  eps[n,x] = (I_n - W R_n)^2 / var(x) per pixel and frame: the pixel error
//                 (sum over n), the frame errors (warp sums, FP64 atomics), the total and
//                 the reference-plane error (eps scattered with the bilinear weights to
//                 u - Delta_n, FP64 atomics into the workspace accumulators, then divided
//                 by the weights that landed)
//   k_trans_acc   per frame and integer shift t of its translation: the sum of eps over the
//                 pixels whose read at u - Delta_n - t is valid, and their count (one block
//                 per 256 pixels and frame; warp sums, shared and then FP64 global atomics)
//   k_trans_fit   per frame: the mean, the first minimum, the 3x3 paraboloid, Delta_n update
#include <cmath>

#include "pxst_common.cuh"

namespace pxst {
namespace {

// A coordinate split once per pixel into an integer and an FP32 fraction in [0, 1), so that
// the per-frame arithmetic is integer adds and FP32 (FP64 is a small fraction of FP32 on this
// GPU): u - Delta_n - t = (ui + k_n - t) + (uf + f_n), with -Delta_n = k_n + f_n from the
// prepared shift table.
__device__ __forceinline__ void split_coord(double v, int &i, float &f) {
    double fl = floor(v);
    float fr = (float)(v - fl);
    if (fr >= 1.0f) {              // a fraction just below 1 rounded up in float32
        fr = 0.0f;
        fl += 1.0;
    }
    i = (int)fl;
    f = fr;
}

// corner (i0, j0) and fractions of u - Delta_n - (da, db)
__device__ __forceinline__ void frame_point(int ui0, float uf0, int ui1, float uf1, const FrameShift &s, int da,
                                            int db, int &i0, float &f0, int &j0, float &f1) {
    f0 = uf0 + s.fy;
    i0 = ui0 + s.ky - da;
    if (f0 >= 1.0f) {
        f0 -= 1.0f;
        ++i0;
    }
    f1 = uf1 + s.fx;
    j0 = ui1 + s.kx - db;
    if (f1 >= 1.0f) {
        f1 -= 1.0f;
        ++j0;
    }
}

struct MeritArgs {
    int N, ny, nx, Ry, Rx;
    const float *frames, *W;
    const uint8_t *mask;
    const float *Iref, *w;
    const double *u, *delta;
    const FrameShift *shifts;      // -Delta_n split (prepared from delta)
    float *var;                    // [P] workspace: var(x), -1 where the pixel does not count
    WsHeader *hdr;
};

__global__ void __launch_bounds__(256) k_pixvar(MeritArgs a) {
    const size_t P = (size_t)a.ny * a.nx;
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    float v = -1.0f;
    if (a.mask[p]) {
        const double u0 = a.u[p], u1 = a.u[P + p];
        if (!isfinite(u0) || !isfinite(u1)) {
            atomicOr(&a.hdr->status, PXST_DEV_NONFINITE_U);
        } else if (fabs(u0) > kMaxCoord || fabs(u1) > kMaxCoord) {
            atomicOr(&a.hdr->status, PXST_DEV_U_RANGE);
        } else {
            const float Wv = a.W[p];
            int ui0, ui1;
            float uf0, uf1;
            split_coord(u0, ui0, uf0);
            split_coord(u1, ui1, uf1);
            float s2 = 0.0f;
            for (int n = 0; n < a.N; ++n) {
                int i0, j0;
                float f0, f1, R;
                frame_point(ui0, uf0, ui1, uf1, a.shifts[n], 0, 0, i0, f0, j0, f1);
                if (!gather_masked(a.Iref, a.w, a.Ry, a.Rx, i0, j0, f0, f1, R)) continue;
                const float t = __ldg(a.frames + (size_t)n * P + p) - Wv;
                s2 = fmaf(t, t, s2);
            }
            v = s2;
        }
    }
    a.var[p] = v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

struct ErrorOut {
    float *pixel_err;      // [P] or null
    double *frame_err;     // [N] or null (accumulated: zeroed by the launcher)
    double *total;         // [1] or null (accumulated)
    float *num, *den;      // [R] accumulators of the reference-plane error, or null
};

constexpr int kErrFramesSmem = 6144;   // frame sums kept in shared memory up to this many frames

// Grid-stride over the pixels: each block keeps its partial frame sums in shared memory
// (one warp sum and one shared atomic per warp and frame) and adds them to the output once,
// so that a frame's sum sees one global atomic per block, not one per warp.
__global__ void __launch_bounds__(256) k_calc_error(MeritArgs a, ErrorOut o) {
    extern __shared__ double s_fe[];                  // [N] when N <= kErrFramesSmem
    __shared__ double s_tot[8];
    const size_t P = (size_t)a.ny * a.nx;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool smem_fe = o.frame_err && a.N <= kErrFramesSmem;
    if (smem_fe)
        for (int n = threadIdx.x; n < a.N; n += blockDim.x) s_fe[n] = 0.0;
    __syncthreads();
    double tot = 0.0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t p_end = (P + blockDim.x - 1) / blockDim.x * blockDim.x;   // whole blocks: warp sums
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < p_end; p += stride) {
        const float var = p < P ? a.var[p] : -1.0f;
        const bool act = var >= 0.0f;
        int ui0 = 0, ui1 = 0;
        float uf0 = 0.0f, uf1 = 0.0f, Wv = 0.0f;
        if (act) {
            split_coord(a.u[p], ui0, uf0);
            split_coord(a.u[P + p], ui1, uf1);
            Wv = a.W[p];
        }
        float pe = 0.0f;
        for (int n = 0; n < a.N; ++n) {
            float eps = 0.0f;
            if (act) {
                int i0, j0;
                float fy, fx, R;
                frame_point(ui0, uf0, ui1, uf1, a.shifts[n], 0, 0, i0, fy, j0, fx);
                if (gather_masked(a.Iref, a.w, a.Ry, a.Rx, i0, j0, fy, fx, R)) {
                    const float d = fmaf(-Wv, R, __ldg(a.frames + (size_t)n * P + p));
                    eps = var > 0.0f ? d * d / var : d * d;
                    if (o.num) {
                        // scatter with make_object_map's bilinear weights (corners off the grid dropped)
                        const float wt[4] = {(1.0f - fy) * (1.0f - fx), (1.0f - fy) * fx, fy * (1.0f - fx),
                                             fy * fx};
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int ii = i0 + (k >> 1), jj = j0 + (k & 1);
                            if (wt[k] == 0.0f || ii < 0 || ii >= a.Ry || jj < 0 || jj >= a.Rx) continue;
                            const size_t c = (size_t)ii * a.Rx + jj;
                            atomicAdd(o.num + c, wt[k] * eps);
                            atomicAdd(o.den + c, wt[k]);
                        }
                    }
                }
            }
            pe += eps;
            if (o.frame_err) {
                const double s = warp_sum((double)eps);
                if (lane == 0 && s != 0.0) {
                    if (smem_fe) atomicAdd(s_fe + n, s);
                    else atomicAdd(o.frame_err + n, s);
                }
            }
        }
        if (p < P && o.pixel_err) o.pixel_err[p] = act ? pe : __int_as_float(0x7fc00000);
        tot += act ? (double)pe : 0.0;
    }
    if (o.total) {
        const double s = warp_sum(tot);
        if (lane == 0) s_tot[warp] = s;
    }
    __syncthreads();
    if (o.total && threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += s_tot[k];
        if (t != 0.0) atomicAdd(o.total, t);
    }
    if (smem_fe)
        for (int n = threadIdx.x; n < a.N; n += blockDim.x)
            if (s_fe[n] != 0.0) atomicAdd(o.frame_err + n, s_fe[n]);
}

__global__ void k_err_normalise(int R, const float *__restrict__ num, const float *__restrict__ den,
                                float *__restrict__ ref_err) {
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < (size_t)R; c += (size_t)gridDim.x * blockDim.x)
        ref_err[c] = den[c] > 0.0f ? num[c] / den[c] : 0.0f;
}

struct TransArgs {
    MeritArgs m;
    int Ty, Tx, quadratic;
    double *acc_sum;               // [N][kTransMax] sums of eps
    unsigned long long *acc_cnt;   // [N][kTransMax] pixel counts
    double *delta_out;             // [N][2]
    double *err_out;               // [N] or null
};

__global__ void __launch_bounds__(256) k_trans_acc(TransArgs t) {
    __shared__ double s_sum[kTransMax];
    __shared__ unsigned int s_cnt[kTransMax];
    const MeritArgs &a = t.m;
    const int wx = 2 * t.Tx + 1, nc = (2 * t.Ty + 1) * wx;
    for (int k = threadIdx.x; k < nc; k += blockDim.x) {
        s_sum[k] = 0.0;
        s_cnt[k] = 0u;
    }
    __syncthreads();
    const size_t P = (size_t)a.ny * a.nx;
    const int n = blockIdx.y;
    const int lane = threadIdx.x & 31;
    // a few blocks per frame, each striding over the pixels: a frame's sums see one global
    // atomic per block and shift
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t p_end = (P + blockDim.x - 1) / blockDim.x * blockDim.x;   // whole warps: warp sums
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < p_end; p += stride) {
        const float var = p < P ? a.var[p] : -1.0f;
        const bool act = var > 0.0f;
        int ui0 = 0, ui1 = 0;
        float uf0 = 0.0f, uf1 = 0.0f, I = 0.0f, Wv = 0.0f;
        if (act) {
            split_coord(a.u[p], ui0, uf0);
            split_coord(a.u[P + p], ui1, uf1);
            I = __ldg(a.frames + (size_t)n * P + p);
            Wv = a.W[p];
        }
        const FrameShift sh = a.shifts[n];
        for (int k = 0; k < nc; ++k) {
            const int da = k / wx - t.Ty, db = k % wx - t.Tx;
            float eps = 0.0f;
            unsigned c = 0u;
            int i0, j0;
            float f0, f1, R;
            frame_point(ui0, uf0, ui1, uf1, sh, da, db, i0, f0, j0, f1);
            if (act && gather_masked(a.Iref, a.w, a.Ry, a.Rx, i0, j0, f0, f1, R)) {
                const float d = fmaf(-Wv, R, I);
                eps = d * d / var;
                c = 1u;
            }
            float s = eps;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                s += __shfl_xor_sync(0xffffffffu, s, off);
                c += __shfl_xor_sync(0xffffffffu, c, off);
            }
            if (lane == 0 && c) {
                atomicAdd(&s_sum[k], (double)s);
                atomicAdd(&s_cnt[k], c);
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nc; k += blockDim.x)
        if (s_cnt[k]) {
            atomicAdd(t.acc_sum + (size_t)n * kTransMax + k, s_sum[k]);
            atomicAdd(t.acc_cnt + (size_t)n * kTransMax + k, (unsigned long long)s_cnt[k]);
        }
}

__global__ void k_trans_fit(TransArgs t) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= t.m.N) return;
    const int wy = 2 * t.Ty + 1, wx = 2 * t.Tx + 1, nc = wy * wx;
    const double *S = t.acc_sum + (size_t)n * kTransMax;
    const unsigned long long *Cn = t.acc_cnt + (size_t)n * kTransMax;
    auto e_of = [&](int k) { return Cn[k] ? S[k] / (double)Cn[k] : (double)INFINITY; };
    int best = -1;
    double be = INFINITY;
    for (int k = 0; k < nc; ++k) {
        const double e = e_of(k);
        if (e < be) {              // strict <: the first minimum in row-major order
            be = e;
            best = k;
        }
    }
    double d0 = t.m.delta[2 * n], d1 = t.m.delta[2 * n + 1];
    if (best >= 0) {
        const int ia = best / wx, ib = best % wx;
        double da = 0.0, db = 0.0;
        if (t.quadratic) {
            float f[9];
            for (int q = 0; q < 9; ++q) {
                const int a2 = ia + q / 3 - 1, b2 = ib + q % 3 - 1;
                f[q] = (a2 < 0 || a2 >= wy || b2 < 0 || b2 >= wx) ? INFINITY : (float)e_of(a2 * wx + b2);
            }
            refine3x3(f, da, db);
        }
        d0 += (double)(ia - t.Ty) + da;
        d1 += (double)(ib - t.Tx) + db;
    }
    t.delta_out[2 * n] = d0;
    t.delta_out[2 * n + 1] = d1;
    if (t.err_out) t.err_out[n] = be;
}

MeritArgs merit_args(const pxst_dims &d, const float *frames, const float *W, const uint8_t *mask,
                     const float *I_ref, const float *w, const double *u, const double *delta,
                     const FrameShift *shifts, float *var, WsHeader *hdr) {
    MeritArgs a;
    a.shifts = shifts;
    a.N = d.n_frames; a.ny = d.ny; a.nx = d.nx; a.Ry = d.ref_ny; a.Rx = d.ref_nx;
    a.frames = frames; a.W = W; a.mask = mask; a.Iref = I_ref; a.w = w; a.u = u; a.delta = delta;
    a.var = var; a.hdr = hdr;
    return a;
}

// ---- regularisation of the pixel map (the "sigma" option of the update) --------------------
// u_f = G * (M u) / G * M over the good pixels, the Gaussian truncated at r = floor(4 sigma + 1/2)
// on each axis; separable: a pass along the rows into (num0, num1, den), then along the
// columns. FP64: the map's coordinates (up to thousands of pixels) need 1e-9 relative.
struct FilterArgs {
    int ny, nx, r;
    double inv2s2;                 // 1 / (2 sigma^2)
    const uint8_t *mask;
    double *u;                     // [2][ny][nx] in: the map; out: the filtered map
    double *num;                   // [2][ny][nx] row-pass numerators
    double *den;                   // [ny][nx] row-pass denominators
};

// the 1-D taps g(k), k = 0..r, once per block (FP64 exp is slow on this GPU)
__device__ __forceinline__ void filter_taps(const FilterArgs &f, double *g) {
    for (int k = threadIdx.x; k <= f.r; k += blockDim.x) g[k] = exp(-(double)k * (double)k * f.inv2s2);
    __syncthreads();
}

__global__ void __launch_bounds__(256) k_filter_rows(FilterArgs f) {
    extern __shared__ double g[];
    filter_taps(f, g);
    const size_t P = (size_t)f.ny * f.nx;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(p / f.nx), j = (int)(p % f.nx);
        double n0 = 0.0, n1 = 0.0, dn = 0.0;
        for (int b = -f.r; b <= f.r; ++b) {
            const int jj = j + b;
            if (jj < 0 || jj >= f.nx) continue;
            const size_t q = (size_t)i * f.nx + jj;
            if (!f.mask[q]) continue;
            const double gk = g[b < 0 ? -b : b];
            n0 = fma(gk, f.u[q], n0);
            n1 = fma(gk, f.u[P + q], n1);
            dn += gk;
        }
        f.num[p] = n0;
        f.num[P + p] = n1;
        f.den[p] = dn;
    }
}

__global__ void __launch_bounds__(256) k_filter_cols(FilterArgs f) {
    extern __shared__ double g[];
    filter_taps(f, g);
    const size_t P = (size_t)f.ny * f.nx;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        if (!f.mask[p]) continue;                  // M = 0 keeps its map
        const int i = (int)(p / f.nx), j = (int)(p % f.nx);
        double n0 = 0.0, n1 = 0.0, dn = 0.0;
        for (int a = -f.r; a <= f.r; ++a) {
            const int ii = i + a;
            if (ii < 0 || ii >= f.ny) continue;
            const size_t q = (size_t)ii * f.nx + j;
            const double gk = g[a < 0 ? -a : a];
            n0 = fma(gk, f.num[q], n0);
            n1 = fma(gk, f.num[P + q], n1);
            dn = fma(gk, f.den[q], dn);
        }
        // dn > 0: the pixel itself is good and lies inside its own support
        f.u[p] = n0 / dn;
        f.u[P + p] = n1 / dn;
    }
}

// ---- fractional candidates (the non-integer option of section "Update pixel mapping") -------
// After the integer search (no fit) every pixel's map is its minimum c*; the candidates
// c* + (a, b) / s, |a|, |b| <= s, are evaluated by the masked rule with fractional reads (one
// thread per pixel, one row of 2s + 1 candidates per pass over the frames); u = the first
// minimum in row-major order. A pixel whose c* has no valid frame keeps its map.
constexpr int kFracMax = 8;

struct FracArgs {
    int N, ny, nx, Ry, Rx, sub;
    const float *frames, *W;
    const uint8_t *mask;
    const float *Iref, *w;
    const FrameShift *shifts;
    double *u;
    float *err_out;
};

__global__ void __launch_bounds__(128) k_frac_refine(FracArgs a) {
    const size_t P = (size_t)a.ny * a.nx;
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P || !a.mask[p]) return;
    const double u0 = a.u[p], u1 = a.u[P + p];
    if (!isfinite(u0) || !isfinite(u1) || fabs(u0) > kMaxCoord || fabs(u1) > kMaxCoord) return;
    const int c0 = (int)floor(u0 + 0.5), c1 = (int)floor(u1 + 0.5);
    const float Wv = a.W[p];
    const int wn = 2 * a.sub + 1;
    const float inv = 1.0f / (float)a.sub;
    unsigned long long key = ~0ull;
    float e_centre = INFINITY;
    for (int ia = 0; ia < wn; ++ia) {
        const float fa = (float)(ia - a.sub) * inv;
        float err[2 * kFracMax + 1], var[2 * kFracMax + 1];
        int nv[2 * kFracMax + 1];
#pragma unroll
        for (int k = 0; k < 2 * kFracMax + 1; ++k) {
            err[k] = var[k] = 0.0f;
            nv[k] = 0;
        }
        for (int n = 0; n < a.N; ++n) {
            const FrameShift s = a.shifts[n];
            const float I = __ldg(a.frames + (size_t)n * P + p);
            const float t = I - Wv;
            float fy = fa + s.fy;
            const float gy = floorf(fy);
            fy -= gy;
            const int i0 = c0 + s.ky + (int)gy;
#pragma unroll
            for (int k = 0; k < 2 * kFracMax + 1; ++k) {
                if (k >= wn) continue;
                float fx = (float)(k - a.sub) * inv + s.fx;
                const float gx = floorf(fx);
                fx -= gx;
                float R;
                if (gather_masked(a.Iref, a.w, a.Ry, a.Rx, i0, c1 + s.kx + (int)gx, fy, fx, R)) {
                    const float d = fmaf(-Wv, R, I);
                    err[k] = fmaf(d, d, err[k]);
                    var[k] = fmaf(t, t, var[k]);
                    ++nv[k];
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 2 * kFracMax + 1; ++k) {
            if (k >= wn) continue;
            const float e = nv[k] == 0 ? INFINITY : (var[k] > 0.0f ? err[k] / var[k] : err[k]);
            if (ia == a.sub && k == a.sub) e_centre = e;
            key = min(key, ((unsigned long long)__float_as_uint(e) << 32) | (unsigned)(ia * wn + k));
        }
    }
    if (!(e_centre < INFINITY)) return;               // no valid frame at c*: the map is kept
    const int best = (int)(key & 0xffffffffu);
    a.u[p] = (double)c0 + (double)(best / wn - a.sub) / a.sub;
    a.u[P + p] = (double)c1 + (double)(best % wn - a.sub) / a.sub;
    if (a.err_out) a.err_out[p] = __uint_as_float((unsigned)(key >> 32));
}

// ---- defocus registration (fit_defocus_registration, section "Initialisation") -----------------
// One pair of map scales: u' = u(x_c) + s (u - u(x_c)) per axis about the central pixel.
__global__ void __launch_bounds__(256) k_scale_map(int ny, int nx, double sy, double sx, const double *__restrict__ u,
                                                   double *__restrict__ us) {
    const size_t P = (size_t)ny * nx, pc = (size_t)(ny / 2) * nx + nx / 2;
    const double c0 = u[pc], c1 = u[P + pc];
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        us[p] = c0 + sy * (u[p] - c0);
        us[P + p] = c1 + sx * (u[P + p] - c1);
    }
}

// sums of I_ref, I_ref^2 and the count over w > 0, then the contrast std / mean
__global__ void __launch_bounds__(256) k_contrast_sums(size_t R, const float *__restrict__ Iref,
                                                       const float *__restrict__ w, double *acc) {
    __shared__ double s1[8], s2[8], sn[8];
    double a1 = 0.0, a2 = 0.0, an = 0.0;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < R; c += (size_t)gridDim.x * blockDim.x)
        if (w[c] > 0.0f) {
            const double v = Iref[c];
            a1 += v;
            a2 = fma(v, v, a2);
            an += 1.0;
        }
    a1 = warp_sum(a1);
    a2 = warp_sum(a2);
    an = warp_sum(an);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s1[warp] = a1;
        s2[warp] = a2;
        sn[warp] = an;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0, tn = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            t1 += s1[k];
            t2 += s2[k];
            tn += sn[k];
        }
        atomicAdd(acc, t1);
        atomicAdd(acc + 1, t2);
        atomicAdd(acc + 2, tn);
    }
}

__global__ void k_contrast_final(int npairs, const double *__restrict__ acc, double *__restrict__ contrast) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npairs) return;
    const double n = acc[3 * k + 2];
    const double mean = n > 0.0 ? acc[3 * k] / n : 0.0;
    const double var = n > 0.0 ? fmax(acc[3 * k + 1] / n - mean * mean, 0.0) : 0.0;
    contrast[k] = (n > 0.0 && mean != 0.0) ? sqrt(var) / mean : 0.0;
}

}  // namespace

cudaError_t launch_scale_map(const pxst_dims &d, double sy, double sx, const double *u, double *us, cudaStream_t s) {
    const size_t P = (size_t)d.ny * d.nx;
    size_t blocks = (P + 255) / 256;
    if (blocks > (size_t)device_sms() * 8) blocks = (size_t)device_sms() * 8;
    k_scale_map<<<(unsigned)blocks, 256, 0, s>>>(d.ny, d.nx, sy, sx, u, us); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_contrast_sums(const pxst_dims &d, const float *I_ref, const float *w, double *acc, cudaStream_t s) {
    const size_t R = (size_t)d.ref_ny * d.ref_nx;
    size_t blocks = (R + 255) / 256;
    if (blocks > (size_t)device_sms() * 4) blocks = (size_t)device_sms() * 4;
    k_contrast_sums<<<(unsigned)blocks, 256, 0, s>>>(R, I_ref, w, acc); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_contrast_final(int npairs, const double *acc, double *contrast, cudaStream_t s) {
    k_contrast_final<<<(npairs + 127) / 128, 128, 0, s>>>(npairs, acc, contrast); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_frac_refine(const pxst_dims &d, int sub, const float *frames, const float *W, const uint8_t *mask,
                               const float *I_ref, const float *w, const FrameShift *shifts, double *u,
                               float *err_out, cudaStream_t s) {
    FracArgs a;
    a.N = d.n_frames; a.ny = d.ny; a.nx = d.nx; a.Ry = d.ref_ny; a.Rx = d.ref_nx; a.sub = sub;
    a.frames = frames; a.W = W; a.mask = mask; a.Iref = I_ref; a.w = w; a.shifts = shifts; a.u = u;
    a.err_out = err_out;
    const size_t P = (size_t)d.ny * d.nx;
    k_frac_refine<<<(unsigned)((P + 127) / 128), 128, 0, s>>>(a); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_filter_map(const pxst_dims &d, double sigma, const uint8_t *mask, double *u, double *num,
                              double *den, cudaStream_t s) {
    if (!(sigma > 0.0)) return cudaSuccess;
    FilterArgs f;
    f.ny = d.ny; f.nx = d.nx;
    f.r = (int)floor(4.0 * sigma + 0.5);
    f.inv2s2 = 1.0 / (2.0 * sigma * sigma);
    f.mask = mask; f.u = u; f.num = num; f.den = den;
    const size_t P = (size_t)d.ny * d.nx;
    size_t blocks = (P + 255) / 256;
    if (blocks > (size_t)device_sms() * 8) blocks = (size_t)device_sms() * 8;
    const size_t smem = sizeof(double) * (f.r + 1);      // r <= 4096 (sigma <= 1024)
    cudaError_t e = cudaSuccess;
    if (smem > 48 * 1024) {
        if ((e = cudaFuncSetAttribute(k_filter_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
                cudaSuccess ||
            (e = cudaFuncSetAttribute(k_filter_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
                cudaSuccess)
            return e;
    }
    k_filter_rows<<<(unsigned)blocks, 256, smem, s>>>(f); note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_filter_cols<<<(unsigned)blocks, 256, smem, s>>>(f); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_pixvar(const pxst_dims &d, const float *frames, const float *W, const uint8_t *mask,
                          const float *I_ref, const float *w, const double *u, const double *delta,
                          const FrameShift *shifts, float *var, WsHeader *hdr, cudaStream_t s) {
    const size_t P = (size_t)d.ny * d.nx;
    k_pixvar<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(merit_args(d, frames, W, mask, I_ref, w, u, delta, shifts, var, hdr)); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_calc_error(const pxst_dims &d, const float *frames, const float *W, const uint8_t *mask,
                              const float *I_ref, const float *w, const double *u, const double *delta,
                              const FrameShift *shifts, const float *var, WsHeader *hdr, float *pixel_err,
                              double *frame_err, double *total, float *ref_err, double *num, double *den,
                              cudaStream_t s) {
    const size_t P = (size_t)d.ny * d.nx, R = (size_t)d.ref_ny * d.ref_nx;
    cudaError_t e;
    if (frame_err && (e = cudaMemsetAsync(frame_err, 0, sizeof(double) * d.n_frames, s)) != cudaSuccess) return e;
    if (total && (e = cudaMemsetAsync(total, 0, sizeof(double), s)) != cudaSuccess) return e;
    if (ref_err) {
        if ((e = cudaMemsetAsync(num, 0, sizeof(float) * R, s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(den, 0, sizeof(float) * R, s)) != cudaSuccess) return e;
    }
    float *numf = reinterpret_cast<float *>(num), *denf = reinterpret_cast<float *>(den);   // R floats each
    ErrorOut o{pixel_err, frame_err, total, ref_err ? numf : nullptr, ref_err ? denf : nullptr};
    size_t blocks = (P + 255) / 256;
    if (blocks > (size_t)device_sms() * 4) blocks = (size_t)device_sms() * 4;
    const size_t smem = (frame_err && d.n_frames <= kErrFramesSmem) ? sizeof(double) * d.n_frames : 0;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(k_calc_error, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    k_calc_error<<<(unsigned)blocks, 256, smem, s>>>(
        merit_args(d, frames, W, mask, I_ref, w, u, delta, shifts, const_cast<float *>(var), hdr), o); note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ref_err) {
        blocks = (R + 255) / 256;
        if (blocks > (size_t)device_sms() * 16) blocks = (size_t)device_sms() * 16;
        k_err_normalise<<<(unsigned)blocks, 256, 0, s>>>((int)R, numf, denf, ref_err); note_launch();
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_update_translations(const pxst_dims &d, int Ty, int Tx, int quadratic, const float *frames,
                                       const float *W, const uint8_t *mask, const float *I_ref, const float *w,
                                       const double *u, const double *delta_in, const FrameShift *shifts,
                                       const float *var, WsHeader *hdr, double *acc_sum,
                                       unsigned long long *acc_cnt, double *delta_out, double *err_out,
                                       cudaStream_t s) {
    const size_t P = (size_t)d.ny * d.nx;
    cudaError_t e;
    if ((e = cudaMemsetAsync(acc_sum, 0, sizeof(double) * kTransMax * d.n_frames, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(acc_cnt, 0, sizeof(unsigned long long) * kTransMax * d.n_frames, s)) != cudaSuccess)
        return e;
    TransArgs t;
    t.m = merit_args(d, frames, W, mask, I_ref, w, u, delta_in, shifts, const_cast<float *>(var), hdr);
    t.Ty = Ty; t.Tx = Tx; t.quadratic = quadratic;
    t.acc_sum = acc_sum; t.acc_cnt = acc_cnt; t.delta_out = delta_out; t.err_out = err_out;
    size_t g = (P + 255) / 256;
    if (g > 32) g = 32;                 // blocks per frame
    dim3 grid((unsigned)g, (unsigned)d.n_frames);
    k_trans_acc<<<grid, 256, 0, s>>>(t); note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_trans_fit<<<(d.n_frames + 127) / 128, 128, 0, s>>>(t); note_launch();
    return cudaGetLastError();
}

}  // namespace pxst
