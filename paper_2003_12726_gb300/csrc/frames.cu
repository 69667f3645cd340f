// frames.cu -- figures of merit (section "Calculate figures of merit") and the
// translation update (section "Update translations") on sm_103a.
//
//   k_pixvar      var(x) = sum over the frames valid at u(x) - Delta_n of (I_n - W)^2, and
//                 (for the translation update) each pixel's record: its map split into
//                 integers and FP32 fractions, var(x) and W
//   k_nanref      the reference with unusable cells (w <= 0) stored as NaN
//   k_calc_error  eps[n,x] = (I_n - W R_n)^2 / var(x) per pixel and frame: the pixel error
//                 (sum over n), the frame errors (FP32 warp sums, FP64 block sums and
//                 atomics), the total and the reference-plane error (eps scattered with the
//                 bilinear weights to u - Delta_n into (sum, weight) pairs by 8-byte atomics,
//                 then divided by the weights that landed)
//   k_trans_acc_patch  per frame and integer shift t (|t| <= 2 per axis) of its translation:
//                 the sum of eps over the pixels whose read at u - Delta_n - t is valid, and
//                 their count; each pixel and frame reads one patch of the reference for
//                 all shifts (k_trans_acc: the same for wider windows, read by read)
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
    PixSplit *split;               // [P] workspace: the split map (written by k_pixvar), or null
    const float *Rm;               // [R] workspace: the NaN-marked reference, or null
    WsHeader *hdr;
};

__global__ void __launch_bounds__(256) k_pixvar(MeritArgs a) {
    const size_t P = (size_t)a.ny * a.nx;
    const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    float v = -1.0f;
    PixSplit rec{0, 0, 0.0f, 0.0f, -1.0f, 0.0f, 0, 0};
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
            rec = PixSplit{ui0, ui1, uf0, uf1, -1.0f, Wv, 0, 0};
            float s2 = 0.0f;
            // four frames per pass, so that their loads are in flight together
#pragma unroll 4
            for (int n = 0; n < a.N; ++n) {
                int i0, j0;
                float f0, f1;
                frame_point(ui0, uf0, ui1, uf1, a.shifts[n], 0, 0, i0, f0, j0, f1);
                // the frame is valid when gather_masked's weight sum is positive: some corner
                // with a non-zero bilinear weight is on the grid with w > 0 (the weights are >= 0)
                const float wt[4] = {(1.0f - f0) * (1.0f - f1), (1.0f - f0) * f1, f0 * (1.0f - f1), f0 * f1};
                bool valid = false;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int ii = i0 + (k >> 1), jj = j0 + (k & 1);
                    const bool on = wt[k] != 0.0f && ii >= 0 && ii < a.Ry && jj >= 0 && jj < a.Rx;
                    const float wk = on ? __ldg(a.w + (size_t)ii * a.Rx + jj) : 0.0f;
                    valid = valid || wk > 0.0f;
                }
                const float t = __ldcs(a.frames + (size_t)n * P + p) - Wv;
                s2 = valid ? fmaf(t, t, s2) : s2;
            }
            v = s2;
        }
    }
    a.var[p] = v;
    if (a.split) {
        rec.var = v;
        a.split[p] = rec;
    }
}

// the record of pixel p, read as two 16-byte loads through the read-only path
__device__ __forceinline__ PixSplit load_split(const PixSplit *sp, size_t p) {
    const int4 *q = reinterpret_cast<const int4 *>(sp + p);
    const int4 x = __ldg(q), y = __ldg(q + 1);
    return PixSplit{x.x, x.y, __int_as_float(x.z), __int_as_float(x.w), __int_as_float(y.x), __int_as_float(y.y), 0, 0};
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
    float2 *nd;            // [R] accumulators (sum of weight x eps, sum of weight) of the
                           // reference-plane error, or null
};

// The reference with its unusable cells (w <= 0) stored as NaN, so that a masked read takes
// one load per corner.
__global__ void k_nanref(int R, const float *__restrict__ Iref, const float *__restrict__ w, float *__restrict__ Rm) {
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < (size_t)R; c += (size_t)gridDim.x * blockDim.x)
        Rm[c] = w[c] > 0.0f ? Iref[c] : __int_as_float(0x7fc00000);
}

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
        const float rvar = var > 0.0f ? 1.0f / var : 1.0f;     // var = 0: eps = d^2
        // a warp none of whose pixels counts adds nothing to any sum
        const int n_end = __any_sync(0xffffffffu, act) ? a.N : 0;
        // the next frame's value is read while this one is scored
        float Inxt = (act && n_end > 0) ? __ldcs(a.frames + p) : 0.0f;
        for (int n = 0; n < n_end; ++n) {
            float eps = 0.0f;
            bool sc = false;                 // this lane scatters frame n
            int i0 = 0, j0 = 0;
            float wt[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            const float I = Inxt;
            if (act && n + 1 < n_end) Inxt = __ldcs(a.frames + (size_t)(n + 1) * P + p);
            if (act) {
                float fy, fx, R;
                frame_point(ui0, uf0, ui1, uf1, a.shifts[n], 0, 0, i0, fy, j0, fx);
                if (gather_rm(a.Rm, a.Ry, a.Rx, i0, j0, fy, fx, R)) {
                    const float d = fmaf(-Wv, R, I);
                    eps = d * d * rvar;
                    sc = o.nd != nullptr;
                    wt[0] = (1.0f - fy) * (1.0f - fx);
                    wt[1] = (1.0f - fy) * fx;
                    wt[2] = fy * (1.0f - fx);
                    wt[3] = fy * fx;
                }
            }
            if (o.nd) {
                // scatter with make_object_map's bilinear weights (corners off the grid
                // dropped), both sums of a cell in one 8-byte atomic. The lanes are consecutive
                // pixels: where lane l's right corners are lane l + 1's left corners, lane l
                // hands them over and lane l + 1 adds both with one atomic per row.
                const int ni0 = __shfl_down_sync(0xffffffffu, i0, 1), nj0 = __shfl_down_sync(0xffffffffu, j0, 1);
                const bool nsc = __shfl_down_sync(0xffffffffu, (int)sc, 1) != 0;
                const bool give = sc && lane < 31 && nsc && ni0 == i0 && nj0 == j0 + 1;
                const bool take = __shfl_up_sync(0xffffffffu, (int)give, 1) != 0 && lane > 0;
                const float g1 = wt[1] * eps, g3 = wt[3] * eps;
                const float t1 = __shfl_up_sync(0xffffffffu, g1, 1), tw1 = __shfl_up_sync(0xffffffffu, wt[1], 1);
                const float t3 = __shfl_up_sync(0xffffffffu, g3, 1), tw3 = __shfl_up_sync(0xffffffffu, wt[3], 1);
                if (sc) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (give && (k & 1)) continue;
                        float vs = wt[k] * eps, vw = wt[k];
                        if (take && k == 0) {
                            vs += t1;
                            vw += tw1;
                        } else if (take && k == 2) {
                            vs += t3;
                            vw += tw3;
                        }
                        const int ii = i0 + (k >> 1), jj = j0 + (k & 1);
                        if (vw == 0.0f || ii < 0 || ii >= a.Ry || jj < 0 || jj >= a.Rx) continue;
                        atomicAdd(o.nd + (size_t)ii * a.Rx + jj, make_float2(vs, vw));
                    }
                }
            }
            pe += eps;
            if (o.frame_err) {
                // the warp's 32 terms are summed in FP32, the warps' sums in FP64
                float s = eps;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
                if (lane == 0 && s != 0.0f) {
                    if (smem_fe) atomicAdd(s_fe + n, (double)s);
                    else atomicAdd(o.frame_err + n, (double)s);
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

__global__ void k_err_normalise(int R, const float2 *__restrict__ nd, float *__restrict__ ref_err) {
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < (size_t)R; c += (size_t)gridDim.x * blockDim.x) {
        const float2 v = nd[c];
        ref_err[c] = v.y > 0.0f ? v.x / v.y : 0.0f;
    }
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
            const PixSplit ps = a.split[p];
            ui0 = ps.i0; ui1 = ps.i1; uf0 = ps.f0; uf1 = ps.f1;
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

// The same sums for small shift windows (|t_y| <= TY, |t_x| <= TX): for a pixel and frame, the
// reads at u - Delta_n - t of every shift t share one set of bilinear weights (an integer
// shift leaves the fraction alone) and lie in one (2TY + 2) x (2TX + 2) patch of the
// NaN-marked reference, which is read once; each masked read then takes the arithmetic of
// gather_masked, corner by corner (the weight sum divides once when every corner is usable).
// Each thread keeps its own sums per shift in registers (FP32 over at most 64 pixels, then
// FP64) and the block sums them once at the end; the next pixel's record is read while this
// one is scored.
template <int TY, int TX>
__global__ void __launch_bounds__(256, (2 * TY + 1) * (2 * TX + 1) > 9 ? 1 : 3) k_trans_acc_patch(TransArgs t) {
    constexpr int WX = 2 * TX + 1, NC = (2 * TY + 1) * WX, PH = 2 * TY + 2, PW = 2 * TX + 2;
    static_assert(PH * PW <= 64, "patch validity bits");
    constexpr unsigned long long ALL = (PH * PW == 64) ? ~0ull : ((1ull << (PH * PW)) - 1ull);
    __shared__ double s_sum[NC];
    __shared__ unsigned int s_cnt[NC];
    const MeritArgs &a = t.m;
    for (int k = threadIdx.x; k < NC; k += blockDim.x) {
        s_sum[k] = 0.0;
        s_cnt[k] = 0u;
    }
    __syncthreads();
    const size_t P = (size_t)a.ny * a.nx;
    const int n = blockIdx.y;
    const FrameShift sh = a.shifts[n];
    const float qnan = __int_as_float(0x7fc00000);
    float acc[NC];
    double accd[NC];
    unsigned cnt[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        acc[k] = 0.0f;
        accd[k] = 0.0;
        cnt[k] = 0u;
    }
    int since = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const PixSplit none{0, 0, 0.0f, 0.0f, -1.0f, 0.0f, 0, 0};
    size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    PixSplit nxt = p < P ? load_split(a.split, p) : none;
    for (; p < P; p += stride) {
        const PixSplit ps = nxt;
        nxt = p + stride < P ? load_split(a.split, p + stride) : none;
        const float var = ps.var;
        if (!(var > 0.0f)) continue;
        const float I = __ldcs(a.frames + (size_t)n * P + p), Wv = ps.W;
        int i0, j0;
        float fy, fx;
        frame_point(ps.i0, ps.f0, ps.i1, ps.f1, sh, 0, 0, i0, fy, j0, fx);
        const float wt[4] = {(1.0f - fy) * (1.0f - fx), (1.0f - fy) * fx, fy * (1.0f - fx), fy * fx};
        // the patch: rows i0 - TY .. i0 + TY + 1, columns j0 - TX .. j0 + TX + 1 (NaN: unusable)
        float pv[PH][PW];
        unsigned long long ok = 0ull;
        const bool inside = i0 - TY >= 0 && i0 + TY + 1 < a.Ry && j0 - TX >= 0 && j0 + TX + 1 < a.Rx;
#pragma unroll
        for (int r = 0; r < PH; ++r)
#pragma unroll
            for (int c = 0; c < PW; ++c) {
                const int ii = i0 - TY + r, jj = j0 - TX + c;
                float v = qnan;
                if (inside || (ii >= 0 && ii < a.Ry && jj >= 0 && jj < a.Rx)) v = __ldg(a.Rm + (size_t)ii * a.Rx + jj);
                pv[r][c] = v;
                if (v == v) ok |= 1ull << (r * PW + c);
            }
        const float rvar = 1.0f / var;
        if (ok == ALL) {
            const float rden = 1.0f / (((wt[0] + wt[1]) + wt[2]) + wt[3]);
#pragma unroll
            for (int da = -TY; da <= TY; ++da)
#pragma unroll
                for (int db = -TX; db <= TX; ++db) {
                    const int r0 = TY - da, c0 = TX - db, k = (da + TY) * WX + (db + TX);
                    float num = wt[0] * pv[r0][c0];
                    num = fmaf(wt[1], pv[r0][c0 + 1], num);
                    num = fmaf(wt[2], pv[r0 + 1][c0], num);
                    num = fmaf(wt[3], pv[r0 + 1][c0 + 1], num);
                    const float d = fmaf(-Wv, num * rden, I);
                    acc[k] = fmaf(d * d, rvar, acc[k]);
                    cnt[k] += 1u;
                }
        } else {
#pragma unroll
            for (int da = -TY; da <= TY; ++da)
#pragma unroll
                for (int db = -TX; db <= TX; ++db) {
                    const int r0 = TY - da, c0 = TX - db, k = (da + TY) * WX + (db + TX);
                    float num = 0.0f, den = 0.0f;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int r = r0 + (q >> 1), c = c0 + (q & 1);
                        if (wt[q] == 0.0f || !((ok >> (r * PW + c)) & 1ull)) continue;
                        num = fmaf(wt[q], pv[r][c], num);
                        den += wt[q];
                    }
                    if (den > 0.0f) {
                        const float d = fmaf(-Wv, num / den, I);
                        acc[k] = fmaf(d * d, rvar, acc[k]);
                        cnt[k] += 1u;
                    }
                }
        }
        if (++since == 64) {
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                accd[k] += (double)acc[k];
                acc[k] = 0.0f;
            }
            since = 0;
        }
    }
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        double sv = accd[k] + (double)acc[k];
        unsigned c = cnt[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, off);
        c = __reduce_add_sync(0xffffffffu, c);
        if (lane == 0 && c) {
            atomicAdd(&s_sum[k], sv);
            atomicAdd(&s_cnt[k], c);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < NC; k += blockDim.x)
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
                     const FrameShift *shifts, float *var, WsHeader *hdr, PixSplit *split = nullptr) {
    MeritArgs a;
    a.shifts = shifts;
    a.N = d.n_frames; a.ny = d.ny; a.nx = d.nx; a.Ry = d.ref_ny; a.Rx = d.ref_nx;
    a.frames = frames; a.W = W; a.mask = mask; a.Iref = I_ref; a.w = w; a.u = u; a.delta = delta;
    a.var = var; a.hdr = hdr; a.split = split; a.Rm = nullptr;
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
                          const FrameShift *shifts, float *var, PixSplit *split, WsHeader *hdr, cudaStream_t s) {
    const size_t P = (size_t)d.ny * d.nx;
    k_pixvar<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(
        merit_args(d, frames, W, mask, I_ref, w, u, delta, shifts, var, hdr, split)); note_launch();
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
    float2 *nd = reinterpret_cast<float2 *>(num);     // R (sum, weight) pairs in num's R doubles
    if (ref_err && (e = cudaMemsetAsync(nd, 0, sizeof(float2) * R, s)) != cudaSuccess) return e;
    ErrorOut o{pixel_err, frame_err, total, ref_err ? nd : nullptr};
    size_t blocks = (P + 255) / 256;
    if (blocks > (size_t)device_sms() * 4) blocks = (size_t)device_sms() * 4;
    const size_t smem = (frame_err && d.n_frames <= kErrFramesSmem) ? sizeof(double) * d.n_frames : 0;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(k_calc_error, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    // the NaN-marked reference in den's space (R floats of R doubles)
    float *Rm = reinterpret_cast<float *>(den);
    size_t rb = (R + 255) / 256;
    if (rb > (size_t)device_sms() * 8) rb = (size_t)device_sms() * 8;
    k_nanref<<<(unsigned)rb, 256, 0, s>>>((int)R, I_ref, w, Rm); note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    MeritArgs ma = merit_args(d, frames, W, mask, I_ref, w, u, delta, shifts, const_cast<float *>(var), hdr);
    ma.Rm = Rm;
    k_calc_error<<<(unsigned)blocks, 256, smem, s>>>(ma, o); note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ref_err) {
        blocks = (R + 255) / 256;
        if (blocks > (size_t)device_sms() * 16) blocks = (size_t)device_sms() * 16;
        k_err_normalise<<<(unsigned)blocks, 256, 0, s>>>((int)R, nd, ref_err); note_launch();
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_update_translations(const pxst_dims &d, int Ty, int Tx, int quadratic, const float *frames,
                                       const float *W, const uint8_t *mask, const float *I_ref, const float *w,
                                       const double *u, const double *delta_in, const FrameShift *shifts,
                                       const float *var, const PixSplit *split, float *Rm, WsHeader *hdr,
                                       double *acc_sum, unsigned long long *acc_cnt, double *delta_out,
                                       double *err_out, cudaStream_t s) {
    const size_t P = (size_t)d.ny * d.nx;
    cudaError_t e;
    if ((e = cudaMemsetAsync(acc_sum, 0, sizeof(double) * kTransMax * d.n_frames, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(acc_cnt, 0, sizeof(unsigned long long) * kTransMax * d.n_frames, s)) != cudaSuccess)
        return e;
    TransArgs t;
    t.m = merit_args(d, frames, W, mask, I_ref, w, u, delta_in, shifts, const_cast<float *>(var), hdr,
                     const_cast<PixSplit *>(split));
    t.Ty = Ty; t.Tx = Tx; t.quadratic = quadratic;
    t.acc_sum = acc_sum; t.acc_cnt = acc_cnt; t.delta_out = delta_out; t.err_out = err_out;
    // small windows take the patch kernel (one instance per window shape) on the NaN-marked
    // reference
    void (*patch)(TransArgs) = nullptr;
    if (Ty == 0 && Tx == 0) patch = k_trans_acc_patch<0, 0>;
    else if (Ty == 0 && Tx == 1) patch = k_trans_acc_patch<0, 1>;
    else if (Ty == 0 && Tx == 2) patch = k_trans_acc_patch<0, 2>;
    else if (Ty == 1 && Tx == 0) patch = k_trans_acc_patch<1, 0>;
    else if (Ty == 1 && Tx == 1) patch = k_trans_acc_patch<1, 1>;
    else if (Ty == 1 && Tx == 2) patch = k_trans_acc_patch<1, 2>;
    else if (Ty == 2 && Tx == 0) patch = k_trans_acc_patch<2, 0>;
    else if (Ty == 2 && Tx == 1) patch = k_trans_acc_patch<2, 1>;
    else if (Ty == 2 && Tx == 2) patch = k_trans_acc_patch<2, 2>;
    size_t g = (P + 255) / 256;
    if (g > 32) g = 32;                 // blocks per frame
    if (patch) {
        const size_t R = (size_t)d.ref_ny * d.ref_nx;
        size_t rb = (R + 255) / 256;
        if (rb > (size_t)device_sms() * 8) rb = (size_t)device_sms() * 8;
        k_nanref<<<(unsigned)rb, 256, 0, s>>>((int)R, I_ref, w, Rm); note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        t.m.Rm = Rm;
        patch<<<dim3((unsigned)g, (unsigned)d.n_frames), 256, 0, s>>>(t);
    } else {
        k_trans_acc<<<dim3((unsigned)g, (unsigned)d.n_frames), 256, 0, s>>>(t);
    }
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_trans_fit<<<(d.n_frames + 127) / 128, 128, 0, s>>>(t); note_launch();
    return cudaGetLastError();
}

}  // namespace pxst
