// omap.cu -- make_object_map ("Make reference image", section "Main loop") and the
// per-candidate reference terms, for sm_103a.
//
//   prepare    : -Delta[n] -> (integer shift, fraction) per frame, and their range.
//   scatter    : each CTA (512 threads, one pixel each) owns a 16 x 32 pixel tile and a
//                chunk of frames, cut into groups of consecutive frames whose reference
//                footprint (the tile's u range widened by the group's translation range,
//                +1 for the bilinear corner) fits in shared memory. Each group adds
//                b*M*W*I and b*M*W^2 there with FP32 shared-memory atomics, then flushes
//                the non-zero cells to the FP64 accumulators in global memory with FP64
//                atomics. A single frame whose footprint does not fit adds straight to
//                global memory.
//   normalise  : I_ref = num / den (FP64 divide) where den > 0, else 0; w = den.
//   refterms   : T[c] = sum_n V R^2 and n_valid[c] = sum_n V over the reference grid.
#include <algorithm>
#include <type_traits>
#include <climits>

#include "pxst_common.cuh"

namespace pxst {
namespace {

// ------------------------------------------------------------------------------------
// Also groups the frames by their fractional shift (fy, fx), compared bit for bit: class
// r is the r-th distinct pair in frame order; fclass[n] is frame n's class.
__global__ void __launch_bounds__(1024) k_prepare(int N, const double *__restrict__ delta,
                                                  WsHeader *hdr, FrameShift *shifts, int *fclass,
                                                  int reset_exact) {
    __shared__ int s[4];
    __shared__ int s_nlead;
    __shared__ unsigned int s_fy[kClassFramesMax], s_fx[kClassFramesMax];
    __shared__ int s_lead[kClassFramesMax];
    const bool classes = fclass != nullptr && N <= kClassFramesMax;
    if (threadIdx.x == 0) {
        s[0] = INT_MAX; s[1] = INT_MIN; s[2] = INT_MAX; s[3] = INT_MIN;
        s_nlead = 0;
    }
    __syncthreads();
    int mn_y = INT_MAX, mx_y = INT_MIN, mn_x = INT_MAX, mx_x = INT_MIN;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        FrameShift fs;
        split_neg_delta(delta[2 * n + 0], fs.ky, fs.fy);
        split_neg_delta(delta[2 * n + 1], fs.kx, fs.fx);
        shifts[n] = fs;
        mn_y = min(mn_y, fs.ky); mx_y = max(mx_y, fs.ky);
        mn_x = min(mn_x, fs.kx); mx_x = max(mx_x, fs.kx);
        if (classes) {
            s_fy[n] = __float_as_uint(fs.fy);
            s_fx[n] = __float_as_uint(fs.fx);
        }
    }
    atomicMin(&s[0], mn_y); atomicMax(&s[1], mx_y);
    atomicMin(&s[2], mn_x); atomicMax(&s[3], mx_x);
    __syncthreads();
    if (threadIdx.x == 0) {
        hdr->kmin_y = s[0]; hdr->kmax_y = s[1];
        hdr->kmin_x = s[2]; hdr->kmax_x = s[3];
        if (reset_exact) hdr->n_exact = 0;
        if (!classes) hdr->n_classes = kMaxClasses + 1;
    }
    if (!classes) return;
    // the first frame with the same pair (the loop ends at m = n at the latest)
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        int m = 0;
        while (s_fy[m] != s_fy[n] || s_fx[m] != s_fx[n]) ++m;
        s_lead[n] = m;
    }
    __syncthreads();
    // each first frame's rank among the first frames (its class); kept in s_fx's place
    // after the pairs are read
    int rank_of[(kClassFramesMax + 1023) / 1024];
    for (int n = threadIdx.x, i = 0; n < N; n += blockDim.x, ++i) {
        int r = -1;
        if (s_lead[n] == n) {
            r = 0;
            for (int m = 0; m < n; ++m) r += s_lead[m] == m;
            atomicMax(&s_nlead, r + 1);
            if (r < kMaxClasses) {
                hdr->cls_fy[r] = __uint_as_float(s_fy[n]);
                hdr->cls_fx[r] = __uint_as_float(s_fx[n]);
            }
        }
        rank_of[i] = r;
    }
    __syncthreads();
    for (int n = threadIdx.x, i = 0; n < N; n += blockDim.x, ++i)
        if (rank_of[i] >= 0) s_fx[n] = (unsigned int)rank_of[i];
    __syncthreads();
    for (int n = threadIdx.x; n < N; n += blockDim.x) fclass[n] = (int)min(s_fx[s_lead[n]], (unsigned)kMaxClasses);
    if (threadIdx.x == 0) hdr->n_classes = s_nlead;
}

// ------------------------------------------------------------------------------------
constexpr int SC_TX = 32, SC_TY = 16;                  // 32 x 16 pixels, one per thread
constexpr int SC_THREADS = SC_TX * SC_TY;
constexpr int SC_CAP = 12288;                          // cells (num + den: 96 KB): 2 CTAs per SM
constexpr int SC_PREFETCH = 8;                         // frames in flight while the previous 8 scatter
constexpr int SC_GROUP_MAX = 512;                      // frames per group (their shifts in shared memory)

struct ScatterArgs {
    int N, ny, nx, Ry, Rx, chunk;
    const float *frames, *W;
    const uint8_t *mask;
    const double *u;
    const FrameShift *shifts;
    WsHeader *hdr;
    double *num, *den;
    float *dcls;           // per-class weight images (NULL: the scatter forms the weights)
};

// One CTA per 16 x 32 pixel tile and chunk of frames (two CTAs per SM, so that one's
// barriers overlap the other's accumulation). The chunk is cut into consecutive
// groups of frames whose footprint (the tile's floor(u) range widened by the group's
// integer shifts, +1 for a carry and +1 for the second corner) fits in shared memory;
// each group is accumulated there with FP32 atomics and flushed to the FP64 accumulators.
__global__ void __launch_bounds__(SC_THREADS, 2) k_scatter(ScatterArgs a) {
    extern __shared__ float sm[];
    float *s_num = sm;
    float *s_den = sm + SC_CAP;
    __shared__ int s_rng[4];
    __shared__ int s_grp[6];       // group [start, end), footprint origin r0, c0, height, width
    __shared__ __align__(16) FrameShift s_sh[SC_GROUP_MAX];   // the group's shifts

    const int x = blockIdx.x * SC_TX + (threadIdx.x % SC_TX);
    const int y = blockIdx.y * SC_TY + (threadIdx.x / SC_TX);
    const int n0 = blockIdx.z * a.chunk, n1 = min(a.N, n0 + a.chunk);
    const size_t P = (size_t)a.ny * a.nx;

    if (threadIdx.x < 4) s_rng[threadIdx.x] = (threadIdx.x & 1) ? INT_MIN : INT_MAX;
    __syncthreads();

    int iy = 0, ix = 0;
    float fy = 0.0f, fx = 0.0f, Wv = 0.0f;
    bool act = false;
    size_t pix = 0;
    if (y < a.ny && x < a.nx) {
        pix = (size_t)y * a.nx + x;
        if (a.mask[pix]) {
            const double u0 = a.u[pix], u1 = a.u[P + pix];
            if (!isfinite(u0) || !isfinite(u1)) {
                atomicOr(&a.hdr->status, PXST_DEV_NONFINITE_U);
            } else if (fabs(u0) > kMaxCoord || fabs(u1) > kMaxCoord) {
                atomicOr(&a.hdr->status, PXST_DEV_U_RANGE);
            } else {
                const double f0 = floor(u0), f1 = floor(u1);
                iy = (int)f0;
                ix = (int)f1;
                fy = (float)(u0 - f0);
                fx = (float)(u1 - f1);
                if (fy >= 1.0f) { fy = 0.0f; iy += 1; }
                if (fx >= 1.0f) { fx = 0.0f; ix += 1; }
                Wv = a.W[pix];
                if (!(Wv > 0.0f) || !isfinite(Wv)) {
                    // the forward model needs a positive whitefield: the pixel adds nothing
                    atomicOr(&a.hdr->status, PXST_DEV_BAD_INPUT);
                    Wv = 0.0f;
                } else {
                    act = true;
                    atomicMin(&s_rng[0], iy); atomicMax(&s_rng[1], iy);
                    atomicMin(&s_rng[2], ix); atomicMax(&s_rng[3], ix);
                }
            }
        }
    }
    __syncthreads();
    if (s_rng[0] == INT_MAX || n0 >= n1) return;      // no active pixel in the tile
    // the weights of pixels whose zero-shift corners stay on the grid for every fraction
    // class are formed per class (k_dscatter, k_dgather); only the others add them here
    const bool split = a.dcls != nullptr && a.hdr->n_classes <= kMaxClasses;
    // one fraction class for every frame (set by k_prepare from the translations)
    const bool uniform = a.hdr->n_classes == 1;
    bool bad_frame = false;
    const bool dom = act && iy >= 0 && iy <= a.Ry - 3 && ix >= 0 && ix <= a.Rx - 3;
    const float WW = (split && dom) ? 0.0f : Wv * Wv;
    const int lane = threadIdx.x & 31;


    for (int gs = n0; gs < n1;) {
        if (threadIdx.x == 0) {
            // extend the group while its footprint fits (at least one frame per group)
            int kmn_y = INT_MAX, kmx_y = INT_MIN, kmn_x = INT_MAX, kmx_x = INT_MIN;
            int ge = gs;
            long long H = 0, Wd = 0;
            while (ge < n1 && ge - gs < SC_GROUP_MAX) {
                const FrameShift f = a.shifts[ge];
                const int a0 = min(kmn_y, f.ky), a1 = max(kmx_y, f.ky);
                const int b0 = min(kmn_x, f.kx), b1 = max(kmx_x, f.kx);
                const long long h = (long long)s_rng[1] + a1 + 2 - ((long long)s_rng[0] + a0) + 1;
                const long long wd = (long long)s_rng[3] + b1 + 2 - ((long long)s_rng[2] + b0) + 1;
                if (ge > gs && h * wd > SC_CAP) break;
                kmn_y = a0; kmx_y = a1; kmn_x = b0; kmx_x = b1;
                H = h; Wd = wd;
                ++ge;
            }
            s_grp[0] = gs;
            s_grp[1] = ge;
            s_grp[2] = s_rng[0] + kmn_y;
            s_grp[3] = s_rng[2] + kmn_x;
            s_grp[4] = (H * Wd <= SC_CAP) ? (int)H : -1;     // -1: add straight to global
            s_grp[5] = (int)Wd;
        }
        __syncthreads();
        const int g0 = s_grp[0], g1 = s_grp[1], r0 = s_grp[2], c0 = s_grp[3];
        const int H = s_grp[4], Wd = s_grp[5];
        const bool fits = H > 0;
        if (fits)
            for (int c = threadIdx.x; c < H * Wd; c += SC_THREADS) {
                s_num[c] = 0.0f;
                s_den[c] = 0.0f;
            }
        for (int q = threadIdx.x; q < g1 - g0; q += SC_THREADS) s_sh[q] = a.shifts[g0 + q];
        __syncthreads();
        // Every lane of a warp (one pixel row, consecutive columns) runs the frame loop so
        // that neighbouring lanes can merge contributions: when lane l+1's left corner is
        // the cell right of lane l's left corner on the same row, lane l hands its right
        // corners to lane l+1, which adds both with one atomic per row. Corners whose
        // bilinear weight is exactly zero are skipped.
        // warps none of whose pixels adds weights here run a loop without them
        const bool warp_den = __any_sync(0xffffffffu, act && WW != 0.0f);
        auto frames_loop = [&](auto den_tag) {
            constexpr bool DEN = decltype(den_tag)::value;
            // frames stream through a register double buffer: the next 8 frames' loads are
            // in flight while the current 8 are scattered (the frames are read once: streaming)
            float In[SC_PREFETCH];
#pragma unroll
            for (int jf = 0; jf < SC_PREFETCH; ++jf)
                In[jf] = (act && g0 + jf < g1) ? __ldcs(a.frames + (size_t)(g0 + jf) * P + pix) : 0.0f;
            for (int n = g0; n < g1; n += SC_PREFETCH) {
                float I[SC_PREFETCH];
#pragma unroll
                for (int jf = 0; jf < SC_PREFETCH; ++jf) {
                    // a non-finite frame value adds nothing (and is reported below)
                    bad_frame |= !isfinite(In[jf]);
                    I[jf] = isfinite(In[jf]) ? In[jf] : 0.0f;
                    const int m = n + SC_PREFETCH + jf;
                    In[jf] = (act && m < g1) ? __ldcs(a.frames + (size_t)m * P + pix) : 0.0f;
                }
#pragma unroll
                for (int jf = 0; jf < SC_PREFETCH; ++jf) {
                    if (n + jf >= g1) break;                    // uniform over the CTA
                    const FrameShift S = s_sh[n + jf - g0];
                    int by = iy + S.ky, bx = ix + S.kx;
                    float sy = fy + S.fy, sx = fx + S.fx;
                    if (sy >= 1.0f) { sy -= 1.0f; by += 1; }
                    if (sx >= 1.0f) { sx -= 1.0f; bx += 1; }
                    if (!act) { by = INT_MIN; bx = INT_MIN; }
                    const float WI = Wv * I[jf];
                    // right corners (top, bottom) and left corners, numerator and weight
                    float rn0 = (1.0f - sy) * sx * WI, rn1 = sy * sx * WI;
                    float ln0 = (1.0f - sy) * (1.0f - sx) * WI, ln1 = sy * (1.0f - sx) * WI;
                    float rd0 = 0.0f, rd1 = 0.0f, ld0 = 0.0f, ld1 = 0.0f;
                    if constexpr (DEN) {
                        rd0 = (1.0f - sy) * sx * WW;
                        rd1 = sy * sx * WW;
                        ld0 = (1.0f - sy) * (1.0f - sx) * WW;
                        ld1 = sy * (1.0f - sx) * WW;
                    }
                    const int pbx = __shfl_up_sync(0xffffffffu, bx, 1);
                    const int pby = __shfl_up_sync(0xffffffffu, by, 1);
                    const float prn0 = __shfl_up_sync(0xffffffffu, rn0, 1);
                    const float prn1 = __shfl_up_sync(0xffffffffu, rn1, 1);
                    float prd0 = 0.0f, prd1 = 0.0f;
                    if constexpr (DEN) {
                        prd0 = __shfl_up_sync(0xffffffffu, rd0, 1);
                        prd1 = __shfl_up_sync(0xffffffffu, rd1, 1);
                    }
                    const bool take = act && lane > 0 && pby == by && pbx != INT_MIN && pbx + 1 == bx;
                    const bool given = __shfl_down_sync(0xffffffffu, take ? 1 : 0, 1) && lane < 31;
                    if (take) {
                        ln0 += prn0;
                        ln1 += prn1;
                        if constexpr (DEN) {
                            ld0 += prd0;
                            ld1 += prd1;
                        }
                    }
                    if (!act) continue;
                    const bool row1 = sy != 0.0f;                // bottom corners carry weight
                    const bool right = sx != 0.0f && !given;     // right corners not handed over
                    if (fits) {
                        const int c00 = (by - r0) * Wd + (bx - c0);
                        atomicAdd(&s_num[c00], ln0);
                        if (DEN && ld0 != 0.0f) atomicAdd(&s_den[c00], ld0);
                        if (right) {
                            atomicAdd(&s_num[c00 + 1], rn0);
                            if (DEN && rd0 != 0.0f) atomicAdd(&s_den[c00 + 1], rd0);
                        }
                        if (row1 || (take && (prn1 != 0.0f || prd1 != 0.0f))) {
                            atomicAdd(&s_num[c00 + Wd], ln1);
                            if (DEN && ld1 != 0.0f) atomicAdd(&s_den[c00 + Wd], ld1);
                        }
                        if (row1 && right) {
                            atomicAdd(&s_num[c00 + Wd + 1], rn1);
                            if (DEN && rd1 != 0.0f) atomicAdd(&s_den[c00 + Wd + 1], rd1);
                        }
                    } else {
                        const float vn[4] = {ln0, right ? rn0 : 0.0f, ln1, right ? rn1 : 0.0f};
                        const float vd[4] = {ld0, right ? rd0 : 0.0f, ld1, right ? rd1 : 0.0f};
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int gy = by + (k >> 1), gx = bx + (k & 1);
                            if (vd[k] == 0.0f && vn[k] == 0.0f) continue;
                            if (gy < 0 || gy >= a.Ry || gx < 0 || gx >= a.Rx) continue;
                            const size_t gi = (size_t)gy * a.Rx + gx;
                            atomicAdd(&a.num[gi], (double)vn[k]);
                            if (DEN && vd[k] != 0.0f) atomicAdd(&a.den[gi], (double)vd[k]);
                        }
                    }
                }
            }
        };
        // every frame with the same fraction (one class): each pixel's corners, weights and
        // the hand-over to the next lane are the same for every frame, and only the group's
        // integer shift moves them
        auto frames_loop_uniform = [&](auto den_tag) {
            constexpr bool DEN = decltype(den_tag)::value;
            int by = iy, bx = ix;
            float sy = fy + a.hdr->cls_fy[0], sx = fx + a.hdr->cls_fx[0];
            if (sy >= 1.0f) { sy -= 1.0f; by += 1; }
            if (sx >= 1.0f) { sx -= 1.0f; bx += 1; }
            if (!act) { by = INT_MIN; bx = INT_MIN; }
            // right corners (top, bottom) and left corners, per unit frame value and weight
            const float wr0 = (1.0f - sy) * sx * Wv, wr1 = sy * sx * Wv;
            const float wl0 = (1.0f - sy) * (1.0f - sx) * Wv, wl1 = sy * (1.0f - sx) * Wv;
            const float dr0 = DEN ? (1.0f - sy) * sx * WW : 0.0f, dr1 = DEN ? sy * sx * WW : 0.0f;
            const float dl0 = DEN ? (1.0f - sy) * (1.0f - sx) * WW : 0.0f, dl1 = DEN ? sy * (1.0f - sx) * WW : 0.0f;
            const int pbx = __shfl_up_sync(0xffffffffu, bx, 1), pby = __shfl_up_sync(0xffffffffu, by, 1);
            const float pwr0 = __shfl_up_sync(0xffffffffu, wr0, 1), pwr1 = __shfl_up_sync(0xffffffffu, wr1, 1);
            const float pdr0 = __shfl_up_sync(0xffffffffu, dr0, 1), pdr1 = __shfl_up_sync(0xffffffffu, dr1, 1);
            const bool take = act && lane > 0 && pby == by && pbx != INT_MIN && pbx + 1 == bx;
            const bool given = __shfl_down_sync(0xffffffffu, take ? 1 : 0, 1) && lane < 31;
            const float tw0 = take ? pwr0 : 0.0f, tw1 = take ? pwr1 : 0.0f;
            const float td0 = take ? pdr0 : 0.0f, td1 = take ? pdr1 : 0.0f;
            const bool row1 = sy != 0.0f, right = sx != 0.0f && !given;
            const bool low = row1 || (take && (pwr1 != 0.0f || pdr1 != 0.0f));
            // the den terms of a frame do not depend on the frame: the per-frame sums
            const float D0 = dl0 + td0, D1 = dl1 + td1;
            const int cb = act ? (by - r0) * Wd + (bx - c0) : 0;
            float In[SC_PREFETCH];
#pragma unroll
            for (int jf = 0; jf < SC_PREFETCH; ++jf)
                In[jf] = (act && g0 + jf < g1) ? __ldcs(a.frames + (size_t)(g0 + jf) * P + pix) : 0.0f;
            for (int n = g0; n < g1; n += SC_PREFETCH) {
                float I[SC_PREFETCH];
#pragma unroll
                for (int jf = 0; jf < SC_PREFETCH; ++jf) {
                    // a non-finite frame value adds nothing (and is reported below)
                    bad_frame |= !isfinite(In[jf]);
                    I[jf] = isfinite(In[jf]) ? In[jf] : 0.0f;
                    const int m = n + SC_PREFETCH + jf;
                    In[jf] = (act && m < g1) ? __ldcs(a.frames + (size_t)m * P + pix) : 0.0f;
                }
#pragma unroll
                for (int jf = 0; jf < SC_PREFETCH; ++jf) {
                    if (n + jf >= g1) break;                    // uniform over the CTA
                    const FrameShift S = s_sh[n + jf - g0];
                    const float Iv = I[jf];
                    const float Ip = __shfl_up_sync(0xffffffffu, Iv, 1);
                    if (!act) continue;
                    const int c00 = cb + S.ky * Wd + S.kx;
                    atomicAdd(&s_num[c00], fmaf(Ip, tw0, Iv * wl0));
                    if (DEN && D0 != 0.0f) atomicAdd(&s_den[c00], D0);
                    if (right) {
                        atomicAdd(&s_num[c00 + 1], Iv * wr0);
                        if (DEN && dr0 != 0.0f) atomicAdd(&s_den[c00 + 1], dr0);
                    }
                    if (low) {
                        atomicAdd(&s_num[c00 + Wd], fmaf(Ip, tw1, Iv * wl1));
                        if (DEN && D1 != 0.0f) atomicAdd(&s_den[c00 + Wd], D1);
                    }
                    if (row1 && right) {
                        atomicAdd(&s_num[c00 + Wd + 1], Iv * wr1);
                        if (DEN && dr1 != 0.0f) atomicAdd(&s_den[c00 + Wd + 1], dr1);
                    }
                }
            }
        };
        if (uniform && fits) {
            if (warp_den)
                frames_loop_uniform(std::true_type{});
            else
                frames_loop_uniform(std::false_type{});
        } else if (warp_den) {
            frames_loop(std::true_type{});
        } else {
            frames_loop(std::false_type{});
        }
        __syncthreads();
        if (fits)
            for (int c = threadIdx.x; c < H * Wd; c += SC_THREADS) {
                const float dn = s_den[c], nm = s_num[c];
                if (dn == 0.0f && nm == 0.0f) continue;
                const int gy = r0 + c / Wd, gx = c0 + c % Wd;
                if (gy < 0 || gy >= a.Ry || gx < 0 || gx >= a.Rx) continue;   // corners off the grid
                const size_t gi = (size_t)gy * a.Rx + gx;
                if (nm != 0.0f) atomicAdd(&a.num[gi], (double)nm);
                if (dn != 0.0f) atomicAdd(&a.den[gi], (double)dn);
            }
        __syncthreads();
        gs = g1;
    }
    if (bad_frame) atomicOr(&a.hdr->status, PXST_DEV_BAD_INPUT);
}

// ------------------------------------------------------------------------------------
// ---- the reference weights per fractional-shift class ----------------------------------
// For a pixel whose corners stay on the grid, frame n adds b(u + f_n - corner) W^2 at
// corner + k_n, where (k_n, f_n) split -Delta_n into an integer and a fraction: the image
// D_f of those terms for a zero integer shift depends on the frame only through its class
// f, and the frame's terms are D_f moved by k_n. So den(c) gains sum_n D_class(n)(c - k_n):
// one scatter of W^2 per class (P x 4 terms) and one gather per cell and frame, instead of
// a shared-memory atomic per pixel, frame and corner.
__global__ void __launch_bounds__(256) k_dzero(size_t R, const WsHeader *__restrict__ hdr, float *__restrict__ dcls) {
    const int nc = hdr->n_classes;
    if (nc > kMaxClasses) return;
    const size_t total = (size_t)nc * R;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
        dcls[i] = 0.0f;
}

// One thread per pixel, blockIdx.y = class: the zero-shift corner terms b W^2, with the
// fraction split and the corner arithmetic of k_scatter.
__global__ void __launch_bounds__(256) k_dscatter(int ny, int nx, int Ry, int Rx, const float *__restrict__ W,
                                                  const uint8_t *__restrict__ mask, const double *__restrict__ u,
                                                  const WsHeader *__restrict__ hdr, float *__restrict__ dcls) {
    const int f = blockIdx.y;
    if (hdr->n_classes > kMaxClasses || f >= hdr->n_classes) return;
    const size_t P = (size_t)ny * nx, R = (size_t)Ry * Rx;
    const size_t pix = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (pix >= P || !mask[pix]) return;
    const double u0 = u[pix], u1 = u[P + pix];
    if (!isfinite(u0) || !isfinite(u1) || fabs(u0) > kMaxCoord || fabs(u1) > kMaxCoord) return;
    const double f0 = floor(u0), f1 = floor(u1);
    int iy = (int)f0, ix = (int)f1;
    float fy = (float)(u0 - f0), fx = (float)(u1 - f1);
    if (fy >= 1.0f) { fy = 0.0f; iy += 1; }
    if (fx >= 1.0f) { fx = 0.0f; ix += 1; }
    if (iy < 0 || iy > Ry - 3 || ix < 0 || ix > Rx - 3) return;      // k_scatter adds these
    const float Wv = W[pix], WW = Wv * Wv;
    if (!(Wv > 0.0f) || !isfinite(Wv)) return;                       // reported by k_scatter
    int by = iy, bx = ix;
    float sy = fy + hdr->cls_fy[f], sx = fx + hdr->cls_fx[f];
    if (sy >= 1.0f) { sy -= 1.0f; by += 1; }
    if (sx >= 1.0f) { sx -= 1.0f; bx += 1; }
    const float b[4] = {(1.0f - sy) * (1.0f - sx) * WW, (1.0f - sy) * sx * WW, sy * (1.0f - sx) * WW, sy * sx * WW};
    float *D = dcls + (size_t)f * R;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (b[k] != 0.0f) atomicAdd(D + (size_t)(by + (k >> 1)) * Rx + (bx + (k & 1)), b[k]);
}

// den(c) += sum_n D_class(n)(c - k_n), FP32 over runs of 32 frames, FP64 across them: a
// correlation of each class's zero-shift weight image with the frames' integer shifts. One
// block per tile of DT_TY x DT_TX cells; thread t takes column t mod 64 of rows t / 64 + 4 j.
// When the tile's window (the tile widened by the range of the integer shifts) fits the
// block's shared memory, each class's D is staged there once (zero off the grid), and every
// frame's reads are shared-memory loads along a row (consecutive lanes, consecutive words);
// otherwise the reads go through the cache. The block stages 256 frames' window offsets at
// a time; a frame of another class than the one staged is skipped.
constexpr int DG_FRAMES = 256;
constexpr int DT_TY = 32, DT_TX = 64, DT_THREADS = 256;
constexpr int DT_RPT = DT_TY * DT_TX / DT_THREADS;       // cells (rows) per thread: 8
constexpr int DT_SMEM = 64 * 1024;                       // the staged window: three blocks per SM
constexpr int DT_CAP = DT_SMEM / 4;
__global__ void __launch_bounds__(DT_THREADS, 3) k_dgather(int N, int Ry, int Rx, const FrameShift *__restrict__ shifts,
                                                          const int *__restrict__ fclass,
                                                          const WsHeader *__restrict__ hdr,
                                                          const float *__restrict__ dcls, double *__restrict__ den) {
    extern __shared__ float s_win[];
    __shared__ int s_off[DG_FRAMES], s_ky[DG_FRAMES], s_kx[DG_FRAMES];
    const int ncls = hdr->n_classes;
    if (ncls > kMaxClasses) return;
    const size_t R = (size_t)Ry * Rx;
    const int gx = (Rx + DT_TX - 1) / DT_TX;               // tiles per row (a 1-D grid of tiles)
    const int ty0 = (int)(blockIdx.x / gx) * DT_TY, tx0 = (int)(blockIdx.x % gx) * DT_TX;
    const int lx = threadIdx.x % DT_TX, ly0 = threadIdx.x / DT_TX;
    const int ky0 = hdr->kmin_y, ky1 = hdr->kmax_y, kx0 = hdr->kmin_x, kx1 = hdr->kmax_x;
    const long long HHl = (long long)DT_TY + ky1 - ky0, HWl = (long long)DT_TX + kx1 - kx0;
    const bool staged = HHl * HWl <= DT_CAP;
    const int HH = staged ? (int)HHl : 0, HW = staged ? (int)HWl : 0;
    const int cx = tx0 + lx;
    double acc[DT_RPT];
    float part[DT_RPT];
#pragma unroll
    for (int j = 0; j < DT_RPT; ++j) {
        acc[j] = 0.0;
        part[j] = 0.0f;
    }
    int run = 0;                                          // frames in the FP32 partial sums
    for (int c = 0; c < ncls; ++c) {
        const float *D = dcls + (size_t)c * R;
        if (staged) {
            __syncthreads();                              // the previous class's reads are done
            const int gy0 = ty0 - ky1, gx0 = tx0 - kx1;
            for (int i = threadIdx.x; i < HH * HW; i += DT_THREADS) {
                const int gy = gy0 + i / HW, gx = gx0 + i % HW;
                s_win[i] = ((unsigned)gy < (unsigned)Ry && (unsigned)gx < (unsigned)Rx) ? __ldg(D + (size_t)gy * Rx + gx)
                                                                                       : 0.0f;
            }
        }
        for (int n0 = 0; n0 < N; n0 += DG_FRAMES) {
            const int nf = min(DG_FRAMES, N - n0);
            __syncthreads();
            for (int q = threadIdx.x; q < nf; q += DT_THREADS) {
                const FrameShift f = shifts[n0 + q];
                s_ky[q] = f.ky;
                s_kx[q] = f.kx;
                // the frame's offset in the window; INT_MIN: another class
                s_off[q] = fclass[n0 + q] == c ? (staged ? (ky1 - f.ky) * HW + (kx1 - f.kx) : 0) : INT_MIN;
            }
            __syncthreads();
            for (int q = 0; q < nf; ++q) {
                const int off = s_off[q];
                if (off == INT_MIN) continue;             // the same for the whole block
                if (staged) {
                    const float *p = s_win + ly0 * HW + lx + off;
#pragma unroll
                    for (int j = 0; j < DT_RPT; ++j) part[j] += p[j * (DT_THREADS / DT_TX) * HW];
                } else {
                    const int ky = s_ky[q], kx = s_kx[q];
                    const int tx = cx - kx;
#pragma unroll
                    for (int j = 0; j < DT_RPT; ++j) {
                        const int ty = ty0 + ly0 + j * (DT_THREADS / DT_TX) - ky;
                        if ((unsigned)ty < (unsigned)Ry && (unsigned)tx < (unsigned)Rx)
                            part[j] += __ldg(D + (size_t)ty * Rx + tx);
                    }
                }
                if (++run == 32) {
                    run = 0;
#pragma unroll
                    for (int j = 0; j < DT_RPT; ++j) {
                        acc[j] += part[j];
                        part[j] = 0.0f;
                    }
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < DT_RPT; ++j) {
        acc[j] += part[j];
        const int cy = ty0 + ly0 + j * (DT_THREADS / DT_TX);
        if (cy < Ry && cx < Rx && acc[j] != 0.0) den[(size_t)cy * Rx + cx] += acc[j];
    }
}

__global__ void __launch_bounds__(256) k_normalise(size_t R, const double *__restrict__ num,
                                                   const double *__restrict__ den,
                                                   float *__restrict__ I_ref,
                                                   float *__restrict__ w) {
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < R;
         c += (size_t)gridDim.x * blockDim.x) {
        const double d = den[c];
        I_ref[c] = d > 0.0 ? (float)(num[c] / d) : 0.0f;
        w[c] = (float)d;
    }
}

// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_refterms(int N, int Ry, int Rx,
                                                  const float *__restrict__ Iref,
                                                  const float *__restrict__ w,
                                                  const FrameShift *__restrict__ shifts,
                                                  float *__restrict__ T,
                                                  int32_t *__restrict__ n_valid) {
    const size_t R = (size_t)Ry * Rx;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < R;
         c += (size_t)gridDim.x * blockDim.x) {
        const int cy = (int)(c / Rx), cx = (int)(c % Rx);
        float t = 0.0f;
        int nv = 0;
        for (int n = 0; n < N; ++n) {
            const FrameShift s = shifts[n];
            float Rv;
            if (gather_masked(Iref, w, Ry, Rx, cy + s.ky, cx + s.kx, s.fy, s.fx, Rv)) {
                t = fmaf(Rv, Rv, t);
                ++nv;
            }
        }
        T[c] = t;
        n_valid[c] = nv;
    }
}

int grid_for(size_t n, int threads) {
    size_t b = (n + threads - 1) / threads;
    const size_t cap = (size_t)device_sms() * 16;
    return (int)(b > cap ? cap : (b == 0 ? 1 : b));
}

}  // namespace

cudaError_t launch_prepare(const pxst_dims &d, const double *delta, WsHeader *hdr,
                           FrameShift *shifts, int *fclass, int reset_exact, cudaStream_t stream) {
    k_prepare<<<1, 1024, 0, stream>>>(d.n_frames, delta, hdr, shifts, fclass, reset_exact); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_scatter(const pxst_dims &d, const float *frames, const float *W,
                           const uint8_t *mask, const double *u, const FrameShift *shifts,
                           WsHeader *hdr, double *num, double *den, float *dcls, const int *fclass,
                           cudaStream_t stream) {
    const size_t R = (size_t)d.ref_ny * d.ref_nx;
    cudaError_t e = cudaMemsetAsync(num, 0, sizeof(double) * R, stream);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(den, 0, sizeof(double) * R, stream);
    if (e != cudaSuccess) return e;
    const int smem = 2 * SC_CAP * (int)sizeof(float);
    e = cudaFuncSetAttribute(k_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    ScatterArgs a;
    a.N = d.n_frames; a.ny = d.ny; a.nx = d.nx; a.Ry = d.ref_ny; a.Rx = d.ref_nx;
    a.frames = frames; a.W = W; a.mask = mask; a.u = u; a.shifts = shifts; a.hdr = hdr;
    a.num = num; a.den = den; a.dcls = (dcls && fclass) ? dcls : nullptr;
    const int gx = (d.nx + SC_TX - 1) / SC_TX;
    const int gy = (d.ny + SC_TY - 1) / SC_TY;
    const long long tiles = (long long)gx * gy;
    // split the frames only when there are too few tiles to fill every SM twice
    const long long fill = 2LL * device_sms();
    long long nch = (fill + tiles - 1) / tiles;
    nch = nch < 1 ? 1 : nch;
    const long long maxch = (d.n_frames + 7) / 8;
    if (nch > maxch) nch = maxch;
    if (nch > 65535) nch = 65535;
    a.chunk = (int)((d.n_frames + nch - 1) / nch);
    nch = (d.n_frames + a.chunk - 1) / a.chunk;
    dim3 grid(gx, gy, (unsigned)nch);
    k_scatter<<<grid, SC_THREADS, smem, stream>>>(a); note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (a.dcls) {
        const size_t P = (size_t)d.ny * d.nx;
        k_dzero<<<device_sms() * 8, 256, 0, stream>>>(R, hdr, dcls); note_launch();
        k_dscatter<<<dim3((unsigned)((P + 255) / 256), kMaxClasses), 256, 0, stream>>>(d.ny, d.nx, d.ref_ny, d.ref_nx,
                                                                                     W, mask, u, hdr, dcls); note_launch();
        e = cudaFuncSetAttribute(k_dgather, cudaFuncAttributeMaxDynamicSharedMemorySize, DT_SMEM);
        if (e != cudaSuccess) return e;
        const long long tiles = (long long)((d.ref_nx + DT_TX - 1) / DT_TX) * ((d.ref_ny + DT_TY - 1) / DT_TY);
        k_dgather<<<(unsigned)tiles, DT_THREADS, DT_SMEM, stream>>>(d.n_frames, d.ref_ny, d.ref_nx, shifts, fclass, hdr,
                                                                    dcls, den);
        note_launch();
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_normalise(const pxst_dims &d, const double *num, const double *den,
                             float *I_ref, float *w, cudaStream_t stream) {
    const size_t R = (size_t)d.ref_ny * d.ref_nx;
    k_normalise<<<grid_for(R, 256), 256, 0, stream>>>(R, num, den, I_ref, w); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_refterms(const pxst_dims &d, const float *I_ref, const float *w,
                            const FrameShift *shifts, float *T, int32_t *n_valid,
                            cudaStream_t stream) {
    const size_t R = (size_t)d.ref_ny * d.ref_nx;
    k_refterms<<<grid_for(R, 256), 256, 0, stream>>>(d.n_frames, d.ref_ny, d.ref_nx, I_ref, w,
                                                     shifts, T, n_valid); note_launch();
    return cudaGetLastError();
}

}  // namespace pxst
