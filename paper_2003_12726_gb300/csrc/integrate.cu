// integrate.cu -- the "integrate" option of update_pixel_map (section "Update pixel
// mapping"): the pixel map is the gradient of a scalar, so it is integrated by least
// squares and differentiated again, which removes its curl.
//
// Equations, one per good pixel p and axis a: the derivative of Psi along a at p, by the
// first of these stencils whose pixels are all good -- central (Psi[p+e] - Psi[p-e]) / 2,
// second-order forward (-3 Psi[p] + 4 Psi[p+e] - Psi[p+2e]) / 2, second-order backward
// (3 Psi[p] - 4 Psi[p-e] + Psi[p-2e]) / 2, first-order forward, first-order backward --
// equals u_a[p]. Psi minimises the squared residuals: conjugate gradients on the normal
// equations G^T G Psi = G^T u from Psi = 0. The output u_a[p] = (G Psi) of each equation.
//
// One cooperative launch runs every step: all blocks are resident (two per SM), the pixels
// are split over them, and a grid barrier (bounded by %globaltimer: a barrier that runs out
// sets PXST_DEV_TIMEOUT and every block leaves) separates the passes. The normal operator
// A = G^T G is applied to the residual, so that q = A d follows by the recurrence
// q = A r + beta q_prev (d = r + beta d_prev): the stencil reads r alone and d, q are each
// pixel's own. At a pixel whose equations along an axis are all central differences A is
// (2 x[p] - x[p - 2e] - x[p + 2e]) / 4 on that axis. Per step, two passes:
//   B  d = r + beta d, q = A r + beta q and the block's part of d.q;
//   C  psi += alpha d, r -= alpha q and the block's part of r.r.
// The dot products are summed from per-block partial sums in one fixed order by every
// block, so the result does not depend on scheduling and every block takes the same
// branch. FP64 throughout.
#include <cuda_runtime.h>

#include <algorithm>

#include "pxst_common.cuh"

namespace pxst {
namespace {

constexpr int IG_THREADS = 512;
constexpr int IG_FAST = 8;     // type bit: the axis' equations that read the pixel are central only

struct IntegArgs {
    int ny, nx;
    double *u;                 // [2][P], in place
    const uint8_t *type;       // [2][P] stencil code of each pixel and axis (0 none) | IG_FAST
    double *psi, *r, *d0, *q;  // [P] each
    double *part;              // [2][gridDim.x] per-block partial sums
    unsigned *bar;             // [2] barrier arrival count and generation
    WsHeader *hdr;
    int max_iter;
    double tol;
    unsigned long long limit_ns;
    double *info;              // [2] steps taken, final relative residual (nullable)
};

// stencil codes: 1 central, 2 forward 2nd order, 3 backward 2nd order, 4 forward, 5 backward
__device__ __forceinline__ int stencil_taps(int code, int (&off)[3], double (&c)[3]) {
    switch (code) {
        case 1: off[0] = 1; c[0] = 0.5; off[1] = -1; c[1] = -0.5; return 2;
        case 2: off[0] = 0; c[0] = -1.5; off[1] = 1; c[1] = 2.0; off[2] = 2; c[2] = -0.5; return 3;
        case 3: off[0] = 0; c[0] = 1.5; off[1] = -1; c[1] = -2.0; off[2] = -2; c[2] = 0.5; return 3;
        case 4: off[0] = 1; c[0] = 1.0; off[1] = 0; c[1] = -1.0; return 2;
        case 5: off[0] = 0; c[0] = 1.0; off[1] = -1; c[1] = -1.0; return 2;
        default: return 0;
    }
}

// the coefficient with which the equation of type `code` reads the pixel `k` steps away
__device__ __forceinline__ double tap_at(int code, int k) {
    int off[3];
    double c[3];
    const int n = stencil_taps(code, off, c);
    double v = 0.0;
#pragma unroll
    for (int t = 0; t < 3; ++t)
        if (t < n && off[t] == k) v = c[t];
    return v;
}

// the stencil code of the pixel at `pos` on a line of `len` pixels (good(k): the pixel k
// steps away is inside and good)
template <class Good>
__device__ __forceinline__ int stencil_code(Good good) {
    if (!good(0)) return 0;
    if (good(1) && good(-1)) return 1;
    if (good(1) && good(2)) return 2;
    if (good(-1) && good(-2)) return 3;
    if (good(1)) return 4;
    if (good(-1)) return 5;
    return 0;
}

// Codes, and the IG_FAST bit where the equations along the axis that read the pixel are the
// central ones at p - e and p + e alone: the pixel and both neighbours are central, the
// pixel two behind is not second-order forward and the one two ahead not second-order
// backward (those would read p as well).
__global__ void __launch_bounds__(256) k_integ_types(int ny, int nx, const uint8_t *__restrict__ M,
                                                     uint8_t *__restrict__ type) {
    const size_t P = (size_t)ny * nx;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(p / nx), j = (int)(p % nx);
        for (int a = 0; a < 2; ++a) {
            const int len = a == 0 ? ny : nx, pos = a == 0 ? i : j;
            auto code_at = [&](int k0) {
                return stencil_code([&](int k) {
                    const int t = pos + k0 + k;
                    if (t < 0 || t >= len) return false;
                    return M[a == 0 ? (size_t)t * nx + j : (size_t)i * nx + t] != 0;
                });
            };
            const int code = code_at(0);
            int v = code;
            if (code == 1 && code_at(-1) == 1 && code_at(1) == 1 && code_at(-2) != 2 && code_at(2) != 3) v |= IG_FAST;
            type[a * P + p] = (uint8_t)v;
        }
    }
}

// Grid barrier for a cooperative launch: the last block to arrive resets the count and
// moves the generation on; the others wait for it, at most limit_ns. false: it ran out
// (the status bit is set) and the caller leaves.
__device__ bool grid_barrier(unsigned *bar, unsigned long long limit_ns, WsHeader *hdr) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = bar + 1;
        const unsigned my = *gen;
        __threadfence();
        s_ok = 1;
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            bar[0] = 0;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            unsigned long long t0, t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
            while (*gen == my) {
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
                if (t - t0 > limit_ns) {
                    atomicOr(&hdr->status, PXST_DEV_TIMEOUT);
                    s_ok = 0;
                    break;
                }
                __nanosleep(20);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return s_ok != 0;
}

// Sum over the block of every thread's v, in one fixed order: the values go to shared memory
// and warp 0 adds them (lane l takes threads l, l + 32, ..., then a butterfly, in which every
// lane ends with the same bits since each step adds the same two values in either order).
// FP64 adds are scarce on this GPU, so the other warps do none. Returned to every thread.
__device__ double block_sum(double v) {
    __shared__ double s_val[IG_THREADS];
    __shared__ double s_tot;
    s_val[threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < IG_THREADS / 32; ++k) t += s_val[threadIdx.x + 32 * k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) s_tot = t;
    }
    __syncthreads();
    return s_tot;
}

// the partial sums of all blocks, read and added by warp 0 of every block (lane l takes
// blocks l, l + 32, ..., then a butterfly): the same value in every block
__device__ double sum_partials(const double *part) {
    __shared__ double s_tot;
    if (threadIdx.x < 32) {
        double t = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += 32) t += __ldcg(part + b);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) s_tot = t;
    }
    __syncthreads();
    const double t = s_tot;
    __syncthreads();
    return t;
}

// the block's sum of v, written to part[blockIdx.x]
__device__ __forceinline__ void put_partial(double v, double *part) {
    const double s = block_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(IG_THREADS, 2) k_integrate(IntegArgs a) {
    const size_t P = (size_t)a.ny * a.nx;
    const size_t stride = (size_t)gridDim.x * blockDim.x, start = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    double *part0 = a.part, *part1 = a.part + gridDim.x;
    const uint8_t *__restrict__ type = a.type;

    // (G^T x)[p] along both axes, x_s[src] = xval(s, src) for each equation src: pixel p
    // collects from the equations of the pixels p - k e (k = -2..2) whose stencil reads p
    auto apply_GT = [&](size_t p, auto xval) {
        const int i = (int)(p / nx), j = (int)(p % nx);
        double y = 0.0;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int len = s == 0 ? ny : nx, pos = s == 0 ? i : j;
            const long step = s == 0 ? nx : 1;
#pragma unroll
            for (int k = -2; k <= 2; ++k) {
                if (pos - k < 0 || pos - k >= len) continue;
                const size_t src = (size_t)((long)p - k * step);
                const int code = type[s * P + src] & 7;
                if (code) y = fma(tap_at(code, k), xval(s, src), y);
            }
        }
        return y;
    };

    // (G^T G x)[p] from x at the stencil points: at a pixel whose equations along both axes
    // are central it is x[p] - (x[p - 2 nx] + x[p + 2 nx] + x[p - 2] + x[p + 2]) / 4
    auto apply_A = [&](size_t p, int t0, int t1, const double *x) {
        if ((t0 & t1) & IG_FAST) {
            const double s4 = (x[p - 2 * (size_t)nx] + x[p + 2 * (size_t)nx]) + (x[p - 2] + x[p + 2]);
            return fma(-0.25, s4, x[p]);
        }
        return apply_GT(p, [&](int s, size_t src) {
            int off[3];
            double c[3];
            const int n = stencil_taps(type[s * P + src] & 7, off, c);
            const long step = s == 0 ? nx : 1;
            double v = 0.0;
            for (int t = 0; t < n; ++t) v = fma(c[t], x[(size_t)((long)src + off[t] * step)], v);
            return v;
        });
    };

    // r = G^T u (b), d = q = psi = 0; |b|^2. A pixel that no equation reads (both codes 0:
    // a bad pixel, or a good one without a good neighbour) keeps r = d = q = psi = 0 and is
    // skipped below.
    double bb;
    {
        double loc = 0.0;
        for (size_t p = start; p < P; p += stride) {
            const bool any = (type[p] | type[P + p]) != 0;
            const double b = any ? apply_GT(p, [&](int s, size_t src) { return a.u[s * P + src]; }) : 0.0;
            a.r[p] = b;
            a.d0[p] = 0.0;
            a.q[p] = 0.0;
            a.psi[p] = 0.0;
            loc = fma(b, b, loc);
        }
        put_partial(loc, part0);
        if (!grid_barrier(a.bar, a.limit_ns, a.hdr)) return;
        bb = sum_partials(part0);
    }
    double rr = bb, beta = 0.0;
    int it = 0;
    double *d = a.d0, *q = a.q, *r = a.r, *psi = a.psi;
    while (it < a.max_iter && rr > a.tol * a.tol * bb && bb > 0.0) {
        // B: d = r + beta d and q = G^T G d = G^T G r + beta q (the operator applied to r, read
        //    at the stencil points; d and q are the pixel's own), and d.q (beta = 0 and
        //    d = q = 0 on the first step)
        double loc = 0.0;
        for (size_t p = start; p < P; p += stride) {
            const int t0 = type[p], t1 = type[P + p];
            if (!(t0 | t1)) continue;
            const double sv = apply_A(p, t0, t1, r);
            const double dp = fma(beta, d[p], r[p]);
            const double qv = fma(beta, q[p], sv);
            d[p] = dp;
            q[p] = qv;
            loc = fma(dp, qv, loc);
        }
        put_partial(loc, part0);
        if (!grid_barrier(a.bar, a.limit_ns, a.hdr)) return;
        const double dq = sum_partials(part0);
        if (!(dq > 0.0)) break;
        const double alpha = rr / dq;
        // C: the solution and the residual, and r.r
        loc = 0.0;
        for (size_t p = start; p < P; p += stride) {
            if (!(type[p] | type[P + p])) continue;
            psi[p] = fma(alpha, d[p], psi[p]);
            const double rv = fma(-alpha, q[p], r[p]);
            r[p] = rv;
            loc = fma(rv, rv, loc);
        }
        put_partial(loc, part1);
        if (!grid_barrier(a.bar, a.limit_ns, a.hdr)) return;
        const double rr_new = sum_partials(part1);
        beta = rr_new / rr;
        rr = rr_new;
        ++it;
    }
    // the output: G psi of every equation (the others keep u); psi is final everywhere
    // (the last barrier followed its last update) and u is no longer read
    for (size_t p = start; p < P; p += stride)
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            int off[3];
            double c[3];
            const int n = stencil_taps(type[s * P + p] & 7, off, c);
            if (!n) continue;
            const long step = s == 0 ? nx : 1;
            double v = 0.0;
            for (int t = 0; t < n; ++t) v = fma(c[t], psi[(size_t)((long)p + off[t] * step)], v);
            a.u[s * P + p] = v;
        }
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.info) {
        a.info[0] = (double)it;
        a.info[1] = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    }
}

}  // namespace

cudaError_t launch_integrate(const pxst_dims &d, const uint8_t *mask, double *u, int max_iter, double tol,
                             double *info, uint8_t *type, double *buf, unsigned *bar, WsHeader *hdr,
                             long long limit_ns, cudaStream_t s) {
    const size_t P = (size_t)d.ny * d.nx;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_integrate, IG_THREADS, 0);
    if (e != cudaSuccess) return e;
    const long long want = (long long)((P + IG_THREADS - 1) / IG_THREADS);
    int blocks = (int)std::min<long long>(want, (long long)std::min(per_sm, 2) * device_sms());
    blocks = blocks < 1 ? 1 : std::min(blocks, kIntegMaxBlocks);
    k_integ_types<<<(unsigned)std::min<size_t>((P + 255) / 256, (size_t)device_sms() * 8), 256, 0, s>>>(
        d.ny, d.nx, mask, type);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s)) != cudaSuccess) return e;
    IntegArgs a;
    a.ny = d.ny; a.nx = d.nx; a.u = u; a.type = type;
    a.psi = buf; a.r = buf + P; a.d0 = buf + 2 * P; a.q = buf + 3 * P;
    a.part = buf + 4 * P;
    a.bar = bar; a.hdr = hdr; a.max_iter = max_iter; a.tol = tol;
    a.limit_ns = limit_ns > 0 ? (unsigned long long)limit_ns : 10000000000ull;
    a.info = info;
    void *args[] = {&a};
    e = cudaLaunchCooperativeKernel((const void *)k_integrate, dim3(blocks), dim3(IG_THREADS), args, 0, s);
    note_launch();
    return e;
}

}  // namespace pxst
