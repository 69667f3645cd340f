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
// One cooperative launch runs every step: all blocks are resident, the pixels are split
// over them, and a grid barrier (bounded by %globaltimer: a barrier that runs out sets
// PXST_DEV_TIMEOUT and every block leaves) separates the stencil passes. Per step:
//   A  d = r + beta d_prev (the new search direction, double-buffered) and g = G d;
//   B  q = G^T g (a gather over the equations that read the pixel) and the block's part
//      of d.q;
//   C  psi += alpha d, r -= alpha q and the block's part of r.r.
// The dot products are summed in block order by every block from per-block partial sums,
// so the result does not depend on scheduling. FP64 throughout.
#include <cuda_runtime.h>

#include <algorithm>

#include "pxst_common.cuh"

namespace pxst {
namespace {

constexpr int IG_THREADS = 256;

struct IntegArgs {
    int ny, nx;
    const uint8_t *mask;
    double *u;                 // [2][P], in place
    const uint8_t *type;       // [2][P] stencil of each pixel and axis (0 none)
    double *psi, *r, *d0, *d1, *q, *g;   // [P] each, g [2][P]
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

__global__ void __launch_bounds__(IG_THREADS) k_integ_types(int ny, int nx, const uint8_t *__restrict__ M,
                                                              uint8_t *__restrict__ type) {
    const size_t P = (size_t)ny * nx;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(p / nx), j = (int)(p % nx);
        for (int a = 0; a < 2; ++a) {
            uint8_t code = 0;
            if (M[p]) {
                const int len = a == 0 ? ny : nx, pos = a == 0 ? i : j;
                auto good = [&](int k) {
                    const int t = pos + k;
                    if (t < 0 || t >= len) return false;
                    return M[a == 0 ? (size_t)t * nx + j : (size_t)i * nx + t] != 0;
                };
                if (good(1) && good(-1)) code = 1;
                else if (good(1) && good(2)) code = 2;
                else if (good(-1) && good(-2)) code = 3;
                else if (good(1)) code = 4;
                else if (good(-1)) code = 5;
            }
            type[a * P + p] = code;
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
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return s_ok != 0;
}

// block sum of v, written to part[blockIdx.x]
__device__ void block_partial(double v, double *part) {
    __shared__ double s_red[IG_THREADS / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < IG_THREADS / 32; ++w) s += s_red[w];
        part[blockIdx.x] = s;
    }
    __syncthreads();
}

// the partial sums in block order (every block computes the same value)
__device__ double sum_partials(const double *part) {
    __shared__ double s_tot;
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) s += ((volatile const double *)part)[b];
        s_tot = s;
    }
    __syncthreads();
    const double t = s_tot;
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(IG_THREADS) k_integrate(IntegArgs a) {
    const size_t P = (size_t)a.ny * a.nx;
    const size_t stride = (size_t)gridDim.x * blockDim.x, start = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const int nx = a.nx, ny = a.ny;
    double *part0 = a.part, *part1 = a.part + gridDim.x;
    // g = the data of every equation; then r = d = G^T g (b), psi = 0; |b|^2
    for (size_t p = start; p < P; p += stride)
        for (int s = 0; s < 2; ++s) a.g[s * P + p] = a.type[s * P + p] ? a.u[s * P + p] : 0.0;
    if (!grid_barrier(a.bar, a.limit_ns, a.hdr)) return;
    // the gather of G^T: pixel p collects, along each axis, from the equations of the
    // pixels p - k e (k = -2..2) whose stencil reads p (tap k)
    auto apply_GT = [&](size_t p) {
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
                const int code = a.type[s * P + src];
                if (code) y = fma(tap_at(code, k), a.g[s * P + src], y);
            }
        }
        return y;
    };
    double bb = 0.0;
    {
        double loc = 0.0;
        for (size_t p = start; p < P; p += stride) {
            const double b = apply_GT(p);
            a.r[p] = b;
            a.d0[p] = b;
            a.psi[p] = 0.0;
            loc = fma(b, b, loc);
        }
        block_partial(loc, part0);
        if (!grid_barrier(a.bar, a.limit_ns, a.hdr)) return;
        bb = sum_partials(part0);
    }
    double rr = bb;
    int it = 0;
    double *dc = a.d0, *dn = a.d1;
    double beta = 0.0;
    bool first = true;
    while (it < a.max_iter && rr > a.tol * a.tol * bb && bb > 0.0) {
        // A: the new direction (d = r + beta d_prev, except on the first step) and g = G d,
        //    taking d at every tap from r and d_prev (neither changes in this pass)
        for (size_t p = start; p < P; p += stride) {
            if (!first) dn[p] = fma(beta, dc[p], a.r[p]);
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                int off[3];
                double c[3];
                const int n = stencil_taps(a.type[s * P + p], off, c);
                const long step = s == 0 ? nx : 1;
                double v = 0.0;
                for (int t = 0; t < n; ++t) {
                    const size_t k = (size_t)((long)p + off[t] * step);
                    const double dk = first ? dc[k] : fma(beta, dc[k], a.r[k]);
                    v = fma(c[t], dk, v);
                }
                a.g[s * P + p] = v;
            }
        }
        if (!first) {
            double *t = dc;
            dc = dn;
            dn = t;
        }
        first = false;
        if (!grid_barrier(a.bar, a.limit_ns, a.hdr)) return;
        // B: q = G^T g and d.q
        double loc = 0.0;
        for (size_t p = start; p < P; p += stride) {
            const double qv = apply_GT(p);
            a.q[p] = qv;
            loc = fma(dc[p], qv, loc);
        }
        block_partial(loc, part0);
        if (!grid_barrier(a.bar, a.limit_ns, a.hdr)) return;
        const double dq = sum_partials(part0);
        if (!(dq > 0.0)) break;
        const double alpha = rr / dq;
        // C: the solution and the residual, and r.r
        loc = 0.0;
        for (size_t p = start; p < P; p += stride) {
            a.psi[p] = fma(alpha, dc[p], a.psi[p]);
            const double rv = fma(-alpha, a.q[p], a.r[p]);
            a.r[p] = rv;
            loc = fma(rv, rv, loc);
        }
        block_partial(loc, part1);
        if (!grid_barrier(a.bar, a.limit_ns, a.hdr)) return;
        const double rr_new = sum_partials(part1);
        beta = rr_new / rr;
        rr = rr_new;
        ++it;
    }
    // the output: G psi of every equation (the others keep u)
    for (size_t p = start; p < P; p += stride)
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            int off[3];
            double c[3];
            const int n = stencil_taps(a.type[s * P + p], off, c);
            if (!n) continue;
            const long step = s == 0 ? nx : 1;
            double v = 0.0;
            for (int t = 0; t < n; ++t) v = fma(c[t], a.psi[(size_t)((long)p + off[t] * step)], v);
            a.g[s * P + p] = v;
        }
    if (!grid_barrier(a.bar, a.limit_ns, a.hdr)) return;
    for (size_t p = start; p < P; p += stride)
#pragma unroll
        for (int s = 0; s < 2; ++s)
            if (a.type[s * P + p]) a.u[s * P + p] = a.g[s * P + p];
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
    int blocks = (int)std::min<long long>(want, (long long)per_sm * device_sms());
    blocks = blocks < 1 ? 1 : std::min(blocks, kIntegMaxBlocks);
    k_integ_types<<<(unsigned)std::min<size_t>((P + IG_THREADS - 1) / IG_THREADS, (size_t)device_sms() * 8),
                    IG_THREADS, 0, s>>>(d.ny, d.nx, mask, type);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s)) != cudaSuccess) return e;
    IntegArgs a;
    a.ny = d.ny; a.nx = d.nx; a.mask = mask; a.u = u; a.type = type;
    a.psi = buf; a.r = buf + P; a.d0 = buf + 2 * P; a.d1 = buf + 3 * P; a.q = buf + 4 * P; a.g = buf + 5 * P;
    a.part = buf + 7 * P;
    a.bar = bar; a.hdr = hdr; a.max_iter = max_iter; a.tol = tol;
    a.limit_ns = limit_ns > 0 ? (unsigned long long)limit_ns : 10000000000ull;
    a.info = info;
    void *args[] = {&a};
    e = cudaLaunchCooperativeKernel((const void *)k_integrate, dim3(blocks), dim3(IG_THREADS), args, 0, s);
    note_launch();
    return e;
}

}  // namespace pxst
