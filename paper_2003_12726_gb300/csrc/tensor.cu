// tensor.cu -- tensor-core (tcgen05) precision forms of update_pixel_map on sm_103a.
//
// Kernels: the operand preparation (k_tprep, k_gtable, k_tsquare), the tensor-core ranking
// of every candidate (k_tsearch, and its masked pass) and a diagnostic contraction (k_tc_check) that checks the tcgen05
// machinery: TMA loads with 128-byte swizzle into shared memory, tcgen05.mma accumulating
// in TMEM, and tcgen05.ld read-back.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <mutex>

#include <cuda_bf16.h>
#include <climits>
#include <type_traits>

#include "pxst_common.cuh"
#include "tc_ptx.cuh"

namespace pxst {

// ---- host: tensor-map encoding through the driver entry point ----------------------------
namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_enc_mu;
}  // namespace

cudaError_t tmap_encode(CUtensorMap *map, CUtensorMapDataType dt, uint32_t rank, void *base,
                        const uint64_t *dims, const uint64_t *strides_bytes, const uint32_t *box, bool swizzle128) {
    {
        std::lock_guard<std::mutex> g(g_enc_mu);
        if (!g_encode) {
            cudaDriverEntryPointQueryResult q;
            void *fn = nullptr;
            cudaError_t e = cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q);
            if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        }
    }
    uint32_t estride[5] = {1, 1, 1, 1, 1};
    CUresult r = g_encode(map, dt, rank, base, dims, strides_bytes, box, estride,
                          CU_TENSOR_MAP_INTERLEAVE_NONE,
                          swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

namespace {

// ---- diagnostic contraction ----------------------------------------------------------------
template <bool TF32>
__global__ void __launch_bounds__(128) k_tc_check(const __grid_constant__ CUtensorMap ta,
                                                  const __grid_constant__ CUtensorMap tb, int K,
                                                  float *__restrict__ D, int *__restrict__ status) {
    constexpr int KB = TF32 ? 32 : 64;       // elements in one 128-byte row
    constexpr int KSTEP = TF32 ? 8 : 16;     // K of one MMA
    constexpr uint32_t IDESC = tc::instr_desc(TF32 ? 2u : 1u, 128, 256);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *As = smem;                      // 128 rows x 128 B
    uint8_t *Bs = smem + 128 * 128;          // 256 rows x 128 B
    __shared__ __align__(8) uint64_t bar_full, bar_mma;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5;
    volatile int *abortp = &abort_flag;
    if (tid == 0) {
        *abortp = 0;
        tc::mbar_init(&bar_full, 1);
        tc::mbar_init(&bar_mma, 1);
        tc::fence_mbar_init();
        tc::prefetch_tmap(&ta);
        tc::prefetch_tmap(&tb);
    }
    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, 256);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tmem_base;

    const int nkb = (K + KB - 1) / KB;
    for (int kb = 0; kb < nkb; ++kb) {
        if (tid == 0 && !*abortp) {
            const uint32_t ph = kb & 1;
            tc::mbar_expect_tx(&bar_full, (128 + 256) * 128);
            tc::tma_load_2d(As, &ta, &bar_full, kb * KB, 0);
            tc::tma_load_2d(Bs, &tb, &bar_full, kb * KB, 0);
            if (!tc::mbar_wait(&bar_full, ph, abortp)) {
                *abortp = 1;
            } else {
                tc::tc_fence_after();
                const uint32_t a0 = tc::smem_u32(As), b0 = tc::smem_u32(Bs);
#pragma unroll
                for (int k = 0; k < KB / KSTEP; ++k)
                    tc::mma<TF32>(tmem, tc::smem_desc_sw128(a0 + k * 32), tc::smem_desc_sw128(b0 + k * 32),
                                  IDESC, (kb > 0 || k > 0) ? 1u : 0u);
                tc::mma_commit(&bar_mma);
                if (!tc::mbar_wait(&bar_mma, ph, abortp)) *abortp = 1;
            }
        }
        __syncthreads();
        if (*abortp) break;
    }
    tc::tc_fence_after();
    if (!*abortp) {
        for (int c = 0; c < 256; c += 32) {
            float v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + c, v);
            const int row = warp * 32 + (tid & 31);
#pragma unroll
            for (int i = 0; i < 32; ++i) D[row * 256 + c + i] = v[i];
        }
    } else if (tid == 0) {
        atomicOr(status, PXST_DEV_TIMEOUT);
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

// ==========================================================================================
// Precision form of update_pixel_map.
//
// Centred operands: A~_n(x) = I_n(x)/W(x) - 1 and G~_n(c) = V_n(c) (R_n(c) - 1), so that for
// a pixel whose candidates are all valid
//     error(c) / var = 1 + (T~(c) - 2 C~(x, c)) / sum_n A~_n(x)^2,
//     C~(x, c) = sum_n A~_n(x) G~_n(c),  T~(c) = sum_n G~_n(c)^2,
// and the candidates of one pixel are ranked by q = T~(c) - 2 C~(x, c). C~ is a dense
// contraction over frames for a tile of pixels against the union of their windows: it
// runs on the tensor cores (BF16 or TF32 operands, FP32 accumulation in TMEM). The best
// few candidates per pixel are then evaluated exactly in FP32 by the search kernel.
// ==========================================================================================

// A~ [Npad/KB][ny][nx][KB] (frame blocks of one 128-byte operand row, zero for masked
// pixels and padding frames): one block per frame block x 64 pixels. The frames are read in
// coalesced rows of 64 pixels, transposed through shared memory and written as 16-byte
// pieces of each pixel's operand row (a warp writes 512 contiguous bytes).
// The frame-block-major layout makes each TMA box a few contiguous runs of pixels.
constexpr int TP_PIX = 64;
template <typename T>
__global__ void __launch_bounds__(256) k_tprep(int N, int ny, int nx, const float *__restrict__ frames,
                                               const float *__restrict__ W,
                                               const uint8_t *__restrict__ mask, T *__restrict__ At,
                                               WsHeader *__restrict__ hdr) {
    constexpr int KB = 128 / sizeof(T);       // frames per operand row
    constexpr int EPP = 16 / sizeof(T);       // elements per 16-byte piece
    __shared__ float tile[KB][TP_PIX + 1];
    const size_t P = (size_t)ny * nx;
    const size_t p0 = (size_t)blockIdx.x * TP_PIX;
    const int kb = blockIdx.y, n0 = kb * KB;
    const int col = threadIdx.x & (TP_PIX - 1), r0 = threadIdx.x / TP_PIX;   // 4 rows of 64
    const size_t p = p0 + col;
    const float Wp = p < P ? __ldg(W + p) : 0.0f;
    const bool on = p < P && mask[p] && Wp > 0.0f && isfinite(Wp);   // usable pixels only
    // the operand only ranks candidates, so I * (1/W) stands in for I / W
    const float rw = on ? __frcp_rn(Wp) : 0.0f;
    float f[KB / 4];
#pragma unroll
    for (int i = 0; i < KB / 4; ++i) {            // every load in flight before the first use
        const int n = n0 + r0 + 4 * i;
        f[i] = (on && n < N) ? __ldcs(frames + (size_t)n * P + p) : 0.0f;
    }
    bool bad = false;
#pragma unroll
    for (int i = 0; i < KB / 4; ++i) bad |= !isfinite(f[i]);
    if (bad) atomicOr(&hdr->status, PXST_DEV_BAD_INPUT);
#pragma unroll
    for (int i = 0; i < KB / 4; ++i) {
        const int n = n0 + r0 + 4 * i;
        tile[r0 + 4 * i][col] = (on && n < N) ? fmaf(f[i], rw, -1.0f) : 0.0f;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < TP_PIX * 8; q += 256) {
        const int pp = q >> 3, piece = q & 7;    // pixel of the block, 16-byte piece of its row
        if (p0 + pp >= P) continue;
        uint4 out;
        T *o = reinterpret_cast<T *>(&out);
#pragma unroll
        for (int e = 0; e < EPP; ++e) o[e] = T(tile[piece * EPP + e][pp]);
        *reinterpret_cast<uint4 *>(At + ((size_t)kb * P + p0 + pp) * KB + piece * EPP) = out;
    }
}

// A~^2 (the masked ranking's variance operand, in A~'s layout) for the tiles the masked
// ranking visits: one block per listed tile, of which those beyond the list's length return
// at once; 16-byte pieces of the tile's operand rows, squared elementwise.
template <typename T>
__global__ void __launch_bounds__(256) k_tsquare(int nkb, int ny, int nx, int pty, int tiles_x,
                                                 const WsHeader *__restrict__ hdr, const int *__restrict__ tile_list,
                                                 const T *__restrict__ At, T *__restrict__ A2) {
    constexpr int KB = 128 / sizeof(T), EPP = 16 / sizeof(T);
    if ((int)blockIdx.x >= hdr->n_edge_tiles) return;
    const int tl = tile_list[blockIdx.x];
    const int tx = 128 / pty;
    const int x0 = (tl % tiles_x) * tx, y0 = (tl / tiles_x) * pty;
    const size_t P = (size_t)ny * nx;
    for (int q = threadIdx.x; q < nkb * 128 * 8; q += 256) {
        const int piece = q & 7, pix = (q >> 3) & 127, kb = q >> 10;
        const int x = x0 + pix % tx, y = y0 + pix / tx;
        if (x >= nx || y >= ny) continue;
        const size_t o = ((size_t)kb * P + (size_t)y * nx + x) * KB + piece * EPP;
        uint4 v = *reinterpret_cast<const uint4 *>(At + o);
        T *e = reinterpret_cast<T *>(&v);
#pragma unroll
        for (int k = 0; k < EPP; ++k) {
            const float f = float(e[k]);
            e[k] = T(f * f);
        }
        *reinterpret_cast<uint4 *>(A2 + o) = v;
    }
}

// The reference with uncovered pixels as NaN (the gathers below and the exact rescore read it).
__global__ void __launch_bounds__(256) k_rmask(size_t R, const float *__restrict__ Iref,
                                               const float *__restrict__ w, float *__restrict__ Rm) {
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < R; c += (size_t)gridDim.x * blockDim.x)
        Rm[c] = __ldg(w + c) > 0.0f ? __ldg(Iref + c) : __int_as_float(0x7fc00000);
}

// G~ [Npad/KB][Ry][Rx][KB], the validity V (0 or 1) in the same layout, T~ and n_valid,
// gathered from the NaN-masked reference: one block per 32 consecutive reference pixels. For
// each frame block the block stages the frames' shifts (and, for whole-pixel shifts, the
// flat offset ky Rx + kx) in shared memory; the 8 warps gather with lanes over the 32 pixels
// (one frame's reads coalesce), each thread forming one 32-bit word of its pixel's operand
// row at a time (two BF16 frames or one FP32 frame), and the words are transposed through
// shared memory and written as 32 operand rows of 128 bytes (4 KB contiguous per array).
// When every shift is a whole pixel, a pixel whose reads stay on the grid for every frame
// reads each frame with one load at its flat offset, without bounds tests.
template <typename T>
__global__ void __launch_bounds__(256) k_gtable(int N, int Npad, int Ry, int Rx, const float *__restrict__ Rm,
                                                const FrameShift *__restrict__ shifts,
                                                const WsHeader *__restrict__ hdr, T *__restrict__ G,
                                                T *__restrict__ V, float *__restrict__ Tt,
                                                int *__restrict__ nvalid) {
    constexpr int KB = 128 / sizeof(T);
    constexpr int EW = 4 / sizeof(T);              // frames per 32-bit word
    constexpr int RW = 33;                         // words per padded shared row (32 + 1)
    __shared__ uint32_t sg[32 * RW], sv[32 * RW];
    __shared__ int s_off[KB], s_ky[KB], s_kx[KB];
    __shared__ float s_fy[KB], s_fx[KB];
    __shared__ float s_t[8][32];
    __shared__ int s_n[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t R = (size_t)Ry * Rx;
    const size_t c0 = (size_t)blockIdx.x * 32, c = c0 + lane;
    const bool inr = c < R;
    const int cy = inr ? (int)(c / Rx) : 0, cx = inr ? (int)(c % Rx) : 0;
    // every frame's whole-pixel read of this pixel stays on the grid (then |ky| < Ry and
    // |kx| < Rx, so c + ky Rx + kx fits an int, as R does)
    const bool interior = inr && cy + hdr->kmin_y >= 0 && cy + hdr->kmax_y < Ry && cx + hdr->kmin_x >= 0 &&
                          cx + hdr->kmax_x < Rx;
    // every frame's shift is a whole pixel (one fraction class, zero)
    const bool whole = hdr->n_classes == 1 && hdr->cls_fy[0] == 0.0f && hdr->cls_fx[0] == 0.0f;
    float t = 0.0f;
    int nv = 0;
    const int nkb = Npad / KB;
    for (int kb = 0; kb < nkb; ++kb) {
        if (threadIdx.x < KB) {
            const int n = kb * KB + threadIdx.x;
            const FrameShift f = n < N ? shifts[n] : FrameShift{0, 0, 0.0f, 0.0f};
            s_ky[threadIdx.x] = f.ky;
            s_kx[threadIdx.x] = f.kx;
            s_fy[threadIdx.x] = f.fy;
            s_fx[threadIdx.x] = f.fx;
            s_off[threadIdx.x] = (int)((long long)f.ky * Rx + f.kx);
        }
        __syncthreads();
        // one word of the pixel's operand row from its frames' reads (g: R - 1, val: valid)
        auto put = [&](int k, const float (&g)[EW], const bool (&val)[EW]) {
            uint32_t wg, wv;
            if constexpr (EW == 2) {
                const __nv_bfloat162 gb = __floats2bfloat162_rn(g[0], g[1]);
                const float g0 = __low2float(gb), g1 = __high2float(gb);
                t = fmaf(g0, g0, t);
                t = fmaf(g1, g1, t);
                wg = *reinterpret_cast<const uint32_t *>(&gb);
                wv = (val[0] ? 0x3f80u : 0u) | (val[1] ? 0x3f800000u : 0u);     // BF16 1.0 in each half
            } else {
                t = fmaf(g[0], g[0], t);
                wg = __float_as_uint(g[0]);
                wv = val[0] ? 0x3f800000u : 0u;
            }
#pragma unroll
            for (int e = 0; e < EW; ++e) nv += val[e] ? 1 : 0;
            sg[lane * RW + k] = wg;
            sv[lane * RW + k] = wv;
        };
        if (whole && interior) {
            // every shift whole and every read of this pixel on the grid: one load per frame
#pragma unroll
            for (int i = 0; i < 32 / 8; ++i) {
                const int k = warp + 8 * i;
                float g[EW];
                bool val[EW];
#pragma unroll
                for (int e = 0; e < EW; ++e) {
                    const int j = k * EW + e;
                    const float Rv = kb * KB + j < N ? __ldg(Rm + ((int)c + s_off[j])) : __int_as_float(0x7fc00000);
                    val[e] = Rv == Rv;
                    g[e] = val[e] ? Rv - 1.0f : 0.0f;
                }
                put(k, g, val);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 32 / 8; ++i) {
                const int k = warp + 8 * i;
                float g[EW];
                bool val[EW];
#pragma unroll
                for (int e = 0; e < EW; ++e) {
                    const int j = k * EW + e, n = kb * KB + j;
                    g[e] = 0.0f;
                    val[e] = false;
                    if (inr && n < N) {
                        float Rv = 0.0f;
                        val[e] = gather_rm(Rm, Ry, Rx, cy + s_ky[j], cx + s_kx[j], s_fy[j], s_fx[j], Rv);
                        if (val[e]) g[e] = Rv - 1.0f;
                    }
                }
                put(k, g, val);
            }
        }
        __syncthreads();
        uint32_t *G32 = reinterpret_cast<uint32_t *>(G) + (size_t)kb * R * 32;
        uint32_t *V32 = reinterpret_cast<uint32_t *>(V) + (size_t)kb * R * 32;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int q = threadIdx.x + 256 * i, r = q >> 5, k = q & 31;
            if (c0 + r < R) {
                G32[(c0 + r) * 32 + k] = sg[r * RW + k];
                V32[(c0 + r) * 32 + k] = sv[r * RW + k];
            }
        }
        // the next frame block's shifts are written after every thread has read this one's
        // words (its first barrier)
    }
    s_t[warp][lane] = t;
    s_n[warp][lane] = nv;
    __syncthreads();
    if (warp == 0 && inr) {
        float tt = 0.0f;
        int nn = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            tt += s_t[k][lane];
            nn += s_n[k][lane];
        }
        Tt[c] = tt;
        nvalid[c] = nn;
    }
}

// Tile shapes (template parameters PTY, CCW): a pixel tile of PTY x (128 / PTY) pixels
// (M = 128) against candidate chunks of (256 / CCW) x CCW reference pixels (N = 256).
// Shape 0: 8 x 16 pixels, 8 x 32 candidates; 1: 4 x 32, 4 x 64; 2: 2 x 64, 2 x 128.
constexpr int TS_STAGES = 4;
constexpr int TS_EPG = 3;                     // epilogue warps per TMEM lane quarter
constexpr int TS_EPI_WARPS = 4 * TS_EPG;      // they split a chunk's 8 segments: g = h, h + 3, ...
constexpr int TS_THREADS = 64 + 32 * TS_EPI_WARPS;   // producer, MMA, epilogue warps
constexpr int TS_A_BYTES = 128 * 128, TS_B_BYTES = 256 * 128;
constexpr int TS_SMEM = TS_STAGES * (TS_A_BYTES + TS_B_BYTES) + 1024;
// masked ranking: each stage holds A~, A~^2, G~ and V; two stages
constexpr int TSM_STAGES = 2;
constexpr int TSM_SMEM = TSM_STAGES * 2 * (TS_A_BYTES + TS_B_BYTES) + 1024;
constexpr int TS_MAX_ORDER = 64;              // chunk rows / columns visited centre-first

struct TSearchArgs {
    int N, Npad, ny, nx, Ry, Rx, Sy, Sx;
    const uint8_t *mask;
    const double *u;
    const float *Tt;
    const int *nvalid;
    WsHeader *hdr;
    int *cand;          // [P][kTopK] window indices of the best candidates, best first (-1: none)
    uint8_t *edge;      // [P] 1: a candidate of the pixel reads an invalid reference pixel
    int *tile_list;     // tiles holding such pixels, hdr->n_edge_tiles of them (any order)
    int tiles_x;        // tiles per detector row (to decode a listed tile)
    const float *W;     // masked ranking: the whitefield (the key of a zero-variance candidate)
    int ares;           // first pass: 0 = A~ streams with G~; k > 0 = A~ resident, k G~ stages
    unsigned long long limit_ns;   // bound of every pipeline wait (pxst_options.timeout_ns)
};

// Insert (qv, idx) into the ascending list bq/bi when it beats an entry (strict <, so of
// equal keys the one seen first stays ahead). Every position is decided from the old list
// in parallel, so the update is three dependent steps deep whatever the list length.
template <int TK>
__device__ __forceinline__ void topk_insert(float (&bq)[TK], int (&bi)[TK], float qv, int idx) {
    bool lt[TK];
#pragma unroll
    for (int m = 0; m < TK; ++m) lt[m] = qv < bq[m];
#pragma unroll
    for (int m = TK - 1; m > 0; --m) {
        bq[m] = lt[m] ? (lt[m - 1] ? bq[m - 1] : qv) : bq[m];
        bi[m] = lt[m] ? (lt[m - 1] ? bi[m - 1] : idx) : bi[m];
    }
    bq[0] = lt[0] ? qv : bq[0];
    bi[0] = lt[0] ? idx : bi[0];
}

// One chunk row of 32 candidates for the warp's 32 pixels: q = T~ - 2 C~, where sT holds
// T~ (+inf for a candidate that is not valid in every frame). Lanes whose window does not
// hold column i (bit i of inmask clear) skip it. The segment's keys are formed first; if
// none of them beats any lane's K-th key (the lists only improve, so none could later in
// the segment either), the segment is done with one vote; otherwise the insertion runs,
// candidate by candidate, only when some lane of the warp improves its list.
template <int TK, bool FULL>
__device__ __forceinline__ void scan_row(const float (&v)[32], const float *__restrict__ sT, uint32_t inmask,
                                         int rowbase, float (&bq)[TK], int (&bi)[TK]) {
    float q[32];
    float mn = INFINITY;
#pragma unroll
    for (int i4 = 0; i4 < 32; i4 += 4) {
        const float4 t4 = *reinterpret_cast<const float4 *>(sT + i4);
        const float tt[4] = {t4.x, t4.y, t4.z, t4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int i = i4 + e;
            q[i] = fmaf(-2.0f, v[i], tt[e]);
            if (!FULL) q[i] = ((inmask >> i) & 1u) ? q[i] : INFINITY;
            mn = fminf(mn, q[i]);
        }
    }
    if (!__any_sync(0xffffffffu, mn < bq[TK - 1])) return;
#pragma unroll
    for (int i = 0; i < 32; ++i)
        if (__any_sync(0xffffffffu, q[i] < bq[TK - 1])) topk_insert<TK>(bq, bi, q[i], rowbase + i);
}

// The masked ranking's segment: with S = sum_n V A~^2 (second accumulator), a candidate's
// error over its valid frames is 1 + (T~ - 2 C~) / S, so the key is (T~ - 2 C~) / S; where
// S = 0 the error is W^2 T~ (not normalised), key W^2 T~ - 1; sT holds T~ (+inf for a
// candidate with no valid frame).
template <int TK>
__device__ __forceinline__ void scan_row_masked(const float (&v)[32], const float (&v2)[32],
                                                const float *__restrict__ sT, uint32_t use, int rowbase, float W2,
                                                float (&bq)[TK], int (&bi)[TK]) {
    float q[32];
    float mn = INFINITY;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const float t = sT[i];
        const float qv = v2[i] > 0.0f ? __fdividef(fmaf(-2.0f, v[i], t), v2[i]) : fmaf(W2, t, -1.0f);
        q[i] = (((use >> i) & 1u) && t < INFINITY) ? qv : INFINITY;
        mn = fminf(mn, q[i]);
    }
    if (!__any_sync(0xffffffffu, mn < bq[TK - 1])) return;
#pragma unroll
    for (int i = 0; i < 32; ++i)
        if (__any_sync(0xffffffffu, q[i] < bq[TK - 1])) topk_insert<TK>(bq, bi, q[i], rowbase + i);
}

// Visit order of n chunk rows (or columns): the one holding the tile's centre first, then
// alternately outwards, so that the best candidates are met early and later chunks rarely
// change a pixel's list.
__device__ inline void centre_first(int *ord, int n, int c) {
    c = min(max(c, 0), n - 1);
    int k = 0;
    ord[k++] = c;
    for (int d = 1; k < n; ++d) {
        if (c + d < n) ord[k++] = c + d;
        if (c - d >= 0 && k < n) ord[k++] = c - d;
    }
}

// MASKED: the second pass over the listed tiles, which ranks every candidate of their pixels
// that have candidates not valid in every frame, with both contractions in TMEM (one
// 512-column buffer: D1 = A~ G~^T at column 0, D2 = A~^2 V^T at column 256).
template <bool TF32, int TK, int PTY, int CCW, bool MASKED>
__global__ void __launch_bounds__(TS_THREADS, 1) k_tsearch(const __grid_constant__ CUtensorMap tA,
                                                           const __grid_constant__ CUtensorMap tB,
                                                           const __grid_constant__ CUtensorMap tA2,
                                                           const __grid_constant__ CUtensorMap tV,
                                                           TSearchArgs a) {
    constexpr int TS_TY = PTY, TS_TX = 128 / PTY;  // pixel tile
    constexpr int TS_CR = 256 / CCW, TS_CC = CCW;  // candidate chunk
    constexpr int SPR = CCW / 32;                  // 32-candidate segments per chunk row
    static_assert(TS_TY * TS_TX == 128 && TS_CR * TS_CC == 256 && SPR >= 1, "tile shape");
    constexpr int KB = TF32 ? 32 : 64;       // frames per 128-byte operand row
    constexpr int KSTEP = TF32 ? 8 : 16;     // frames per MMA
    constexpr uint32_t IDESC = tc::instr_desc(TF32 ? 2u : 1u, 128, 256);
    constexpr int NBUF = MASKED ? 1 : 2;                                // TMEM accumulator buffers
    // A-resident mode: the tile's A~ (the same for every chunk) is loaded once, before the
    // chunks, and only G~ streams through the stage ring
    const int ares = MASKED ? 0 : a.ares;
    const int NS = ares ? ares : (MASKED ? TSM_STAGES : TS_STAGES);    // pipeline stages
    const int SB = ares ? TS_B_BYTES : (MASKED ? 2 : 1) * (TS_A_BYTES + TS_B_BYTES);   // bytes per stage
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t bar_full[TS_STAGES], bar_empty[TS_STAGES], bar_tfull[2], bar_tempty[2];
    __shared__ __align__(8) uint64_t bar_afull;       // A-resident mode: every A~ block landed
    __shared__ int s_tile_edge;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ int s_box[4];
    __shared__ int s_ci[128], s_cj[128], s_act[128];
    __shared__ int s_rord[TS_MAX_ORDER], s_cord[TS_MAX_ORDER];
    __shared__ __align__(16) float s_T[2][256];
    __shared__ uint32_t s_vm[2][8];
    __shared__ float s_mq[TS_EPG - 1][128][TK];      // the lists of the warps h > 0, merged by h = 0
    __shared__ int s_mi[TS_EPG - 1][128][TK];
    __shared__ uint8_t s_medge[TS_EPG - 1][128];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const size_t P = (size_t)a.ny * a.nx;
    int tile_x = blockIdx.x, tile_y = blockIdx.y;
    if (MASKED) {
        // the listed tiles only
        if ((int)blockIdx.x >= a.hdr->n_edge_tiles) return;
        const int t = a.tile_list[blockIdx.x];
        tile_x = t % a.tiles_x;
        tile_y = t / a.tiles_x;
    }
    const int x0 = tile_x * TS_TX, y0 = tile_y * TS_TY;
    volatile int *abortp = &abort_flag;

    if (tid < 4) s_box[tid] = (tid & 1) ? INT_MIN : INT_MAX;
    if (tid == 0) {
        *abortp = 0;
        s_tile_edge = 0;
    }
    __syncthreads();
    if (tid < 128) {
        const int x = x0 + (tid % TS_TX), y = y0 + (tid / TS_TX);
        int act = 0, ci = 0, cj = 0;
        if (x < a.nx && y < a.ny) {
            const size_t pix = (size_t)y * a.nx + x;
            const double u0 = a.u[pix], u1 = a.u[P + pix];
            const float Wp = a.W[pix];
            if (a.mask[pix] && isfinite(u0) && isfinite(u1) && fabs(u0) <= kMaxCoord && fabs(u1) <= kMaxCoord &&
                Wp > 0.0f && isfinite(Wp)) {
                ci = (int)floor(u0 + 0.5);
                cj = (int)floor(u1 + 0.5);
                act = 1;
                atomicMin(&s_box[0], ci); atomicMax(&s_box[1], ci);
                atomicMin(&s_box[2], cj); atomicMax(&s_box[3], cj);
            }
        }
        s_act[tid] = act;
        s_ci[tid] = ci;
        s_cj[tid] = cj;
    }
    __syncthreads();
    if (s_box[0] == INT_MAX) return;                  // nothing to do in this tile

    const int ur0 = s_box[0] - a.Sy, uc0 = s_box[2] - a.Sx;
    const int nrc = (s_box[1] - s_box[0] + 2 * a.Sy + TS_CR) / TS_CR;
    const int ncc = (s_box[3] - s_box[2] + 2 * a.Sx + TS_CC) / TS_CC;
    const int nchunks = nrc * ncc;
    const int nkb = a.Npad / KB;
    const bool ordered = nrc <= TS_MAX_ORDER && ncc <= TS_MAX_ORDER;
    uint8_t *stage0 = smem + (ares ? nkb * TS_A_BYTES : 0);     // the stage ring

    if (tid == 0) {
        for (int i = 0; i < NS; ++i) {
            tc::mbar_init(&bar_full[i], 1);
            tc::mbar_init(&bar_empty[i], 1);
        }
        tc::mbar_init(&bar_afull, 1);
        for (int i = 0; i < NBUF; ++i) {
            tc::mbar_init(&bar_tfull[i], 1);
            tc::mbar_init(&bar_tempty[i], TS_EPI_WARPS);
        }
        tc::fence_mbar_init();
        tc::prefetch_tmap(&tA);
        tc::prefetch_tmap(&tB);
        if (MASKED) {
            tc::prefetch_tmap(&tA2);
            tc::prefetch_tmap(&tV);
        }
        if (ordered) {
            centre_first(s_rord, nrc, ((s_box[0] + s_box[1]) / 2 - ur0) / TS_CR);
            centre_first(s_cord, ncc, ((s_box[2] + s_box[3]) / 2 - uc0) / TS_CC);
        }
    }
    if (warp == 1) {
        tc::tmem_alloc(&tmem_base, 512);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tmem_base;
    // origin (reference row, column) of the j-th chunk visited
    auto chunk_origin = [&](int j, int &row0, int &col0) {
        const int jr = j / ncc, jc = j % ncc;
        row0 = ur0 + TS_CR * (ordered ? s_rord[jr] : jr);
        col0 = uc0 + TS_CC * (ordered ? s_cord[jc] : jc);
    };

    if (warp == 0) {
        // ---- TMA producer ---------------------------------------------------------------
        if (lane == 0) {
            if (ares) {
                // the tile's A~, all frame blocks, once
                tc::mbar_expect_tx(&bar_afull, (uint32_t)(nkb * TS_A_BYTES));
                for (int kb = 0; kb < nkb; ++kb) tc::tma_load_4d(smem + kb * TS_A_BYTES, &tA, &bar_afull, 0, x0, y0, kb);
            }
            int it = 0;
            for (int j = 0; j < nchunks && !*abortp; ++j) {
                int row0, col0;
                chunk_origin(j, row0, col0);
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % NS;
                    if (!tc::mbar_wait(&bar_empty[s], ((it / NS) & 1) ^ 1, abortp, a.limit_ns)) {
                        *abortp = 1;
                        break;
                    }
                    if (ares) {
                        tc::mbar_expect_tx(&bar_full[s], SB);
                        tc::tma_load_4d(stage0 + s * SB, &tB, &bar_full[s], 0, col0, row0, kb);
                        continue;
                    }
                    // stage layout: A~ | G~ (| A~^2 | V)
                    uint8_t *As = smem + s * SB;
                    uint8_t *Bs = As + TS_A_BYTES;
                    tc::mbar_expect_tx(&bar_full[s], SB);
                    tc::tma_load_4d(As, &tA, &bar_full[s], 0, x0, y0, kb);
                    tc::tma_load_4d(Bs, &tB, &bar_full[s], 0, col0, row0, kb);
                    if (MASKED) {
                        tc::tma_load_4d(Bs + TS_B_BYTES, &tA2, &bar_full[s], 0, x0, y0, kb);
                        tc::tma_load_4d(Bs + TS_B_BYTES + TS_A_BYTES, &tV, &bar_full[s], 0, col0, row0, kb);
                    }
                }
            }
            // let every copy this CTA issued land before the CTA can exit
            for (int k = 0; k < NS && k < it; ++k) {
                const int i2 = it - 1 - k, s = i2 % NS;
                volatile int never = 0;
                tc::mbar_wait(&bar_full[s], (i2 / NS) & 1, &never, a.limit_ns);
            }
            if (ares) {
                volatile int never = 0;
                tc::mbar_wait(&bar_afull, 0, &never, a.limit_ns);
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer -------------------------------------------------------------------
        if (lane == 0) {
            int it = 0;
            if (ares && !tc::mbar_wait(&bar_afull, 0, abortp, a.limit_ns)) *abortp = 1;
            for (int j = 0; j < nchunks && !*abortp; ++j) {
                const int buf = j % NBUF;
                if (!tc::mbar_wait(&bar_tempty[buf], ((j / NBUF) & 1) ^ 1, abortp, a.limit_ns)) {
                    *abortp = 1;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t d = tmem + buf * 256;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % NS;
                    if (!tc::mbar_wait(&bar_full[s], (it / NS) & 1, abortp, a.limit_ns)) {
                        *abortp = 1;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint32_t a0 = ares ? tc::smem_u32(smem + kb * TS_A_BYTES) : tc::smem_u32(smem + s * SB);
                    const uint32_t b0 = ares ? tc::smem_u32(stage0 + s * SB) : a0 + TS_A_BYTES;
                    const uint32_t a20 = b0 + TS_B_BYTES, v0 = a20 + TS_A_BYTES;
#pragma unroll
                    for (int k = 0; k < KB / KSTEP; ++k) {
                        tc::mma<TF32>(d, tc::smem_desc_sw128(a0 + k * 32), tc::smem_desc_sw128(b0 + k * 32),
                                      IDESC, (kb > 0 || k > 0) ? 1u : 0u);
                        if (MASKED)
                            tc::mma<TF32>(tmem + 256, tc::smem_desc_sw128(a20 + k * 32),
                                          tc::smem_desc_sw128(v0 + k * 32), IDESC, (kb > 0 || k > 0) ? 1u : 0u);
                    }
                    tc::mma_commit(&bar_empty[s]);
                }
                if (*abortp) break;
                tc::mma_commit(&bar_tfull[buf]);
            }
        }
    } else {
        // ---- epilogue: 4 x TS_EPG warps; TMEM lane quarter q = warp % 4; the chunk's 8 segments
        //      of 32 candidates (TMEM columns 32 g ..) are split h, h + TS_EPG, ... -------------
        const int ew = warp - 2;                      // the segment this warp stages (if < 8)
        const int q = warp & 3, h = ew >> 2;
        const int p = q * 32 + lane;                  // pixel of the tile = TMEM lane
        const bool act = s_act[p] != 0;
        const int ci = s_ci[p], cj = s_cj[p];
        const int wxn = 2 * a.Sx + 1;
        float bq[TK];
        int bi[TK];
#pragma unroll
        for (int m = 0; m < TK; ++m) {
            bq[m] = INFINITY;
            bi[m] = -1;
        }
        bool edge = false;
        // masked pass: the pixels it ranks (those with candidates not valid in every frame)
        bool mine = act;
        float W2 = 0.0f;
        if (MASKED && act) {
            const size_t pix = (size_t)(y0 + p / TS_TX) * a.nx + (x0 + p % TS_TX);
            mine = a.edge[pix] != 0;
            const float Wv = a.W[pix];
            W2 = Wv * Wv;
        }
        // T~ and validity of segment `ew` of chunk j (+inf / clear bit: not valid in every
        // frame; in the masked pass: with no valid frame)
        auto fetch = [&](int j, float &t, bool &ok) {
            int row0, col0;
            chunk_origin(j, row0, col0);
            const int gy = row0 + ew / SPR, gx = col0 + (ew % SPR) * 32 + lane;
            t = INFINITY;
            ok = false;
            if (gy >= 0 && gy < a.Ry && gx >= 0 && gx < a.Rx) {
                const size_t c = (size_t)gy * a.Rx + gx;
                const int nv = __ldg(a.nvalid + c);
                ok = MASKED ? nv > 0 : nv == a.N;
                if (ok) t = __ldg(a.Tt + c);
            }
        };
        if (ew < 8) {
            float t;
            bool ok;
            fetch(0, t, ok);
            s_T[0][ew * 32 + lane] = t;
            const uint32_t vm = __ballot_sync(0xffffffffu, ok);
            if (lane == 0) s_vm[0][ew] = vm;
        }
        asm volatile("bar.sync 1, %0;" ::"n"(32 * TS_EPI_WARPS) : "memory");
        for (int j = 0; j < nchunks; ++j) {
            const int buf = j % NBUF, sbuf = j & 1;       // accumulator buffer, staged-terms buffer
            int row0, col0;
            chunk_origin(j, row0, col0);
            float tn = INFINITY;
            bool okn = false;
            if (j + 1 < nchunks && ew < 8) fetch(j + 1, tn, okn);
            // a wait that ran out stops every epilogue warp after the same barrier below
            const bool ok = __all_sync(0xffffffffu, tc::mbar_wait(&bar_tfull[buf], (j / NBUF) & 1, abortp, a.limit_ns));
            if (!ok) *abortp = 1;
            tc::tc_fence_after();
            if (ok) {
#pragma unroll 1
                for (int g = h; g < 8; g += TS_EPG) {
                    const int r = g / SPR, c0 = col0 + (g % SPR) * 32;
                    const int aa = row0 + r - ci;
                    // this pixel's window columns within the segment: [ilo, ihi]
                    const int ilo = max(0, cj - a.Sx - c0), ihi = min(31, cj + a.Sx - c0);
                    const uint32_t colmask =
                        ilo > ihi ? 0u : ((ihi == 31 ? 0xffffffffu : ((1u << (ihi + 1)) - 1u)) & ~((1u << ilo) - 1u));
                    const uint32_t inmask = (mine && aa >= -a.Sy && aa <= a.Sy) ? colmask : 0u;
                    if (__all_sync(0xffffffffu, inmask == 0u)) continue;
                    float v[32];
                    tc::tmem_ld32(tmem + buf * 256 + g * 32 + ((uint32_t)(q * 32) << 16), v);
                    const uint32_t vm = s_vm[sbuf][g];
                    const uint32_t use = inmask & vm;
                    const int rowbase = (aa + a.Sy) * wxn + (c0 - cj + a.Sx);
                    if (MASKED) {
                        float v2[32];
                        tc::tmem_ld32(tmem + 256 + g * 32 + ((uint32_t)(q * 32) << 16), v2);
                        scan_row_masked<TK>(v, v2, &s_T[sbuf][g * 32], use, rowbase, W2, bq, bi);
                    } else {
                        edge = edge || (inmask & ~vm) != 0u;
                        if (__all_sync(0xffffffffu, use == 0xffffffffu))
                            scan_row<TK, true>(v, &s_T[sbuf][g * 32], use, rowbase, bq, bi);
                        else
                            scan_row<TK, false>(v, &s_T[sbuf][g * 32], use, rowbase, bq, bi);
                    }
                }
            }
            tc::tc_fence_before();
            if (j + 1 < nchunks && ew < 8) {
                s_T[sbuf ^ 1][ew * 32 + lane] = tn;
                const uint32_t vm = __ballot_sync(0xffffffffu, okn);
                if (lane == 0) s_vm[sbuf ^ 1][ew] = vm;
            }
            asm volatile("bar.sync 1, %0;" ::"n"(32 * TS_EPI_WARPS) : "memory");
            if (lane == 0) tc::mbar_arrive(&bar_tempty[buf]);
            if (*abortp) break;
        }
        // merge the lists of each pixel (in warp order h = 1, 2, ...), write the result
        if (h > 0) {
#pragma unroll
            for (int m = 0; m < TK; ++m) {
                s_mq[h - 1][p][m] = bq[m];
                s_mi[h - 1][p][m] = bi[m];
            }
            s_medge[h - 1][p] = edge ? 1 : 0;
        }
        asm volatile("bar.sync 1, %0;" ::"n"(32 * TS_EPI_WARPS) : "memory");
        if (h == 0 && mine && !*abortp) {
#pragma unroll
            for (int w = 0; w < TS_EPG - 1; ++w)
#pragma unroll
                for (int m = 0; m < TK; ++m)
                    if (s_mq[w][p][m] < bq[TK - 1]) topk_insert<TK>(bq, bi, s_mq[w][p][m], s_mi[w][p][m]);
            const int x = x0 + (p % TS_TX), y = y0 + (p / TS_TX);
            const size_t pix = (size_t)y * a.nx + x;
#pragma unroll
            for (int m = 0; m < kTopK; ++m) a.cand[pix * kTopK + m] = m < TK ? bi[m] : -1;
            if (!MASKED) {
                bool e = edge;
#pragma unroll
                for (int w = 0; w < TS_EPG - 1; ++w) e = e || s_medge[w][p];
                a.edge[pix] = e ? 1 : 0;
                if (e) {
                    atomicAdd(&a.hdr->n_exact, 1);
                    s_tile_edge = 1;
                }
            }
        }
    }
    if (tid == 0 && *abortp) atomicOr(&a.hdr->status, PXST_DEV_TIMEOUT);
    tc::tc_fence_before();
    __syncthreads();
    // the tile holds pixels for the masked pass
    if (!MASKED && tid == 0 && s_tile_edge && !*abortp)
        a.tile_list[atomicAdd(&a.hdr->n_edge_tiles, 1)] = tile_y * a.tiles_x + tile_x;
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
}

}  // namespace

// ---- host launchers for the precision form --------------------------------------------------

cudaError_t launch_tprep(const pxst_dims &d, int form, int Npad, const float *frames, const float *W,
                         const uint8_t *mask, void *At, WsHeader *hdr, cudaStream_t stream) {
    const size_t P = (size_t)d.ny * d.nx;
    const int KB = form == PXST_FORM_TF32 ? 32 : 64;
    dim3 grid((unsigned)((P + TP_PIX - 1) / TP_PIX), (unsigned)(Npad / KB));
    if (form == PXST_FORM_TF32)
        k_tprep<float><<<grid, 256, 0, stream>>>(d.n_frames, d.ny, d.nx, frames, W, mask, static_cast<float *>(At),
                                                 hdr);
    else
        k_tprep<__nv_bfloat16><<<grid, 256, 0, stream>>>(d.n_frames, d.ny, d.nx, frames, W, mask,
                                                         static_cast<__nv_bfloat16 *>(At), hdr);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_gtable(const pxst_dims &d, int form, int Npad, const float *I_ref, const float *w,
                          const FrameShift *shifts, const WsHeader *hdr, void *G, void *V, float *Tt, int *nvalid,
                          float *Rm, cudaStream_t stream) {
    const size_t R = (size_t)d.ref_ny * d.ref_nx;
    k_rmask<<<(unsigned)std::min<size_t>((R + 255) / 256, (size_t)device_sms() * 16), 256, 0, stream>>>(R, I_ref, w, Rm); note_launch();
    const unsigned blocks = (unsigned)((R + 31) / 32);
    if (form == PXST_FORM_TF32)
        k_gtable<float><<<blocks, 256, 0, stream>>>(d.n_frames, Npad, d.ref_ny, d.ref_nx, Rm, shifts, hdr,
                                                     static_cast<float *>(G), static_cast<float *>(V), Tt, nvalid);
    else
        k_gtable<__nv_bfloat16><<<blocks, 256, 0, stream>>>(d.n_frames, Npad, d.ref_ny, d.ref_nx, Rm, shifts, hdr,
                                                             static_cast<__nv_bfloat16 *>(G),
                                                             static_cast<__nv_bfloat16 *>(V), Tt, nvalid);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_tsearch(const pxst_dims &d, const pxst_options &o, int Npad, const void *At, void *A2,
                           const void *G, const void *V, const uint8_t *mask, const float *W, const double *u,
                           const float *Tt, const int *nvalid, WsHeader *hdr, int *cand, uint8_t *edge,
                           int *tile_list, cudaStream_t stream) {
    const bool tf32 = o.form == PXST_FORM_TF32;
    const uint64_t es = tf32 ? 4 : 2;
    const uint32_t kb = tf32 ? 32 : 64;
    const CUtensorMapDataType dt = tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUtensorMap tA, tB, tA2, tV;
    const uint64_t nkb = (uint64_t)Npad / kb, row = (uint64_t)kb * es;     // 128-byte rows
    const uint64_t dA[4] = {kb, (uint64_t)d.nx, (uint64_t)d.ny, nkb};
    const uint64_t sA[3] = {row, row * d.nx, row * d.nx * d.ny};
    // tile shape: pixel tile rows and candidate chunk columns
    const int shape = (o.tile >= 0 && o.tile <= 2) ? o.tile : 0;
    const uint32_t pty = 8u >> shape, ccw = 32u << shape;
    const uint32_t bA[4] = {kb, 128 / pty, pty, 1};
    const uint64_t dB[4] = {kb, (uint64_t)d.ref_nx, (uint64_t)d.ref_ny, nkb};
    const uint64_t sB[3] = {row, row * d.ref_nx, row * d.ref_nx * d.ref_ny};
    const uint32_t bB[4] = {kb, ccw, 256 / ccw, 1};
    cudaError_t e;
    if ((e = tmap_encode(&tA, dt, 4, const_cast<void *>(At), dA, sA, bA)) != cudaSuccess) return e;
    if ((e = tmap_encode(&tB, dt, 4, const_cast<void *>(G), dB, sB, bB)) != cudaSuccess) return e;
    if ((e = tmap_encode(&tA2, dt, 4, const_cast<void *>(A2), dA, sA, bA)) != cudaSuccess) return e;
    if ((e = tmap_encode(&tV, dt, 4, const_cast<void *>(V), dB, sB, bB)) != cudaSuccess) return e;
    TSearchArgs a;
    a.N = d.n_frames; a.Npad = Npad; a.ny = d.ny; a.nx = d.nx; a.Ry = d.ref_ny; a.Rx = d.ref_nx;
    a.Sy = o.win_y; a.Sx = o.win_x; a.mask = mask; a.u = u; a.Tt = Tt; a.nvalid = nvalid; a.hdr = hdr;
    a.cand = cand; a.edge = edge; a.tile_list = tile_list; a.W = W;
    a.limit_ns = o.timeout_ns > 0 ? (unsigned long long)o.timeout_ns : 1000000000ull;
    const unsigned gx = (d.nx + 128 / pty - 1) / (128 / pty), gy = (d.ny + pty - 1) / pty;
    a.tiles_x = (int)gx;
    // list length: the candidates the rescore reads (4 unless more are asked for)
    const int rk = o.rescore_k ? o.rescore_k : (d.n_frames < 128 ? 8 : 4);
    // the ranking of every tile, then the masked ranking of the tiles it listed (a grid of
    // one CTA per tile, of which those beyond the list's length return at once)
    auto go = [&](auto plain, auto masked) {
        // A~ resident when it and three (else two) G~ stages fit the CTA's shared memory
        cudaFuncAttributes fa;
        cudaError_t r = cudaFuncGetAttributes(&fa, plain);
        if (r != cudaSuccess) return r;
        int dev = 0, optin = 0;
        if ((r = cudaGetDevice(&dev)) != cudaSuccess) return r;
        if ((r = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return r;
        int smem = TS_SMEM;
        a.ares = 0;
        for (int st = 3; st >= 2 && !a.ares; --st) {
            const long long need = 1024 + (long long)nkb * TS_A_BYTES + (long long)st * TS_B_BYTES;
            if (need + (long long)fa.sharedSizeBytes <= optin) {
                a.ares = st;
                smem = (int)need;
            }
        }
        r = cudaFuncSetAttribute(plain, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (r != cudaSuccess) return r;
        plain<<<dim3(gx, gy), TS_THREADS, smem, stream>>>(tA, tB, tA2, tV, a); note_launch();
        if ((r = cudaGetLastError()) != cudaSuccess) return r;
        if (tf32)
            k_tsquare<float><<<gx * gy, 256, 0, stream>>>((int)nkb, d.ny, d.nx, (int)pty, (int)gx, hdr, tile_list,
                                                          static_cast<const float *>(At), static_cast<float *>(A2));
        else
            k_tsquare<__nv_bfloat16><<<gx * gy, 256, 0, stream>>>(
                (int)nkb, d.ny, d.nx, (int)pty, (int)gx, hdr, tile_list, static_cast<const __nv_bfloat16 *>(At),
                static_cast<__nv_bfloat16 *>(A2));
        note_launch();
        if ((r = cudaGetLastError()) != cudaSuccess) return r;
        a.ares = 0;
        r = cudaFuncSetAttribute(masked, cudaFuncAttributeMaxDynamicSharedMemorySize, TSM_SMEM);
        if (r != cudaSuccess) return r;
        masked<<<gx * gy, TS_THREADS, TSM_SMEM, stream>>>(tA, tB, tA2, tV, a); note_launch();
        return cudaGetLastError();
    };
    auto by_shape = [&](auto tf32_tag, auto tk_tag) {
        constexpr bool T = decltype(tf32_tag)::value;
        constexpr int K = decltype(tk_tag)::value;
        switch (shape) {
            case 1: return go(k_tsearch<T, K, 4, 64, false>, k_tsearch<T, K, 4, 64, true>);
            case 2: return go(k_tsearch<T, K, 2, 128, false>, k_tsearch<T, K, 2, 128, true>);
            default: return go(k_tsearch<T, K, 8, 32, false>, k_tsearch<T, K, 8, 32, true>);
        }
    };
    using t_ = std::true_type;
    using f_ = std::false_type;
    if (tf32)
        e = rk <= 4 ? by_shape(t_{}, std::integral_constant<int, 4>{}) : by_shape(t_{}, std::integral_constant<int, 8>{});
    else
        e = rk <= 4 ? by_shape(f_{}, std::integral_constant<int, 4>{}) : by_shape(f_{}, std::integral_constant<int, 8>{});
    return e;
}

}  // namespace pxst

using namespace pxst;

extern "C" pxst_status pxst_tensor_check(int32_t form, int32_t K, const void *A, const void *B, float *D,
                                         int32_t *status, void *stream) {
    if ((form != PXST_FORM_BF16 && form != PXST_FORM_TF32) || K < 1 || !A || !B || !D || !status)
        return PXST_ERR_ARG;
    const bool tf32 = form == PXST_FORM_TF32;
    const size_t es = tf32 ? 4 : 2;
    if ((K * es) % 16 != 0 || (reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15))
        return PXST_ERR_ARG;
    const CUtensorMapDataType dt = tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const uint32_t kb = tf32 ? 32 : 64;
    CUtensorMap ta, tb;
    uint64_t dA[2] = {(uint64_t)K, 128}, dB[2] = {(uint64_t)K, 256};
    uint64_t st[1] = {(uint64_t)K * es};
    uint32_t boxA[2] = {kb, 128}, boxB[2] = {kb, 256};
    if (tmap_encode(&ta, dt, 2, const_cast<void *>(A), dA, st, boxA) != cudaSuccess ||
        tmap_encode(&tb, dt, 2, const_cast<void *>(B), dB, st, boxB) != cudaSuccess)
        return PXST_ERR_CUDA;
    const int smem = (128 + 256) * 128 + 1024;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (tf32) {
        e = cudaFuncSetAttribute(k_tc_check<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) {
            k_tc_check<true><<<1, 128, smem, s>>>(ta, tb, K, D, status);
            note_launch();
        }
    } else {
        e = cudaFuncSetAttribute(k_tc_check<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) {
            k_tc_check<false><<<1, 128, smem, s>>>(ta, tb, K, D, status);
            note_launch();
        }
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? PXST_OK : PXST_ERR_CUDA;
}
