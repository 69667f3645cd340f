// tensor.cu -- tensor-core (tcgen05) precision forms of update_pixel_map on sm_103a.
//
// This file holds the diagnostic contraction used to check the tcgen05 machinery: one
// CTA computes D[128][256] = A[128][K] . B[256][K]^T with both operands K-major in global
// memory, loaded by TMA with 128-byte swizzle, the MMA accumulating in TMEM, and the
// accumulator read back with tcgen05.ld.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <mutex>

#include "pxst_common.cuh"
#include "tc_ptx.cuh"

namespace pxst {

// ---- host: tensor-map encoding through the driver entry point ----------------------------
namespace {
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_enc_mu;
}  // namespace

cudaError_t tmap_encode(CUtensorMap *map, CUtensorMapDataType dt, uint32_t rank, void *base,
                        const uint64_t *dims, const uint64_t *strides_bytes, const uint32_t *box) {
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
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
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
    if (tid == 0) {
        abort_flag = 0;
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
        if (tid == 0 && !abort_flag) {
            const uint32_t ph = kb & 1;
            tc::mbar_expect_tx(&bar_full, (128 + 256) * 128);
            tc::tma_load_2d(As, &ta, &bar_full, kb * KB, 0);
            tc::tma_load_2d(Bs, &tb, &bar_full, kb * KB, 0);
            if (!tc::mbar_wait(&bar_full, ph, &abort_flag)) {
                abort_flag = 1;
            } else {
                tc::tc_fence_after();
                const uint32_t a0 = tc::smem_u32(As), b0 = tc::smem_u32(Bs);
#pragma unroll
                for (int k = 0; k < KB / KSTEP; ++k)
                    tc::mma<TF32>(tmem, tc::smem_desc_sw128(a0 + k * 32), tc::smem_desc_sw128(b0 + k * 32),
                                  IDESC, (kb > 0 || k > 0) ? 1u : 0u);
                tc::mma_commit(&bar_mma);
                if (!tc::mbar_wait(&bar_mma, ph, &abort_flag)) abort_flag = 1;
            }
        }
        __syncthreads();
        if (abort_flag) break;
    }
    tc::tc_fence_after();
    if (!abort_flag) {
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

}  // namespace
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
        if (e == cudaSuccess) k_tc_check<true><<<1, 128, smem, s>>>(ta, tb, K, D, status);
    } else {
        e = cudaFuncSetAttribute(k_tc_check<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) k_tc_check<false><<<1, 128, smem, s>>>(ta, tb, K, D, status);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? PXST_OK : PXST_ERR_CUDA;
}
