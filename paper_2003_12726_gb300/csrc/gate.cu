// gate.cu -- a stream-ordered wait for an external producer (pxst_wait_flag).
//
// A reconstruction can be queued while its scan is still being acquired: the producer
// (a host thread writing pinned host memory, or a copy into device memory) raises a 32-bit
// counter, and the kernels queued after the wait run once it reaches the target. The wait
// is one thread polling with back-off, bounded by %globaltimer: when the limit passes it
// sets PXST_DEV_TIMEOUT in the workspace's status word and returns, so the stream never
// hangs and the GPU stays usable.
#include "pxst_common.cuh"

namespace pxst {
namespace {

__global__ void __launch_bounds__(32) k_wait_flag(const volatile int32_t *flag, int32_t target,
                                                  unsigned long long limit_ns, WsHeader *hdr) {
    if (threadIdx.x != 0) return;
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (unsigned sleep = 32;;) {
        if (*flag >= target) break;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > limit_ns) {
            atomicOr(&hdr->status, PXST_DEV_TIMEOUT);
            break;
        }
        __nanosleep(sleep);
        sleep = sleep < 8192 ? 2 * sleep : sleep;
    }
    __threadfence();
}

}  // namespace
}  // namespace pxst

using namespace pxst;

extern "C" pxst_status pxst_wait_flag(const int32_t *flag, int32_t target, int64_t timeout_ns, void *workspace,
                                      size_t ws_bytes, void *stream) {
    if (!flag || !workspace || timeout_ns < 0 || ws_bytes < sizeof(WsHeader)) return PXST_ERR_ARG;
    if (((uintptr_t)workspace & 255) != 0 || ((uintptr_t)flag & 3) != 0) return PXST_ERR_ARG;
    const unsigned long long limit = timeout_ns > 0 ? (unsigned long long)timeout_ns : 1000000000ull;
    k_wait_flag<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(flag, target, limit,
                                                                 static_cast<WsHeader *>(workspace));
    note_launch();
    return cudaGetLastError() == cudaSuccess ? PXST_OK : PXST_ERR_CUDA;
}
