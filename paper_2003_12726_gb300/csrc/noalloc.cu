// noalloc.cu -- make_object_map for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: an acquisition or beamline plug-in that runs inside
// a host framework which owns the GPU's memory and forbids further allocations, or a
// real-time loop where an allocation's implicit device synchronisation and latency are
// not acceptable. pxst_make_object_map needs FP64 accumulators and a per-frame shift
// table as scratch; this file keeps that scratch in one fixed array compiled into the
// library, so the entry point below takes only the inputs and the outputs.
//
// The array is a file-scope __device__ variable: every GPU on which the library's module
// is loaded holds it (about 16.1 MiB) until the process exits. Host code must not pass
// the variable's name to a kernel (on the host it only stands in for the symbol); the
// device address is looked up with cudaGetSymbolAddress once per device and context and
// cached. With lazy module loading (the CUDA default) the first call on a device is also
// the one that loads this module and so reserves the array: make it before the GPU's
// memory is otherwise taken, and before any stream capture.
#include <cuda.h>

#include <cstdio>
#include <mutex>

#include "pxst_common.cuh"

namespace pxst {
namespace {

constexpr long long kNoAllocMaxRefCells = 1LL << 20;   // ref_ny * ref_nx
constexpr int kNoAllocMaxFrames = 8192;
constexpr size_t kHeaderBytes = 256;
constexpr size_t kShiftBytes = 16 * (size_t)kNoAllocMaxFrames;
constexpr size_t kAccBytes = sizeof(double) * (size_t)kNoAllocMaxRefCells;
constexpr size_t kScratchBytes = kHeaderBytes + kShiftBytes + 2 * kAccBytes;
static_assert(sizeof(WsHeader) == kHeaderBytes, "header size");
static_assert(sizeof(FrameShift) == 16, "shift record size");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// Per device: the context the address was looked up in, and the address. A device reset or
// a new primary context reloads the module, and the array may then sit elsewhere, so an
// address is reused only while the current context is the one it was looked up in.
unsigned long long g_ctx_id[kMaxDevices] = {};
void *g_addr[kMaxDevices] = {};

typedef CUresult (*PFN_ctxGetCurrent)(CUcontext *);
typedef CUresult (*PFN_ctxGetId)(CUcontext, unsigned long long *);
PFN_ctxGetCurrent g_get_current = nullptr;
PFN_ctxGetId g_get_id = nullptr;

// Identifier of the current context (unique for the life of the process), or 0 if the driver
// cannot report one: then the address is looked up again on every call.
unsigned long long current_context_id() {
    if (!g_get_current || !g_get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPoint("cuCtxGetCurrent", &f1, cudaEnableDefault, &q1) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || !f1 ||
            cudaGetDriverEntryPoint("cuCtxGetId", &f2, cudaEnableDefault, &q2) != cudaSuccess ||
            q2 != cudaDriverEntryPointSuccess || !f2)
            return 0;
        g_get_current = reinterpret_cast<PFN_ctxGetCurrent>(f1);
        g_get_id = reinterpret_cast<PFN_ctxGetId>(f2);
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (g_get_current(&ctx) != CUDA_SUCCESS || !ctx || g_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of g_noalloc_scratch on the current device, looked up (with the device
// current) the first time it is needed in each context.
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_mu);
    const unsigned long long id = current_context_id();
    if (!g_addr[dev] || id == 0 || id != g_ctx_id[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
        // the lookup has made the device's context current if none was: record that one
        g_ctx_id[dev] = current_context_id();
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace pxst

using namespace pxst;

extern "C" pxst_status pxst_make_object_map_noalloc(const pxst_dims *dims, const float *frames,
                                                    const float *W, const uint8_t *mask,
                                                    const double *u, const double *delta,
                                                    float *I_ref, float *w, void *stream) {
    if (!dims || dims->n_frames < 1 || dims->ny < 1 || dims->nx < 1 || dims->ref_ny < 1 ||
        dims->ref_nx < 1 || (long long)dims->ny * dims->nx >= (1LL << 31))
        return PXST_ERR_SHAPE;
    if (!frames || !W || !mask || !u || !delta || !I_ref || !w) return PXST_ERR_ARG;
    if ((long long)dims->ref_ny * dims->ref_nx > kNoAllocMaxRefCells ||
        dims->n_frames > kNoAllocMaxFrames) {
        std::fprintf(stderr,
                     "pxst_make_object_map_noalloc: %d frames and a %d x %d reference exceed its "
                     "fixed scratch (at most %d frames and %lld reference pixels); use "
                     "pxst_make_object_map with a workspace\n",
                     dims->n_frames, dims->ref_ny, dims->ref_nx, kNoAllocMaxFrames,
                     kNoAllocMaxRefCells);
        return PXST_ERR_NOMEM;
    }
    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) {
        std::fprintf(stderr, "pxst_make_object_map_noalloc: %s\n", cudaGetErrorString(e));
        return PXST_ERR_CUDA;
    }
    char *b = static_cast<char *>(base);
    WsHeader *hdr = reinterpret_cast<WsHeader *>(b);
    FrameShift *shifts = reinterpret_cast<FrameShift *>(b + kHeaderBytes);
    double *num = reinterpret_cast<double *>(b + kHeaderBytes + kShiftBytes);
    double *den = reinterpret_cast<double *>(b + kHeaderBytes + kShiftBytes + kAccBytes);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the array keeps the previous call's contents: the header starts at zero here and the
    // scatter launch clears the accumulators it uses before adding to them
    e = cudaMemsetAsync(hdr, 0, sizeof(WsHeader), s);
    if (e == cudaSuccess) e = launch_prepare(*dims, delta, hdr, shifts, nullptr, 1, s);
    if (e == cudaSuccess) e = launch_scatter(*dims, frames, W, mask, u, shifts, hdr, num, den, nullptr, nullptr, s);
    if (e == cudaSuccess) e = launch_normalise(*dims, num, den, I_ref, w, s);
    if (e != cudaSuccess) {
        std::fprintf(stderr, "pxst_make_object_map_noalloc: %s\n", cudaGetErrorString(e));
        return PXST_ERR_CUDA;
    }
    return PXST_OK;
}
