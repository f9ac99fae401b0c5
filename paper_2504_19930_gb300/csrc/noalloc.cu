// noalloc.cu -- pf_measure_matrices_noalloc: the measurement of caller-given
// matrices without any device allocation.
//
// pf_measure_matrices grows a per-context device buffer on demand (cudaMalloc)
// for the matrices it uploads and the moments the kernel accumulates.  Some
// callers cannot allocate once they are running: an acquisition or control
// loop that must not stall on the allocator or fail for lack of memory midway,
// a process held to a fixed device-memory budget after start-up, or code that
// runs where allocation calls are not permitted.  This variant keeps that
// scratch in a file-scope __device__ array of fixed size, which every GPU that
// loads the library holds until the process exits.
#include <cmath>
#include <mutex>

#include "../../include/pfreg.h"
#include "kernels.h"

namespace pfreg {
// Measurement set-up of a context (defined with the context in api.cu).
int ctx_measure_setup(pf_ctx *c, MeasureArgs *ma, bool *img, bool *mask, cudaStream_t *stream, int *device);
int set_error(int code, const char *msg);
}  // namespace pfreg

using namespace pfreg;

namespace {

constexpr int kNoAllocMaxMatrices = PF_NOALLOC_MAX_MATRICES;

// The shared scratch: matrices [4096][12] fp32 (192 KiB), then the moment
// accumulators [4096][12] u64 (384 KiB).
struct NoAllocScratch {
    float mats[kNoAllocMaxMatrices * 12];
    unsigned long long mom[kNoAllocMaxMatrices * kMomStride];
};
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// In host code g_noalloc_scratch names a host-side stand-in, not device
// memory.  Its device address differs per device; it is looked up once per
// device, with that device current (the caller has checked that the
// context's device is the current one), and cached here.
constexpr int kMaxDevices = 256;
std::mutex g_mu;
NoAllocScratch *g_scratch_addr[kMaxDevices] = {};

int scratch_for_device(int dev, NoAllocScratch **out) {
    if (dev < 0 || dev >= kMaxDevices) return set_error(PF_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return set_error(PF_ECUDA, "cudaGetSymbolAddress of the no-alloc scratch failed");
        g_scratch_addr[dev] = static_cast<NoAllocScratch *>(p);
    }
    *out = g_scratch_addr[dev];
    return PF_OK;
}

// b + 0 turns a -0 offset into +0 (the measurement relies on no -0 offsets),
// as pf_measure_matrices does on the host.
__global__ void k_canonical_offsets(float *mats, int M) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
#pragma unroll
    for (int r = 0; r < 3; ++r) mats[12 * (size_t)i + 4 * r + 3] = __fadd_rn(mats[12 * (size_t)i + 4 * r + 3], 0.0f);
}

}  // namespace

extern "C" int pf_measure_matrices_noalloc(pf_ctx *c, const float *mats, int32_t M, const float a[3],
                                           uint64_t *moments_out) {
    if (!c || !mats || !a || !moments_out) return set_error(PF_EINVAL, "NULL argument");
    if (M < 1 || M > kNoAllocMaxMatrices)
        return set_error(PF_EINVAL, "M outside [1, PF_NOALLOC_MAX_MATRICES = 4096] (no-alloc scratch capacity)");
    for (size_t i = 0; i < 12 * (size_t)M; ++i)
        if (!std::isfinite(mats[i])) return set_error(PF_EINVAL, "matrix entry is not finite");
    if (!std::isfinite(a[0]) || !std::isfinite(a[1]) || !std::isfinite(a[2]))
        return set_error(PF_EINVAL, "a is not finite");
    MeasureArgs ma;
    bool img = false, mask = false;
    cudaStream_t s = nullptr;
    int ctx_dev = -1;
    int rc = ctx_measure_setup(c, &ma, &img, &mask, &s, &ctx_dev);
    if (rc) return rc;
    // The scratch is per device and the context's stream belongs to its
    // device: the symbol address is only valid with that device current.
    int cur = -1;
    const cudaError_t ed = cudaGetDevice(&cur);
    if (ed != cudaSuccess) return set_error(PF_ECUDA, cudaGetErrorString(ed));
    if (cur != ctx_dev)
        return set_error(PF_EINVAL, "the current device is not the context's device: make the device the context "
                                    "was created on current (cudaSetDevice) before calling");
    NoAllocScratch *scr = nullptr;
    if ((rc = scratch_for_device(ctx_dev, &scr))) return rc;
    cudaError_t e = cudaMemcpyAsync(scr->mats, mats, sizeof(float) * 12 * (size_t)M, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(scr->mom, 0, sizeof(unsigned long long) * kMomStride * (size_t)M, s);
    if (e == cudaSuccess) {
        k_canonical_offsets<<<(M + 127) / 128, 128, 0, s>>>(scr->mats, M);
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        ma.mats = scr->mats;
        ma.mom = scr->mom;
        ma.P = M;
        for (int d = 0; d < 3; ++d) ma.g.a[d] = a[d];
        e = launch_measure(ma, img, mask, s);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(moments_out, scr->mom, sizeof(uint64_t) * kMomStride * (size_t)M, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_error(PF_ECUDA, cudaGetErrorString(e));
    return PF_OK;
}
