// probe.cu -- a read-bandwidth probe (no counterpart in the paper).
//
// The measurement kernel gathers from an L2-resident source, so its memory
// roof is the L2 -> SM read bandwidth, which no vendor figure on this machine
// states.  This kernel streams a device buffer with 16-byte loads that bypass
// L1 (ld.global.cg), so every byte it reads comes from L2 (or, for a buffer
// larger than L2, from HBM); the caller times it with CUDA events.
#include <cstdint>

#include "../../include/pfreg.h"
#include "kernels.h"

namespace pfreg {
int set_error(int code, const char *msg);
}  // namespace pfreg

using namespace pfreg;

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeUnroll = 8;

__device__ __forceinline__ uint4 load_cg(const uint4 *p) {
    uint4 v;
    asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// Each thread reads elements t, t + T, t + 2T, ... (T = all threads), eight
// independent loads in flight, `reps` times over the buffer.  The XOR of
// everything read is folded into *sink only for one impossible-looking value,
// which keeps the loads without adding traffic.
__global__ void __launch_bounds__(kProbeThreads) k_read_probe(const uint4 *__restrict__ buf, size_t n16, int reps,
                                                             unsigned long long *sink) {
    const size_t T = (size_t)gridDim.x * blockDim.x;
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (int r = 0; r < reps; ++r) {
        for (size_t i = t0; i < n16; i += T * kProbeUnroll) {
            uint4 v[kProbeUnroll];
#pragma unroll
            for (int u = 0; u < kProbeUnroll; ++u) {
                const size_t j = i + (size_t)u * T;
                v[u] = j < n16 ? load_cg(buf + j) : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int u = 0; u < kProbeUnroll; ++u) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
        }
    }
    if (acc == 0x9E3779B9u) atomicAdd(sink, 1ull);
}

}  // namespace

extern "C" int pf_probe_read(const void *buf, int64_t bytes, int32_t reps, uint64_t *sink, void *stream) {
    if (!buf || !sink) return set_error(PF_EINVAL, "NULL argument");
    if (bytes < 16 || bytes % 16 != 0) return set_error(PF_EINVAL, "bytes must be a positive multiple of 16");
    if (reinterpret_cast<uintptr_t>(buf) % 16 != 0) return set_error(PF_EINVAL, "buf must be 16-byte aligned");
    if (reps < 1 || reps > 100000) return set_error(PF_EINVAL, "reps outside [1, 100000]");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return set_error(PF_ECUDA, "device query failed");
    const size_t n16 = (size_t)bytes / 16;
    // 8 CTAs of 256 threads per SM: 64 warps, each with 8 loads in flight
    size_t grid = (size_t)sms * 8;
    const size_t need = (n16 + kProbeThreads - 1) / kProbeThreads;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    k_read_probe<<<(unsigned)grid, kProbeThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const uint4 *>(buf), n16, reps, reinterpret_cast<unsigned long long *>(sink));
    count_launches(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(PF_ECUDA, cudaGetErrorString(e));
    return PF_OK;
}
