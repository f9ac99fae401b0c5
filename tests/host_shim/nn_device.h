/* Device intrinsics and types the proposal network's CUDA-core kernels use,
 * for compiling them on the host: bf16 stored as the upper half of the fp32
 * pattern rounded to nearest with ties to even (no non-finite values reach
 * these kernels), the fast exponential, logarithm and cosine as the functions
 * they name, a float atomicAdd (one host thread runs every context of the
 * emulation) and the device's integer min / max.  Include after
 * tests/host_shim/warp_emulation.h.  Test infrastructure only. */
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

struct __nv_bfloat16 {
    uint16_t x;
};
inline __nv_bfloat16 __float2bfloat16_rn(float v) {
    uint32_t u;
    std::memcpy(&u, &v, sizeof u);
    return __nv_bfloat16{(uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16)};
}
inline float __expf(float x) { return std::exp(x); }
inline float __logf(float x) { return std::log(x); }
inline float __cosf(float x) { return std::cos(x); }
inline float atomicAdd(float *p, float v) {
    const float old = *p;
    *p = old + v;
    return old;
}
using std::max;
using std::min;
