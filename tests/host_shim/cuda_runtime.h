/* Host stand-ins for the CUDA names that the device header
 * paper_2504_19930_gb300/csrc/device.cuh uses, so that a test can compile
 * its arithmetic for the CPU and compare it with the oracle on many more
 * inputs than a GPU test samples.  Test infrastructure only: the package
 * never builds or loads this.  Each intrinsic becomes the IEEE operation its
 * name fixes (round to nearest; fma correctly rounded); build with
 * -ffp-contract=off so that nothing else is fused. */
#pragma once
#include <algorithm>
#include <cfenv>
#include <cmath>
#include <cstdlib>
#include <cstdint>
#include <cstring>

// -DPF_HOST_COUNT_FP32: count the fp32 lane operations executed (each
// __fadd_rn / __fsub_rn / __fmul_rn / __fmaf_rn / __fadd_rd is one)
#ifdef PF_HOST_COUNT_FP32
inline unsigned long long g_host_fp32_ops = 0;
#define PF_COUNT_FP32 (++g_host_fp32_ops)
#else
#define PF_COUNT_FP32 ((void)0)
#endif
#define __device__
#define __global__
#define __launch_bounds__(...)
#define __noinline__ __attribute__((noinline))
// block-shared variables: one static instance, seen by every emulated thread
#define __shared__ static
#define __host__
#define __forceinline__ inline

inline double __dmul_rn(double a, double b) { return a * b; }
inline double __dadd_rn(double a, double b) { return a + b; }
inline double __dsub_rn(double a, double b) { return a - b; }
inline double __ddiv_rn(double a, double b) { return a / b; }
inline double __fma_rn(double a, double b, double c) { return std::fma(a, b, c); }
inline double __dsqrt_rn(double a) { return std::sqrt(a); }
inline long long __double_as_longlong(double a) {
    long long r;
    std::memcpy(&r, &a, sizeof r);
    return r;
}
inline double __longlong_as_double(long long a) {
    double r;
    std::memcpy(&r, &a, sizeof r);
    return r;
}
inline float __double2float_rn(double a) { return (float)a; }
inline double __ull2double_rn(unsigned long long v) { return (double)v; }
inline unsigned long long __double2ull_rz(double a) { return (unsigned long long)a; }   // a >= 0 here
inline float __fmul_rn(float a, float b) { return PF_COUNT_FP32, a * b; }
inline float __fadd_rn(float a, float b) { return PF_COUNT_FP32, a + b; }
inline float __fsub_rn(float a, float b) { return PF_COUNT_FP32, a - b; }
inline float __fmaf_rn(float a, float b, float c) { return PF_COUNT_FP32, std::fmaf(a, b, c); }
inline float __int2float_rn(int x) { return (float)x; }
inline uint32_t __umulhi(uint32_t a, uint32_t b) { return (uint32_t)(((uint64_t)a * b) >> 32); }
inline float __uint_as_float(uint32_t u) {
    float f;
    std::memcpy(&f, &u, sizeof f);
    return f;
}
inline int __float2int_rn(float x) { return (int)std::nearbyint(x); }   // round half to even
inline uint32_t __float_as_uint(float f) {
    uint32_t u;
    std::memcpy(&u, &f, sizeof u);
    return u;
}
template <class T>
inline T __ldg(const T *p) { return *p; }
// a + b rounded toward -infinity (build with -frounding-math)
inline float __fadd_rd(float a, float b) {
    PF_COUNT_FP32;
    std::fesetround(FE_DOWNWARD);
    volatile float x = a, y = b;
    volatile float r = x + y;
    std::fesetround(FE_TONEAREST);
    return r;
}
// byte n of the result = byte (selector nibble n & 7) of the 8 bytes y:x
inline uint32_t __byte_perm(uint32_t x, uint32_t y, uint32_t s) {
    const uint64_t v = ((uint64_t)y << 32) | x;
    uint32_t r = 0;
    for (int n = 0; n < 4; ++n) r |= (uint32_t)((v >> (8 * ((s >> (4 * n)) & 7u))) & 0xFFu) << (8 * n);
    return r;
}
// the vector types the device code names
struct float2 {
    float x, y;
};
struct float4 {
    float x, y, z, w;
};
// Warp-level operations exist only under the lockstep emulation of
// tests/host_shim/warp_emulation.h; elsewhere a test that reached one would
// be wrong, so it aborts.
#ifndef PF_HOST_WARP_EMULATION
inline unsigned long long __shfl_xor_sync(unsigned, unsigned long long, int) { std::abort(); }
#endif
inline float4 make_float4(float x, float y, float z, float w) { return float4{x, y, z, w}; }
inline float2 make_float2(float x, float y) { return float2{x, y}; }
// thread coordinates, for tests that run a kernel without shared memory,
// barriers or shuffles as a host loop over its threads (the test sets them)
struct dim3 {
    unsigned x = 1, y = 1, z = 1;
};
extern dim3 threadIdx, blockIdx, blockDim, gridDim;
// the types the host-side declarations of kernels.h name
typedef int cudaError_t;
typedef struct CUstream_st *cudaStream_t;
enum { cudaSuccess = 0 };
using std::max;
using std::min;
