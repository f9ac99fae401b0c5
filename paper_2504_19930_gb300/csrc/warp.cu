// warp.cu -- the sequence warp (Abstract; Sec. 3.3: the transform estimated
// on the end-diastolic frame is applied to every frame of the cycle).
//
// out(p) = rint(trilinear(frame, q(p))) (round half to even, 0..255) or the
// nearest voxel, 0 where q(p) is outside the source grid.  A persistent grid
// (a few CTAs per SM) walks the target rows, one row per warp at a time:
// lanes take x = lane + 32 j; where a voxel samples is the same in every
// frame, so it is computed once and every frame is sampled there (voxels
// outside the row's conservative inside range are written 0 without
// sampling).  Each CTA
// first builds the pose's matrix in shared memory (six lanes take the fp64
// sin/cos in parallel), so a launch covers up to 64 frames with one pose
// passed by value.
//
// Debug build (-DPF_DEBUG=1): every gather index is checked against the
// frame before the load; an index outside sets a device flag, records the
// first bad index and skips the load (the voxel reads 0) -- nothing traps.
#include <type_traits>

#include "kernels.h"

#ifndef PF_DEBUG
#define PF_DEBUG 0
#endif

namespace pfreg {

namespace {

constexpr int kWarpThreads = 256;

#if PF_DEBUG
__device__ unsigned long long g_wdbg_hits;
__device__ long long g_wdbg_first;
// true when idx < limit; otherwise counts the hit, keeps the first bad index
__device__ __forceinline__ bool wdbg_ok(unsigned long long idx, unsigned long long limit) {
    if (idx < limit) return true;
    if (atomicAdd(&g_wdbg_hits, 1ull) == 0ull) g_wdbg_first = (long long)idx;
    return false;
}
#endif

struct WarpArgs {
    WarpFrames f;
    float pose[6];
    Geometry g;
    int interp;
    int n_frames;
};

// integer value of a float holding a non-negative integer below 2^23
__device__ __forceinline__ uint32_t uint_of(float v) {
    return __float_as_uint(__fadd_rn(v, 8388608.0f)) - 0x4B000000u;
}

// Where one output voxel samples the source: the same for every frame (the
// frames share the pose), so it is computed once and reused.  WIDE: the
// frame has 2^31 voxels or more (64-bit offsets).  valid = false: the voxel
// is outside the source grid (or, in the debug build, its gather index
// failed the bounds check) and is written 0.
template <bool WIDE>
struct Sample {
    typename std::conditional<WIDE, size_t, uint32_t>::type i;   // nearest voxel, or the base corner
    float fx, fy, fz;                                            // trilinear fractions
    bool valid;
};

template <bool WIDE>
__device__ __forceinline__ Sample<WIDE> sample_at(const WarpArgs &a, const float *M, int x, float K0, float K1,
                                                  float K2) {
    using idx_t = typename std::conditional<WIDE, size_t, uint32_t>::type;
    const int SX = a.g.sd[0], SY = a.g.sd[1], SZ = a.g.sd[2];
    const idx_t sx = (idx_t)SX, sxy = (idx_t)SX * (idx_t)SY;
    const float dx = __fsub_rn((float)x, a.g.a[0]);
    const float qx = __fadd_rn(__fmul_rn(M[0], dx), K0);
    const float qy = __fadd_rn(__fmul_rn(M[4], dx), K1);
    const float qz = __fadd_rn(__fmul_rn(M[8], dx), K2);
    Sample<WIDE> s;
    s.i = 0;
    s.fx = s.fy = s.fz = 0.0f;
    if (a.interp == 0) {
        const float hx = __fadd_rn(qx, 0.5f), hy = __fadd_rn(qy, 0.5f), hz = __fadd_rn(qz, 0.5f);
        s.valid = hx >= 0.0f && hx < (float)SX && hy >= 0.0f && hy < (float)SY && hz >= 0.0f && hz < (float)SZ;
        if (s.valid)
            s.i = (idx_t)uint_of(floorf(hx)) + sx * (idx_t)uint_of(floorf(hy)) + sxy * (idx_t)uint_of(floorf(hz));
#if PF_DEBUG
        if (s.valid && !wdbg_ok((unsigned long long)s.i, (unsigned long long)sxy * (unsigned long long)SZ))
            s.valid = false;
#endif
        return s;
    }
    s.valid = qx >= 0.0f && qx <= (float)(SX - 1) && qy >= 0.0f && qy <= (float)(SY - 1) && qz >= 0.0f &&
              qz <= (float)(SZ - 1);
    if (!s.valid) return s;
    const float fx0 = fminf(floorf(qx), (float)(SX - 2));
    const float fy0 = fminf(floorf(qy), (float)(SY - 2));
    const float fz0 = fminf(floorf(qz), (float)(SZ - 2));
    s.fx = __fsub_rn(qx, fx0);
    s.fy = __fsub_rn(qy, fy0);
    s.fz = __fsub_rn(qz, fz0);
    s.i = (idx_t)uint_of(fx0) + sx * (idx_t)uint_of(fy0) + sxy * (idx_t)uint_of(fz0);
#if PF_DEBUG
    // the farthest corner read is i + sxy + sx + 1
    if (!wdbg_ok((unsigned long long)s.i + sxy + sx + 1, (unsigned long long)sxy * (unsigned long long)SZ))
        s.valid = false;
#endif
    return s;
}

// The sample of one frame: the nearest voxel, or the trilinear interpolation
// of the 8 corners rounded half to even and clamped to 0..255.
template <bool WIDE>
__device__ __forceinline__ uint8_t sample_frame(const uint8_t *__restrict__ S, const Sample<WIDE> &s, int interp,
                                                size_t sx, size_t sxy) {
    if (interp == 0) return __ldg(S + s.i);
    const uint8_t *p = S + s.i;
    const float v000 = __ldg(p), v100 = __ldg(p + 1);
    const float v010 = __ldg(p + sx), v110 = __ldg(p + sx + 1);
    const float v001 = __ldg(p + sxy), v101 = __ldg(p + sxy + 1);
    const float v011 = __ldg(p + sxy + sx), v111 = __ldg(p + sxy + sx + 1);
    const float c00 = lerp_rn(v000, v100, s.fx), c10 = lerp_rn(v010, v110, s.fx);
    const float c01 = lerp_rn(v001, v101, s.fx), c11 = lerp_rn(v011, v111, s.fx);
    const float c0 = lerp_rn(c00, c10, s.fy), c1 = lerp_rn(c01, c11, s.fy);
    const int v = __float2int_rn(lerp_rn(c0, c1, s.fz));
    return (uint8_t)(v < 0 ? 0 : (v > 255 ? 255 : v));
}

// One target row per warp at a time (a persistent grid walks the rows);
// lane takes x = lane + 32 j, computes where that voxel samples once and
// then samples every frame there, four frames at a time so that their
// gathers are in flight together.  Voxels outside the row's conservative
// inside range, or outside the source, are written 0 in every frame.
template <bool WIDE>
__global__ void __launch_bounds__(kWarpThreads) k_warp(const WarpArgs a) {
    __shared__ double sc[6];
    __shared__ float Ms[12];
    if (threadIdx.x < 6) {
        sc[threadIdx.x] = taylor_sincos(a.pose[threadIdx.x % 3], threadIdx.x >= 3);
    }
    __syncthreads();
    if (threadIdx.x == 0) matrix_from_sincos(a.pose, sc[0], sc[3], sc[1], sc[4], sc[2], sc[5], a.g, Ms);
    __syncthreads();
    float M[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) M[j] = Ms[j];
    const float r0[3] = {M[0], M[4], M[8]};
    const float SXf = (float)a.g.sd[0], SYf = (float)a.g.sd[1], SZf = (float)a.g.sd[2];
    float lo[3], hi[3];
    lo[0] = lo[1] = lo[2] = a.interp ? 0.0f : -0.5f;
    hi[0] = a.interp ? SXf - 1.0f : SXf - 0.5f;
    hi[1] = a.interp ? SYf - 1.0f : SYf - 0.5f;
    hi[2] = a.interp ? SZf - 1.0f : SZf - 0.5f;
    const int TX = a.g.td[0], TY = a.g.td[1];
    const int lane = threadIdx.x & 31;
    const size_t sx = (size_t)a.g.sd[0], sxy = (size_t)a.g.sd[0] * (size_t)a.g.sd[1];
    const int nf = a.n_frames;
    const long long rows = (long long)TY * a.g.td[2];
    const long long nwarps = (long long)gridDim.x * (kWarpThreads / 32);
    for (long long r = (long long)blockIdx.x * (kWarpThreads / 32) + (threadIdx.x >> 5); r < rows; r += nwarps) {
        const int y = (int)(r % TY), z = (int)(r / TY);
        const float dy = __fsub_rn((float)y, a.g.a[1]), dz = __fsub_rn((float)z, a.g.a[2]);
        const float K[3] = {row_K(M[1], M[2], M[3], dy, dz), row_K(M[5], M[6], M[7], dy, dz),
                            row_K(M[9], M[10], M[11], dy, dz)};
        int xb, xe;
        row_interval(r0, K, a.g.a[0], lo, hi, TX, xb, xe);
        const size_t row0 = (size_t)r * TX;
        for (int x = lane; x < TX; x += 32) {
            Sample<WIDE> s;
            s.valid = false;
            if (x >= xb && x < xe) s = sample_at<WIDE>(a, M, x, K[0], K[1], K[2]);
            const size_t o = row0 + (size_t)x;
            if (!s.valid) {
                for (int f = 0; f < nf; ++f) a.f.out[f][o] = 0;
                continue;
            }
            int f = 0;
            for (; f + 4 <= nf; f += 4) {
                const uint8_t v0 = sample_frame<WIDE>(a.f.in[f], s, a.interp, sx, sxy);
                const uint8_t v1 = sample_frame<WIDE>(a.f.in[f + 1], s, a.interp, sx, sxy);
                const uint8_t v2 = sample_frame<WIDE>(a.f.in[f + 2], s, a.interp, sx, sxy);
                const uint8_t v3 = sample_frame<WIDE>(a.f.in[f + 3], s, a.interp, sx, sxy);
                a.f.out[f][o] = v0;
                a.f.out[f + 1][o] = v1;
                a.f.out[f + 2][o] = v2;
                a.f.out[f + 3][o] = v3;
            }
            for (; f < nf; ++f) a.f.out[f][o] = sample_frame<WIDE>(a.f.in[f], s, a.interp, sx, sxy);
        }
    }
}

}  // namespace

cudaError_t launch_warp(const WarpFrames &f, int n, const float pose[6], Geometry g, int interp,
                        cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    WarpArgs a;
    a.f = f;
    for (int j = 0; j < 6; ++j) a.pose[j] = pose[j];
    a.g = g;
    a.interp = interp;
    a.n_frames = n;
    const bool wide = (long long)g.sd[0] * g.sd[1] * g.sd[2] >= (1ll << 31);
    const long long rows = (long long)g.td[1] * g.td[2];
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wide ? k_warp<true> : k_warp<false>,
                                                                  kWarpThreads, 0);
    if (e != cudaSuccess) return e;
    long long grid = (long long)sms * (per_sm > 0 ? per_sm : 1);
    const long long need = (rows + kWarpThreads / 32 - 1) / (kWarpThreads / 32);
    if (grid > need) grid = need;
    if (wide)
        k_warp<true><<<(unsigned)grid, kWarpThreads, 0, s>>>(a);
    else
        k_warp<false><<<(unsigned)grid, kWarpThreads, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

// Bounds-check counters of the debug build (all zero otherwise).
cudaError_t warp_debug_bounds(bool clear, unsigned long long *hits, long long *first, bool *on) {
#if PF_DEBUG
    *on = true;
    cudaError_t e = cudaMemcpyFromSymbol(hits, g_wdbg_hits, sizeof *hits);
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(first, g_wdbg_first, sizeof *first);
    if (e == cudaSuccess && clear) {
        const unsigned long long z = 0;
        const long long zf = 0;
        e = cudaMemcpyToSymbol(g_wdbg_hits, &z, sizeof z);
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_wdbg_first, &zf, sizeof zf);
    }
    return e;
#else
    *on = false;
    *hits = 0;
    *first = 0;
    (void)clear;
    return cudaSuccess;
#endif
}

}  // namespace pfreg
