// warp.cu -- the sequence warp (Abstract; Sec. 3.3: the transform estimated
// on the end-diastolic frame is applied to every frame of the cycle).
//
// out(p) = rint(trilinear(frame, q(p))) (round half to even, 0..255) or the
// nearest voxel, 0 where q(p) is outside the source grid.  A persistent grid
// (a few CTAs per SM) walks frame-major over groups of 4 consecutive target
// voxels of a row; each CTA first builds the pose's matrix in shared memory
// (six lanes take the fp64 sin/cos in parallel), so a launch covers up to 64
// frames with one pose passed by value.
#include "kernels.h"

namespace pfreg {

namespace {

constexpr int kWarpThreads = 256;
constexpr int kVox = 4;   // target voxels per thread

struct WarpArgs {
    WarpFrames f;
    float pose[6];
    Geometry g;
    int interp;
    int n_frames;
    int row_groups;   // ceil(X / kVox)
};

__device__ __forceinline__ uint8_t warp_voxel(const uint8_t *__restrict__ S, const WarpArgs &a,
                                              const float *M, int x, float K0, float K1, float K2) {
    const int SX = a.g.sd[0], SY = a.g.sd[1], SZ = a.g.sd[2];
    const size_t SXY = (size_t)SX * SY;
    const float dx = __fsub_rn((float)x, a.g.a[0]);
    const float qx = __fadd_rn(__fmul_rn(M[0], dx), K0);
    const float qy = __fadd_rn(__fmul_rn(M[4], dx), K1);
    const float qz = __fadd_rn(__fmul_rn(M[8], dx), K2);
    if (a.interp == 0) {
        const float hx = __fadd_rn(qx, 0.5f), hy = __fadd_rn(qy, 0.5f), hz = __fadd_rn(qz, 0.5f);
        if (!(hx >= 0.0f && hx < (float)SX && hy >= 0.0f && hy < (float)SY && hz >= 0.0f && hz < (float)SZ))
            return 0;
        return __ldg(S + (size_t)(int)floorf(hx) + (size_t)SX * (size_t)(int)floorf(hy) +
                     SXY * (size_t)(int)floorf(hz));
    }
    if (!(qx >= 0.0f && qx <= (float)(SX - 1) && qy >= 0.0f && qy <= (float)(SY - 1) && qz >= 0.0f &&
          qz <= (float)(SZ - 1)))
        return 0;
    const float fx0 = fminf(floorf(qx), (float)(SX - 2));
    const float fy0 = fminf(floorf(qy), (float)(SY - 2));
    const float fz0 = fminf(floorf(qz), (float)(SZ - 2));
    const float fx = __fsub_rn(qx, fx0), fy = __fsub_rn(qy, fy0), fz = __fsub_rn(qz, fz0);
    const uint8_t *p = S + (size_t)(int)fx0 + (size_t)SX * (size_t)(int)fy0 + SXY * (size_t)(int)fz0;
    const float v000 = __ldg(p), v100 = __ldg(p + 1);
    const float v010 = __ldg(p + SX), v110 = __ldg(p + SX + 1);
    const float v001 = __ldg(p + SXY), v101 = __ldg(p + SXY + 1);
    const float v011 = __ldg(p + SXY + SX), v111 = __ldg(p + SXY + SX + 1);
    const float c00 = lerp_rn(v000, v100, fx), c10 = lerp_rn(v010, v110, fx);
    const float c01 = lerp_rn(v001, v101, fx), c11 = lerp_rn(v011, v111, fx);
    const float c0 = lerp_rn(c00, c10, fy), c1 = lerp_rn(c01, c11, fy);
    const int v = __float2int_rn(lerp_rn(c0, c1, fz));
    return (uint8_t)(v < 0 ? 0 : (v > 255 ? 255 : v));
}

__global__ void __launch_bounds__(kWarpThreads) k_warp(const WarpArgs a) {
    __shared__ double sc[6];
    __shared__ float Ms[12];
    if (threadIdx.x < 6) {
        const double ang = (double)a.pose[threadIdx.x % 3];
        sc[threadIdx.x] = threadIdx.x < 3 ? taylor_sin(ang) : taylor_cos(ang);
    }
    __syncthreads();
    if (threadIdx.x == 0) matrix_from_sincos(a.pose, sc[0], sc[3], sc[1], sc[4], sc[2], sc[5], a.g, Ms);
    __syncthreads();
    float M[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) M[j] = Ms[j];

    const int TX = a.g.td[0], TY = a.g.td[1], TZ = a.g.td[2];
    const long long per_frame = (long long)a.row_groups * TY * TZ;
    const long long total = per_frame * a.n_frames;
    for (long long gi = (long long)blockIdx.x * kWarpThreads + threadIdx.x; gi < total;
         gi += (long long)gridDim.x * kWarpThreads) {
        const int f = (int)(gi / per_frame);
        const long long li = gi - (long long)f * per_frame;
        const int r = (int)(li / a.row_groups);
        const int x0 = (int)(li - (long long)r * a.row_groups) * kVox;
        const int y = r % TY, z = r / TY;
        const float dy = __fsub_rn((float)y, a.g.a[1]), dz = __fsub_rn((float)z, a.g.a[2]);
        const float K0 = row_K(M[1], M[2], M[3], dy, dz);
        const float K1 = row_K(M[5], M[6], M[7], dy, dz);
        const float K2 = row_K(M[9], M[10], M[11], dy, dz);
        const uint8_t *S = a.f.in[f];
        uint8_t *O = a.f.out[f] + (size_t)r * TX;
        uint8_t v[kVox];
#pragma unroll
        for (int j = 0; j < kVox; ++j) v[j] = (x0 + j < TX) ? warp_voxel(S, a, M, x0 + j, K0, K1, K2) : 0;
        if (x0 + kVox <= TX && ((reinterpret_cast<uintptr_t>(O + x0) & 3) == 0)) {
            *reinterpret_cast<uint32_t *>(O + x0) =
                (uint32_t)v[0] | ((uint32_t)v[1] << 8) | ((uint32_t)v[2] << 16) | ((uint32_t)v[3] << 24);
        } else {
#pragma unroll
            for (int j = 0; j < kVox; ++j)
                if (x0 + j < TX) O[x0 + j] = v[j];
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
    a.row_groups = (g.td[0] + kVox - 1) / kVox;
    const long long total = (long long)a.row_groups * g.td[1] * g.td[2] * n;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_warp, kWarpThreads, 0);
    if (e != cudaSuccess) return e;
    long long grid = (long long)sms * (per_sm > 0 ? per_sm : 1);
    const long long need = (total + kWarpThreads - 1) / kWarpThreads;
    if (grid > need) grid = need;
    k_warp<<<(unsigned)grid, kWarpThreads, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pfreg
