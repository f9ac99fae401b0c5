// measure.cu -- the measurement step (Fig. 1 caption: the similarity of the
// source warped by each particle's transform is the particle's measurement).
//
// One work item = (particle p, block of target rows); a persistent grid
// strides over the items, consecutive items sharing a particle.  Each warp
// sweeps one target row at a time, lane = x offset, so a warp's gathers follow
// the rotated row through the L2-resident source.  Per row the x-range that
// can map inside the source is computed first (row_interval) and only that
// range is visited; every visited voxel still takes the exact fp32 inside
// test, so the result equals the full sweep.
//
// Image mode (trilinear, Sec. 3.3): the source is read in a quad-packed copy
// Q[x,y,z] = S[x,y,z] | S[x+1,y,z]<<8 | S[x,y+1,z]<<16 | S[x+1,y+1,z]<<24, so
// the eight corners are two 32-bit gathers (planes z and z+1).  Bytes become
// floats with a byte permute into 2^23 + b (exact differences, one subtract
// for the base).  The sample s is rounded to s_q = rint(2^15 s) exactly as
// the bits of fp32 (s + 256); the moments n, S1, S2 (128-bit), ST, T1, T2 are
// exact integers, so the atomics give order-free, deterministic bits.
// Mask mode (nearest neighbour): counts n, A, B, C; the source mask is one
// bit per voxel, in shared memory when it fits.
#include "kernels.h"

namespace pfreg {

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr float kTwo23 = 8388608.0f;
constexpr uint32_t kTwo23Bits = 0x4B000000u;   // bits of 2^23
constexpr uint32_t k256Bits = 0x43800000u;     // bits of 256.0f

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// 2^23 + byte k of w, as a float (exact).
__device__ __forceinline__ float byte_biased(uint32_t w, uint32_t k) {
    return __uint_as_float(__byte_perm(w, kTwo23Bits, 0x7540u | k));
}

// lerp with biased end points A = 2^23 + a, B = 2^23 + b: a + f*(b - a).
__device__ __forceinline__ float lerp_biased(float A, float B, float f) {
    return __fadd_rn(__fsub_rn(A, kTwo23), __fmul_rn(f, __fsub_rn(B, A)));
}

// Integer value of an integral float v in [0, 2^22).
__device__ __forceinline__ uint32_t int_of(float v) {
    return __float_as_uint(__fadd_rn(v, kTwo23)) - kTwo23Bits;
}

struct ImgAcc {
    uint32_t n = 0, S1 = 0, T1 = 0, T2 = 0;
    unsigned long long S2 = 0, ST = 0;
};
struct MaskAcc {
    uint32_t n = 0, A = 0, B = 0, C = 0;
};

struct Row {
    float K0, K1, K2;
    size_t trow;
};

template <bool IMG, bool MASK>
__device__ __forceinline__ void eval_voxel(const MeasureArgs &a, const uint32_t *__restrict__ bits,
                                           const float r0x, const float r0y, const float r0z,
                                           const Row &row, int x, float xf, ImgAcc &ia, MaskAcc &ma) {
    const int SX = a.g.sd[0], SY = a.g.sd[1], SZ = a.g.sd[2];
    const uint32_t SXY = (uint32_t)SX * (uint32_t)SY;
    const float dx = __fsub_rn(xf, a.g.a[0]);
    const float qx = __fadd_rn(__fmul_rn(r0x, dx), row.K0);
    const float qy = __fadd_rn(__fmul_rn(r0y, dx), row.K1);
    const float qz = __fadd_rn(__fmul_rn(r0z, dx), row.K2);
    if (IMG) {
        const float Dm1x = (float)(SX - 1), Dm1y = (float)(SY - 1), Dm1z = (float)(SZ - 1);
        const bool in = (qx >= 0.0f) & (qx <= Dm1x) & (qy >= 0.0f) & (qy <= Dm1y) & (qz >= 0.0f) &
                        (qz <= Dm1z);
        // base corner min(floor q, D-2); clamped into the grid for voxels outside
        const float fx0 = fminf(fmaxf(floorf(qx), 0.0f), (float)(SX - 2));
        const float fy0 = fminf(fmaxf(floorf(qy), 0.0f), (float)(SY - 2));
        const float fz0 = fminf(fmaxf(floorf(qz), 0.0f), (float)(SZ - 2));
        const float fx = __fsub_rn(qx, fx0), fy = __fsub_rn(qy, fy0), fz = __fsub_rn(qz, fz0);
        const uint32_t idx = int_of(fx0) + (uint32_t)SX * int_of(fy0) + SXY * int_of(fz0);
        const uint32_t w0 = __ldg(a.src_quad + idx);
        const uint32_t w1 = __ldg(a.src_quad + idx + SXY);
        const float c00 = lerp_biased(byte_biased(w0, 0), byte_biased(w0, 1), fx);
        const float c10 = lerp_biased(byte_biased(w0, 2), byte_biased(w0, 3), fx);
        const float c01 = lerp_biased(byte_biased(w1, 0), byte_biased(w1, 1), fx);
        const float c11 = lerp_biased(byte_biased(w1, 2), byte_biased(w1, 3), fx);
        const float c0 = lerp_rn(c00, c10, fy), c1 = lerp_rn(c01, c11, fy);
        const float s = lerp_rn(c0, c1, fz);
        const uint32_t sq = __float_as_uint(__fadd_rn(s, 256.0f)) - k256Bits;   // rint(2^15 s)
        const uint32_t t = __ldg(a.tgt_img + row.trow + x);
        if (in) {
            ia.n += 1;
            ia.S1 += sq;
            ia.S2 += (unsigned long long)sq * sq;
            ia.ST += (unsigned long long)sq * t;
            ia.T1 += t;
            ia.T2 += t * t;
        }
    }
    if (MASK) {
        const float hx = __fadd_rn(qx, 0.5f), hy = __fadd_rn(qy, 0.5f), hz = __fadd_rn(qz, 0.5f);
        const bool in = (hx >= 0.0f) & (hx < (float)SX) & (hy >= 0.0f) & (hy < (float)SY) & (hz >= 0.0f) &
                        (hz < (float)SZ);
        if (in) {
            const uint32_t si = int_of(floorf(hx)) + (uint32_t)SX * int_of(floorf(hy)) + SXY * int_of(floorf(hz));
            const uint32_t sb = (bits[si >> 5] >> (si & 31)) & 1u;
            const uint32_t tb = __ldg(a.tgt_mask + row.trow + x);
            ma.n += 1;
            ma.A += sb;
            ma.B += tb;
            ma.C += sb & tb;
        }
    }
}

template <bool IMG, bool MASK, bool MASK_SMEM>
__global__ void __launch_bounds__(kThreads) k_measure(const MeasureArgs a) {
    extern __shared__ uint32_t smem_bits[];
    __shared__ unsigned long long red[kWarps][kMomStride];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int SX = a.g.sd[0], SY = a.g.sd[1], SZ = a.g.sd[2];
    const int TX = a.g.td[0], TY = a.g.td[1];
    const int rows = a.g.td[1] * a.g.td[2];

    const uint32_t *bits = a.src_bits;
    if (MASK && MASK_SMEM) {
        const int nwords = (int)(((size_t)SX * SY * SZ + 31) / 32);
        for (int i = threadIdx.x; i < nwords; i += kThreads) smem_bits[i] = a.src_bits[i];
        __syncthreads();
        bits = smem_bits;
    }
    float lo[3], hi[3];
    lo[0] = lo[1] = lo[2] = MASK ? -0.5f : 0.0f;
    hi[0] = MASK ? (float)SX - 0.5f : (float)(SX - 1);
    hi[1] = MASK ? (float)SY - 0.5f : (float)(SY - 1);
    hi[2] = MASK ? (float)SZ - 0.5f : (float)(SZ - 1);

    const long long items = (long long)a.P * a.n_rowblocks;
    for (long long item = blockIdx.x; item < items; item += gridDim.x) {
        const int p = (int)(item / a.n_rowblocks);
        const int rb = (int)(item - (long long)p * a.n_rowblocks);
        const float *Mp = a.mats + 12 * (size_t)p;
        float M[12];
#pragma unroll
        for (int i = 0; i < 12; ++i) M[i] = __ldg(Mp + i);
        const float r0[3] = {M[0], M[4], M[8]};
        ImgAcc ia;
        MaskAcc ma;

        const int row_end = min(rows, (rb + 1) * a.rows_per_item);
        for (int r = rb * a.rows_per_item + warp; r < row_end; r += kWarps) {
            const int y = r % TY, z = r / TY;
            const float dy = __fsub_rn((float)y, a.g.a[1]);
            const float dz = __fsub_rn((float)z, a.g.a[2]);
            Row row;
            row.K0 = row_K(M[1], M[2], M[3], dy, dz);
            row.K1 = row_K(M[5], M[6], M[7], dy, dz);
            row.K2 = row_K(M[9], M[10], M[11], dy, dz);
            row.trow = (size_t)r * TX;
            const float K[3] = {row.K0, row.K1, row.K2};
            int xb, xe;
            row_interval(r0, K, a.g.a[0], lo, hi, TX, xb, xe);
            int x = xb + lane;
            float xf = (float)x;
            for (; x + 32 < xe; x += 64, xf += 64.0f) {
                eval_voxel<IMG, MASK>(a, bits, r0[0], r0[1], r0[2], row, x, xf, ia, ma);
                eval_voxel<IMG, MASK>(a, bits, r0[0], r0[1], r0[2], row, x + 32, xf + 32.0f, ia, ma);
            }
            if (x < xe) eval_voxel<IMG, MASK>(a, bits, r0[0], r0[1], r0[2], row, x, xf, ia, ma);
        }

        // block reduction and one integer atomic per moment (S2: 128-bit)
        unsigned long long v[kMomStride] = {0};
        if (IMG) {
            v[0] = __reduce_add_sync(0xffffffffu, ia.n);
            v[1] = warp_sum64(ia.S1);
            v[2] = warp_sum64(ia.S2);
            v[4] = warp_sum64(ia.ST);
            v[5] = __reduce_add_sync(0xffffffffu, ia.T1);
            v[6] = warp_sum64(ia.T2);
        }
        if (MASK) {
            v[8] = __reduce_add_sync(0xffffffffu, ma.n);
            v[9] = __reduce_add_sync(0xffffffffu, ma.A);
            v[10] = __reduce_add_sync(0xffffffffu, ma.B);
            v[11] = __reduce_add_sync(0xffffffffu, ma.C);
        }
        if (lane == 0) {
#pragma unroll
            for (int j = 0; j < kMomStride; ++j) red[warp][j] = v[j];
        }
        __syncthreads();
        if (threadIdx.x < kMomStride) {
            const int j = threadIdx.x;
            const bool used = (j < 8) ? (IMG && j != 3 && j != 7) : MASK;
            if (used) {
                unsigned long long s = 0;
#pragma unroll
                for (int w = 0; w < kWarps; ++w) s += red[w][j];
                unsigned long long *dst = a.mom + (size_t)p * kMomStride;
                if (s) {
                    const unsigned long long old = atomicAdd(dst + j, s);
                    if (j == 2 && old + s < old) atomicAdd(dst + 3, 1ull);   // carry into S2's high word
                }
            }
        }
        __syncthreads();
    }
}

template <bool IMG, bool MASK, bool SMEM>
cudaError_t launch_variant(const MeasureArgs &a, size_t smem, cudaStream_t s) {
    auto kern = k_measure<IMG, MASK, SMEM>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const long long items = (long long)a.P * a.n_rowblocks;
    // persistent grid: every SM full, a few items per CTA
    long long grid = (long long)sms * per_sm * (SMEM ? 1 : 4);
    if (grid > items) grid = items;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, kThreads, smem, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

__global__ void k_pack_quads(const uint8_t *__restrict__ S, int SX, int SY, int SZ, uint32_t *__restrict__ Q) {
    const size_t n = (size_t)SX * SY * SZ;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % SX);
        const int y = (int)((i / SX) % SY);
        const bool xn = x + 1 < SX, yn = y + 1 < SY;
        const uint32_t b0 = S[i];
        const uint32_t b1 = xn ? S[i + 1] : 0u;
        const uint32_t b2 = yn ? S[i + SX] : 0u;
        const uint32_t b3 = (xn && yn) ? S[i + SX + 1] : 0u;
        Q[i] = b0 | (b1 << 8) | (b2 << 16) | (b3 << 24);
    }
}

}  // namespace

// Rows per work item: each thread then visits at most 255 voxels of one
// particle per item, which keeps its 32-bit partial sums exact.
int rows_per_item_for(int X) {
    const int segs = (X + 31) / 32;
    int per_warp = 255 / segs;
    if (per_warp < 1) per_warp = 1;
    return per_warp * kWarps;
}

cudaError_t launch_pack_quads(const uint8_t *src, const int32_t dims[3], uint32_t *quad, cudaStream_t s) {
    const size_t n = (size_t)dims[0] * dims[1] * dims[2];
    unsigned g = (unsigned)((n + 255) / 256);
    if (g > 8192) g = 8192;
    k_pack_quads<<<g, 256, 0, s>>>(src, dims[0], dims[1], dims[2], quad);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_measure(const MeasureArgs &a, bool img, bool mask, cudaStream_t s) {
    if (a.P <= 0) return cudaSuccess;
    const size_t nvox = (size_t)a.g.sd[0] * a.g.sd[1] * a.g.sd[2];
    const size_t smem_bits = ((nvox + 31) / 32) * 4;
    const bool smem = mask && smem_bits <= 160 * 1024;
    if (img && mask) return smem ? launch_variant<true, true, true>(a, smem_bits, s)
                                 : launch_variant<true, true, false>(a, 0, s);
    if (img) return launch_variant<true, false, false>(a, 0, s);
    return smem ? launch_variant<false, true, true>(a, smem_bits, s)
                : launch_variant<false, true, false>(a, 0, s);
}

}  // namespace pfreg
