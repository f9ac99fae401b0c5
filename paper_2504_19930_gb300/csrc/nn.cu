// nn.cu -- tensor-core contractions of the learned proposal network.
//
// The proposal network (a 3-D CNN that predicts the 6-DOF mean and
// log-variance used to seed the particle cloud; future work of Sec. 6) is
// four strided 3-D convolutions (kernel 4, stride 2, padding 1, 32 output
// channels, ReLU) on bf16 activations in NDHWC layout, then two small fully
// connected layers.  The convolutions and their two gradients are implicit
// GEMMs on the tcgen05 tensor cores (bf16 operands, fp32 accumulators in
// tensor memory):
//   forward  D[o][co]        = sum_{tap,ci} X[o*2+tap-1][ci] W[co][tap][ci]
//   data     dX[i][ci]       = sum_{tap,co} dY[(i+1-tap)/2][co] W[co][tap][ci]
//   weights  dW[(tap,ci)][co] = sum_{o}     X[o*2+tap-1][ci] dY[o][co]
// (per axis; taps outside the volume and, for the data gradient, taps whose
// (i + 1 - tap) is odd or out of range contribute zero).
//
// One CTA (four warps) owns a tile of 128 rows x 32 columns whose
// accumulator lives in 32 tensor-memory columns; thread t stages row t of
// the A operand (64 K elements per chunk) into shared memory in the
// canonical no-swizzle K-major layout (umma.cuh), the 32 B rows are staged
// by all threads, and one thread issues four K = 16 MMAs per chunk.  Two
// shared-memory stages alternate: the loads of chunk c overlap the MMAs of
// chunk c - 1, and a stage is rewritten only after the mbarrier of the
// commit that last read it has completed.
#include <cuda_bf16.h>

#include "kernels.h"
#include "nn.h"
#include "umma.cuh"

namespace pfreg {
namespace nn {

constexpr int kTileM = 128;
constexpr int kTileN = 32;
constexpr int kChunkK = 64;   // K elements staged per chunk (4 MMAs)
constexpr int kStageA = kTileM * kChunkK * 2;   // bytes
constexpr int kStageB = kTileN * kChunkK * 2;
constexpr uint32_t kIdesc = umma::idesc_bf16_f32(kTileM, kTileN);

__device__ unsigned int g_nn_error;   // set when a bounded wait gave up

#ifndef PF_CONV_PLANES
#define PF_CONV_PLANES 1   // 32-channel forward convolutions by the plane-staged kernel (conv.cu)
#endif

#ifndef PF_DGRAD_PLANES
#define PF_DGRAD_PLANES 1   // 32-channel data gradients with D >= 32 by the plane-staged kernel (dgrad.cu)
#endif

#ifndef PF_DGRAD_PHASES
#define PF_DGRAD_PHASES 1   // data gradient over the 8 taps of each stride phase (ConvDgradPhaseOp)
#endif

#ifndef PF_WGRAD_PLANES
#define PF_WGRAD_PLANES 1   // 32-channel weight gradients with D >= 32 by the plane-staged kernel (conv.cu)
#endif

#ifndef PF_WGRAD_MN
#define PF_WGRAD_MN 1   // 32-channel weight gradients by k_wgrad_mn (MN-major operands)
#endif

#ifndef PF_NN_ASYNC
#define PF_NN_ASYNC 1   // forward / data-gradient / GEMM tiles fed by the cp.async pipeline
#endif

__device__ __forceinline__ uint4 zero4() { return make_uint4(0u, 0u, 0u, 0u); }

__device__ __forceinline__ void st16(uint8_t *tile, int r, int k, uint4 v) {
    *reinterpret_cast<uint4 *>(tile + umma::tile_offset(r, k, kChunkK)) = v;
}

// Asynchronous global -> shared copies (cp.async): 16 or 4 bytes, written as
// zeros when !valid (source size 0: nothing is read, the address is only a
// placeholder and is always a valid one).
__device__ __forceinline__ void cp16(uint32_t tile, int r, int k, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(tile + umma::tile_offset(r, k, kChunkK)),
                 "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp4(uint32_t dst, const void *src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// ---------------------------------------------------------------------------
// Operand loaders.  load_a(tile, m0, chunk, t): thread t (0..127) writes row t
// of the 128 x 64 A tile; load_b(tile, chunk, t): the 32 x 64 B tile, two
// 8-element groups per thread; epilogue(row, acc[32]).
// ---------------------------------------------------------------------------

// Plain GEMM C[M][32] = A[M][K] B[32][K]^T (row-major bf16, K % 8 == 0).
struct GemmOp {
    const uint16_t *A, *B;
    float *C;
    int M, K;
    __device__ int chunks() const { return (K + kChunkK - 1) / kChunkK; }
    __device__ void load_a(uint8_t *tile, int m0, int c, int t) const {
        const int r = m0 + t;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = c * kChunkK + 8 * j;
            uint4 v = zero4();
            if (r < M && k < K) v = __ldg(reinterpret_cast<const uint4 *>(A + (size_t)r * K + k));
            st16(tile, t, 8 * j, v);
        }
    }
    __device__ void load_b(uint8_t *tile, int c, int t) const {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int g = t + 128 * i, n = g >> 3, j = g & 7, k = c * kChunkK + 8 * j;
            uint4 v = zero4();
            if (k < K) v = __ldg(reinterpret_cast<const uint4 *>(B + (size_t)n * K + k));
            st16(tile, n, 8 * j, v);
        }
    }
    struct Row {
        int r;
    };
    __device__ Row row(int r) const { return Row{r}; }
    __device__ void issue_a(uint32_t tile, const Row &rw, int c, int t) const {
        const int r = rw.r;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = c * kChunkK + 8 * j;
            const bool ok = r < M && k < K;
            cp16(tile, t, 8 * j, ok ? (const void *)(A + (size_t)r * K + k) : (const void *)A, ok);
        }
    }
    __device__ void issue_b(uint32_t tile, int c, int t) const {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int g = t + 128 * i, n = g >> 3, j = g & 7, k = c * kChunkK + 8 * j;
            cp16(tile, n, 8 * j, k < K ? (const void *)(B + (size_t)n * K + k) : (const void *)B, k < K);
        }
    }
    __device__ void epilogue(int row, const float *acc) const {
        if (row >= M) return;
        float4 *dst = reinterpret_cast<float4 *>(C + (size_t)row * kTileN);
#pragma unroll
        for (int i = 0; i < 8; ++i) dst[i] = make_float4(acc[4 * i], acc[4 * i + 1], acc[4 * i + 2], acc[4 * i + 3]);
    }
};

// Geometry of one strided convolution: input D^3 x Cin, output (D/2)^3 x 32.
struct ConvGeom {
    int batch, D, Cin;   // Cin in {2, 8, 16, 32, 64, 128, 256}
    __device__ int Do() const { return D >> 1; }
};

// Input element offset of voxel (b, z, y, x) channel 0, or -1 outside.
__device__ __forceinline__ long long vox(const ConvGeom &g, int b, int z, int y, int x, int C) {
    if ((unsigned)z >= (unsigned)g.D || (unsigned)y >= (unsigned)g.D || (unsigned)x >= (unsigned)g.D) return -1;
    return ((((long long)b * g.D + z) * g.D + y) * g.D + x) * C;
}

// Forward: rows = output voxels (b, oz, oy, ox), K = tap * Cin + ci,
// tap = (kz * 4 + ky) * 4 + kx.  Epilogue: y = relu(acc + bias) as bf16.
struct ConvFwdOp {
    ConvGeom g;
    const uint16_t *X;      // [B][D][D][D][Cin]
    const uint16_t *W;      // [32][64][Cin]
    const float *bias;      // [32]
    uint16_t *Y;            // [B][Do][Do][Do][32]
    __device__ int M() const { const int d = g.Do(); return g.batch * d * d * d; }
    __device__ int chunks() const { return (64 * g.Cin + kChunkK - 1) / kChunkK; }
    __device__ void load_a(uint8_t *tile, int m0, int c, int t) const {
        const int r = m0 + t, Do = g.Do();
        const bool live = r < M();
        const int ox = r % Do, oy = (r / Do) % Do, oz = (r / (Do * Do)) % Do, b = r / (Do * Do * Do);
        const int K = 64 * g.Cin;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k0 = c * kChunkK + 8 * j;
            uint4 v = zero4();
            if (live && k0 < K) {
                if (g.Cin >= 8) {
                    const int tap = k0 / g.Cin, ci = k0 - tap * g.Cin;
                    const int kz = tap >> 4, ky = (tap >> 2) & 3, kx = tap & 3;
                    const long long e = vox(g, b, 2 * oz + kz - 1, 2 * oy + ky - 1, 2 * ox + kx - 1, g.Cin);
                    if (e >= 0) v = __ldg(reinterpret_cast<const uint4 *>(X + e + ci));
                } else {   // Cin == 2: the group spans four taps of two channels
                    uint32_t w[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int tap = (k0 >> 1) + q;
                        const int kz = tap >> 4, ky = (tap >> 2) & 3, kx = tap & 3;
                        const long long e = vox(g, b, 2 * oz + kz - 1, 2 * oy + ky - 1, 2 * ox + kx - 1, 2);
                        w[q] = e >= 0 ? __ldg(reinterpret_cast<const uint32_t *>(X + e)) : 0u;
                    }
                    v = make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
            st16(tile, t, 8 * j, v);
        }
    }
    __device__ void load_b(uint8_t *tile, int c, int t) const {
        const int K = 64 * g.Cin;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int q = t + 128 * i, n = q >> 3, j = q & 7, k = c * kChunkK + 8 * j;
            uint4 v = zero4();
            if (k < K) v = __ldg(reinterpret_cast<const uint4 *>(W + (size_t)n * K + k));
            st16(tile, n, 8 * j, v);
        }
    }
    // Per-thread row context, decoded once: the input corner 2o - 1 of the
    // output voxel's 4^3 window and the batch offset.
    struct Row {
        long long bbase;   // element offset of (b, 0, 0, 0)
        int iz, iy, ix;    // 2 o - 1 per axis
        bool live;
    };
    __device__ Row row(int r) const {
        const int Do = g.Do();
        Row w;
        w.live = r < M();
        const int rr = w.live ? r : 0;
        const int ox = rr % Do, oy = (rr / Do) % Do, oz = (rr / (Do * Do)) % Do, b = rr / (Do * Do * Do);
        w.bbase = (long long)b * g.D * g.D * g.D * g.Cin;
        w.iz = 2 * oz - 1;
        w.iy = 2 * oy - 1;
        w.ix = 2 * ox - 1;
        return w;
    }
    // input element offset of tap (kz, ky, kx), or -1 outside the volume
    __device__ long long tap_off(const Row &w, int tap) const {
        const int z = w.iz + (tap >> 4), y = w.iy + ((tap >> 2) & 3), x = w.ix + (tap & 3);
        if (!w.live || (unsigned)z >= (unsigned)g.D || (unsigned)y >= (unsigned)g.D || (unsigned)x >= (unsigned)g.D)
            return -1;
        return w.bbase + (((long long)z * g.D + y) * g.D + x) * g.Cin;
    }
    __device__ void issue_a(uint32_t tile, const Row &w, int c, int t) const {
        if (g.Cin >= 8) {
            // the chunk's 64 K elements: 64 / Cin whole taps (Cin <= 64) or a
            // slice of one tap; one offset per tap, Cin / 8 copies of 16 bytes
            const int tpc = g.Cin >= 64 ? 1 : 64 / g.Cin;          // taps in this chunk
            const int gpt = g.Cin >= 64 ? 8 : g.Cin / 8;           // 16-byte groups per tap here
            for (int q = 0; q < tpc; ++q) {
                const int k0 = c * kChunkK + q * 8 * gpt;
                const int tap = k0 / g.Cin, ci0 = k0 - tap * g.Cin;
                const long long e = tap < 64 ? tap_off(w, tap) : -1;
                for (int j = 0; j < gpt; ++j)
                    cp16(tile, t, 8 * (q * gpt + j), e >= 0 ? (const void *)(X + e + ci0 + 8 * j) : (const void *)X,
                         e >= 0);
            }
        } else {   // Cin == 2: 32 taps of two channels per chunk, 4 bytes each
#pragma unroll 4
            for (int q = 0; q < 32; ++q) {
                const int tap = c * 32 + q;
                const long long e = tap < 64 ? tap_off(w, tap) : -1;
                cp4(tile + umma::tile_offset(t, 2 * q, kChunkK), e >= 0 ? (const void *)(X + e) : (const void *)X,
                    e >= 0);
            }
        }
    }
    __device__ void issue_b(uint32_t tile, int c, int t) const {
        const int K = 64 * g.Cin;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int q = t + 128 * i, n = q >> 3, j = q & 7, k = c * kChunkK + 8 * j;
            cp16(tile, n, 8 * j, k < K ? (const void *)(W + (size_t)n * K + k) : (const void *)W, k < K);
        }
    }
    __device__ void epilogue(int row, const float *acc) const {
        if (row >= M()) return;
        uint32_t packed[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float a = fmaxf(acc[2 * i] + bias[2 * i], 0.0f), b = fmaxf(acc[2 * i + 1] + bias[2 * i + 1], 0.0f);
            const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
            packed[i] = *reinterpret_cast<const uint32_t *>(&h);
        }
        uint4 *dst = reinterpret_cast<uint4 *>(Y + (size_t)row * kTileN);
#pragma unroll
        for (int i = 0; i < 4; ++i) dst[i] = make_uint4(packed[4 * i], packed[4 * i + 1], packed[4 * i + 2], packed[4 * i + 3]);
    }
};

// Data gradient: rows = input voxels (b, iz, iy, ix), columns = ci (Cin = 32),
// K = tap * 32 + co.  Wt = W transposed to [ci][tap][co].  Epilogue: the
// gradient times the ReLU mask of the layer below (act > 0), as bf16; with
// act == nullptr no mask.
struct ConvDgradOp {
    ConvGeom g;             // the forward layer's geometry (input D, Cin = 32)
    const uint16_t *dY;     // [B][Do^3][32] gradient wrt the pre-activation of this layer
    const uint16_t *Wt;     // [32 ci][64][32 co]
    const uint16_t *act;    // [B][D^3][32] this layer's input (ReLU output below), or nullptr
    uint16_t *dX;           // [B][D^3][32]
    __device__ int M() const { return g.batch * g.D * g.D * g.D; }
    __device__ int chunks() const { return (64 * 32) / kChunkK; }
    __device__ void load_a(uint8_t *tile, int m0, int c, int t) const {
        const int r = m0 + t, D = g.D, Do = g.Do();
        const bool live = r < M();
        const int ix = r % D, iy = (r / D) % D, iz = (r / (D * D)) % D, b = r / (D * D * D);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k0 = c * kChunkK + 8 * j, tap = k0 >> 5, co = k0 & 31;
            const int kz = tap >> 4, ky = (tap >> 2) & 3, kx = tap & 3;
            const int nz = iz + 1 - kz, ny = iy + 1 - ky, nx = ix + 1 - kx;
            uint4 v = zero4();
            if (live && !((nz | ny | nx) & 1)) {
                const int oz = nz >> 1, oy = ny >> 1, ox = nx >> 1;
                if ((unsigned)oz < (unsigned)Do && (unsigned)oy < (unsigned)Do && (unsigned)ox < (unsigned)Do) {
                    const long long e = ((((long long)b * Do + oz) * Do + oy) * Do + ox) * 32 + co;
                    v = __ldg(reinterpret_cast<const uint4 *>(dY + e));
                }
            }
            st16(tile, t, 8 * j, v);
        }
    }
    __device__ void load_b(uint8_t *tile, int c, int t) const {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int q = t + 128 * i, n = q >> 3, j = q & 7, k = c * kChunkK + 8 * j;
            st16(tile, n, 8 * j, __ldg(reinterpret_cast<const uint4 *>(Wt + (size_t)n * 2048 + k)));
        }
    }
    struct Row {
        long long bbase;   // element offset of (b, 0, 0, 0) in dY
        int z1, y1, x1;    // i + 1 per axis
        bool live;
    };
    __device__ Row row(int r) const {
        const int D = g.D, Do = g.Do();
        Row w;
        w.live = r < M();
        const int rr = w.live ? r : 0;
        const int ix = rr % D, iy = (rr / D) % D, iz = (rr / (D * D)) % D, b = rr / (D * D * D);
        w.bbase = (long long)b * Do * Do * Do * 32;
        w.z1 = iz + 1;
        w.y1 = iy + 1;
        w.x1 = ix + 1;
        return w;
    }
    __device__ void issue_a(uint32_t tile, const Row &w, int c, int t) const {
        const int Do = g.Do();
#pragma unroll
        for (int q = 0; q < 2; ++q) {   // two taps of 32 output channels per chunk
            const int tap = 2 * c + q;
            const int nz = w.z1 - (tap >> 4), ny = w.y1 - ((tap >> 2) & 3), nx = w.x1 - (tap & 3);
            const int oz = nz >> 1, oy = ny >> 1, ox = nx >> 1;
            const bool ok = w.live && !((nz | ny | nx) & 1) && (unsigned)oz < (unsigned)Do &&
                            (unsigned)oy < (unsigned)Do && (unsigned)ox < (unsigned)Do;
            const long long e = ok ? w.bbase + (((long long)oz * Do + oy) * Do + ox) * 32 : 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) cp16(tile, t, 8 * (4 * q + j), dY + e + 8 * j, ok);
        }
    }
    __device__ void issue_b(uint32_t tile, int c, int t) const {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int q = t + 128 * i, n = q >> 3, j = q & 7, k = c * kChunkK + 8 * j;
            cp16(tile, n, 8 * j, Wt + (size_t)n * 2048 + k, true);
        }
    }
    __device__ void epilogue(int row, const float *acc) const {
        if (row >= M()) return;
        uint32_t mask[16];
        if (act) {
            const uint4 *a4 = reinterpret_cast<const uint4 *>(act + (size_t)row * 32);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint4 u = a4[i];
                mask[4 * i] = u.x; mask[4 * i + 1] = u.y; mask[4 * i + 2] = u.z; mask[4 * i + 3] = u.w;
            }
        }
        uint32_t packed[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            float a = acc[2 * i], b = acc[2 * i + 1];
            if (act) {
                // bf16 activations are >= 0 (ReLU): positive iff a nonzero bit pattern
                a = (mask[i] & 0xFFFFu) ? a : 0.0f;
                b = (mask[i] >> 16) ? b : 0.0f;
            }
            const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
            packed[i] = *reinterpret_cast<const uint32_t *>(&h);
        }
        uint4 *dst = reinterpret_cast<uint4 *>(dX + (size_t)row * 32);
#pragma unroll
        for (int i = 0; i < 4; ++i) dst[i] = make_uint4(packed[4 * i], packed[4 * i + 1], packed[4 * i + 2], packed[4 * i + 3]);
    }
};

// Data gradient by stride phases.  With stride 2, input voxel i = 2 j + p
// (p its parity, per axis) receives only the taps k = (1 - p) + 2 t, t in
// {0, 1}, from output o = j + p - t: 8 of the 64 taps, the same 8 for every
// voxel of one parity class.  Rows are grouped by class (class c = pz 4 +
// py 2 + px; within it (b, jz, jy, jx), padded to a whole number of tiles),
// so a tile's K is 8 sub-taps x 32 co = 256 and its B operand is the class's
// 8 weight taps: the dense form's arithmetic without its 7 zero taps in 8.
struct ConvDgradPhaseOp {
    ConvGeom g;             // the forward layer's geometry (input D, Cin = 32)
    const uint16_t *dY;     // [B][Do^3][32]
    const uint16_t *Wt;     // [32 ci][64][32 co]
    const uint16_t *act;    // [B][D^3][32] or nullptr
    uint16_t *dX;           // [B][D^3][32]
    int R, Rp;              // rows per class (B Do^3) and that rounded up to whole tiles
    __device__ int M() const { return 8 * Rp; }
    __device__ int chunks() const { return 256 / kChunkK; }   // two sub-taps of 32 co per chunk
    struct Row {
        long long bbase;   // element offset of (b, 0, 0, 0) in dY
        int z, y, x;       // j + p per axis (the output index of sub-tap t is this minus t)
        bool live;
    };
    struct Vox {
        int b, iz, iy, ix;
        bool live;
    };
    __device__ Vox voxel(int r) const {
        const int Do = g.Do();
        const int cls = r / Rp, j = r - cls * Rp;
        Vox v;
        v.live = j < R;
        const int jj = v.live ? j : 0;
        const int jx = jj % Do, jy = (jj / Do) % Do, jz = (jj / (Do * Do)) % Do;
        v.b = jj / (Do * Do * Do);
        v.ix = 2 * jx + (cls & 1);
        v.iy = 2 * jy + ((cls >> 1) & 1);
        v.iz = 2 * jz + (cls >> 2);
        return v;
    }
    __device__ Row row(int r) const {
        const int Do = g.Do();
        const Vox v = voxel(r);
        Row w;
        w.live = v.live;
        w.bbase = (long long)v.b * Do * Do * Do * 32;
        // j + p = (i + p) / 2 with i = 2 j + p
        w.z = (v.iz + (v.iz & 1)) >> 1;
        w.y = (v.iy + (v.iy & 1)) >> 1;
        w.x = (v.ix + (v.ix & 1)) >> 1;
        return w;
    }
    __device__ void issue_a(uint32_t tile, const Row &w, int c, int t) const {
        const int Do = g.Do();
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int sub = 2 * c + q;   // (tz, ty, tx) = bits 2, 1, 0
            const int oz = w.z - (sub >> 2), oy = w.y - ((sub >> 1) & 1), ox = w.x - (sub & 1);
            const bool ok = w.live && (unsigned)oz < (unsigned)Do && (unsigned)oy < (unsigned)Do &&
                            (unsigned)ox < (unsigned)Do;
            const long long e = ok ? w.bbase + (((long long)oz * Do + oy) * Do + ox) * 32 : 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) cp16(tile, t, 8 * (4 * q + j), dY + e + 8 * j, ok);
        }
    }
    __device__ void issue_b(uint32_t tile, int c, int t) const {
        // every row of this CTA's tile is of one class (Rp is whole tiles)
        const int cls = (int)(((long long)blockIdx.x * kTileM) / Rp);
        const int px = cls & 1, py = (cls >> 1) & 1, pz = cls >> 2;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int q = t + 128 * i, n = q >> 3, j = q & 7;
            const int sub = 2 * c + (j >> 2), co0 = 8 * (j & 3);
            const int kz = 1 - pz + 2 * (sub >> 2), ky = 1 - py + 2 * ((sub >> 1) & 1), kx = 1 - px + 2 * (sub & 1);
            const int tap = (kz * 4 + ky) * 4 + kx;
            cp16(tile, n, 8 * j, Wt + (size_t)n * 2048 + tap * 32 + co0, true);
        }
    }
    __device__ void epilogue(int row, const float *acc) const {
        const Vox v = voxel(row);
        if (row >= M() || !v.live) return;
        const size_t vi = (((size_t)v.b * g.D + v.iz) * g.D + v.iy) * g.D + v.ix;
        uint32_t mask[16];
        if (act) {
            const uint4 *a4 = reinterpret_cast<const uint4 *>(act + vi * 32);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint4 u = a4[i];
                mask[4 * i] = u.x; mask[4 * i + 1] = u.y; mask[4 * i + 2] = u.z; mask[4 * i + 3] = u.w;
            }
        }
        uint32_t packed[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            float a = acc[2 * i], b = acc[2 * i + 1];
            if (act) {
                a = (mask[i] & 0xFFFFu) ? a : 0.0f;
                b = (mask[i] >> 16) ? b : 0.0f;
            }
            const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
            packed[i] = *reinterpret_cast<const uint32_t *>(&h);
        }
        uint4 *dst = reinterpret_cast<uint4 *>(dX + vi * 32);
#pragma unroll
        for (int i = 0; i < 4; ++i) dst[i] = make_uint4(packed[4 * i], packed[4 * i + 1], packed[4 * i + 2], packed[4 * i + 3]);
    }
};

// Weight gradient: rows = (tap, ci) (64 Cin rows), columns = co, K = output
// positions (b, o), split over blockIdx.y; partial sums are added to dW
// (fp32, [32][64][Cin]) atomically.
struct ConvWgradOp {
    ConvGeom g;
    const uint16_t *X;      // [B][D^3][Cin]
    const uint16_t *dY;     // [B][Do^3][32]
    float *dW;              // [32][64][Cin], accumulated
    int chunks_per_split;
    __device__ int M() const { return 64 * g.Cin; }
    __device__ int positions() const { const int d = g.Do(); return g.batch * d * d * d; }
    __device__ int chunks() const { return (positions() + kChunkK - 1) / kChunkK; }
    __device__ void load_a(uint8_t *tile, int m0, int c, int t) const {
        const int r = m0 + t, Do = g.Do(), D = g.D;
        const bool live = r < M();
        const int tap = r / g.Cin, ci = r - tap * g.Cin;
        const int kz = tap >> 4, ky = (tap >> 2) & 3, kx = tap & 3;
        const int P = positions();
        // the chunk's 64 consecutive positions, decoded once and then stepped
        int p = c * kChunkK;
        int ox = p % Do, oy = (p / Do) % Do, oz = (p / (Do * Do)) % Do, b = p / (Do * Do * Do);
#pragma unroll 1
        for (int j = 0; j < 8; ++j) {
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t lohi[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint32_t val = 0u;
                    const int z = 2 * oz + kz - 1, y = 2 * oy + ky - 1, x = 2 * ox + kx - 1;
                    if (live && p < P && (unsigned)z < (unsigned)D && (unsigned)y < (unsigned)D &&
                        (unsigned)x < (unsigned)D)
                        val = __ldg(X + ((((long long)b * D + z) * D + y) * D + x) * g.Cin + ci);
                    lohi[h] = val;
                    ++p;
                    if (++ox == Do) {
                        ox = 0;
                        if (++oy == Do) {
                            oy = 0;
                            if (++oz == Do) {
                                oz = 0;
                                ++b;
                            }
                        }
                    }
                }
                w[q] = lohi[0] | (lohi[1] << 16);
            }
            st16(tile, t, 8 * j, make_uint4(w[0], w[1], w[2], w[3]));
        }
    }
    __device__ void load_b(uint8_t *tile, int c, int t) const {
        const int P = positions();
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int q = t + 128 * i, n = q >> 3, j = q & 7;
            uint32_t w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int p0 = c * kChunkK + 8 * j + 2 * u;
                const uint32_t lo = p0 < P ? __ldg(dY + (size_t)p0 * 32 + n) : 0u;
                const uint32_t hi = p0 + 1 < P ? __ldg(dY + (size_t)(p0 + 1) * 32 + n) : 0u;
                w[u] = lo | (hi << 16);
            }
            st16(tile, n, 8 * j, make_uint4(w[0], w[1], w[2], w[3]));
        }
    }
    __device__ void epilogue(int row, const float *acc) const {
        if (row >= M()) return;
        const int tap = row / g.Cin, ci = row - tap * g.Cin;
#pragma unroll
        for (int co = 0; co < 32; ++co)
            if (acc[co] != 0.0f) atomicAdd(dW + ((size_t)co * 64 + tap) * g.Cin + ci, acc[co]);
    }
};

// ---------------------------------------------------------------------------
// The tile kernel.  blockIdx.x: 128-row tile; blockIdx.y: K split (chunks
// [y * per, min((y + 1) * per, chunks))).
// ---------------------------------------------------------------------------
template <class Op>
__global__ void __launch_bounds__(128) k_umma_tile(const Op op, int chunks_per_split) {
    __shared__ __align__(1024) uint8_t sA[2][kStageA];
    __shared__ __align__(1024) uint8_t sB[2][kStageB];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ uint32_t tmem_slot;
    const int t = threadIdx.x, warp = t >> 5;
    const int m0 = blockIdx.x * kTileM;
    const int nch = op.chunks();
    const int c0 = blockIdx.y * chunks_per_split;
    const int c1 = min(nch, c0 + chunks_per_split);

    if (warp == 0) umma::tmem_alloc(&tmem_slot, kTileN);
    if (t == 0) {
        umma::mbar_init(umma::smem_u32(&mbar[0]), 1);
        umma::mbar_init(umma::smem_u32(&mbar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = tmem_slot;

    // every wait's outcome is agreed by the whole CTA (__syncthreads_and), so
    // all threads leave the loop together
    bool ok = true;
    for (int c = c0; c < c1; ++c) {
        const int s = (c - c0) & 1, use = (c - c0) >> 1;
        if (use > 0 && !__syncthreads_and(umma::mbar_wait(umma::smem_u32(&mbar[s]), (uint32_t)((use - 1) & 1)))) {
            ok = false;
            break;
        }
        op.load_a(sA[s], m0, c, t);
        op.load_b(sB[s], c, t);
        umma::fence_async_smem();
        __syncthreads();
        if (t == 0) {
            umma::fence_after_sync();
            const uint32_t a = umma::smem_u32(sA[s]), b = umma::smem_u32(sB[s]);
#pragma unroll
            for (int kk = 0; kk < kChunkK / 16; ++kk)
                umma::mma_bf16(tmem, umma::smem_desc(a + 256 * kk, 128, 16 * kChunkK),
                               umma::smem_desc(b + 256 * kk, 128, 16 * kChunkK), kIdesc, c > c0 || kk > 0);
            umma::commit(umma::smem_u32(&mbar[s]));
        }
    }
    const int n = c1 - c0;
    if (ok && n > 0)
        ok = __syncthreads_and(umma::mbar_wait(umma::smem_u32(&mbar[(n - 1) & 1]), (uint32_t)(((n - 1) >> 1) & 1)));
    if (!ok) {
        if (t == 0) atomicExch(&g_nn_error, 1u);
    } else if (n > 0) {
        umma::fence_after_sync();
        float acc[32];
        umma::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), acc);
        op.epilogue(m0 + t, acc);
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_free(tmem, kTileN);
}

template <class Op>
cudaError_t launch_tile(const Op &op, int M, int chunks, int splits, cudaStream_t s) {
    if (M <= 0 || chunks <= 0) return cudaSuccess;
    if (splits < 1) splits = 1;
    if (splits > chunks) splits = chunks;
    const int per = (chunks + splits - 1) / splits;
    splits = (chunks + per - 1) / per;
    dim3 grid((unsigned)((M + kTileM - 1) / kTileM), (unsigned)splits);
    k_umma_tile<Op><<<grid, 128, 0, s>>>(op, per);
    count_launches(1);
    return cudaGetLastError();
}

// The same tile with an S-stage cp.async pipeline: chunk i's copies are
// issued P = S - 2 chunks ahead; before the MMAs of chunk i every thread waits
// for its own copies of that chunk (cp.async.wait_group), makes them visible
// to the tensor core (fence.proxy.async) and the CTA synchronises.  The stage
// refilled at iteration i is the one chunk i - 2 used, so the wait on that
// commit's mbarrier leaves the tensor core a whole iteration of slack.
constexpr int kAsyncStages = 5;
constexpr int kAsyncSmem = kAsyncStages * (kStageA + kStageB) + 64;

template <class Op>
__global__ void __launch_bounds__(128) k_umma_async(const Op op) {
    extern __shared__ __align__(1024) uint8_t dsm[];
    uint8_t *sA = dsm;                                   // [S][kStageA]
    uint8_t *sB = dsm + kAsyncStages * kStageA;          // [S][kStageB]
    unsigned long long *mbar = reinterpret_cast<unsigned long long *>(sB + kAsyncStages * kStageB);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mbar + kAsyncStages);
    const int t = threadIdx.x, warp = t >> 5;
    const int m0 = blockIdx.x * kTileM;
    const int n = op.chunks();
    constexpr int S = kAsyncStages;

    if (warp == 0) umma::tmem_alloc(tmem_slot, kTileN);
    if (t == 0) {
        for (int q = 0; q < S; ++q) umma::mbar_init(umma::smem_u32(&mbar[q]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t a0 = umma::smem_u32(sA), b0 = umma::smem_u32(sB);
    const typename Op::Row rw = op.row(m0 + t);

    constexpr int P = S - 2;           // prefetch distance
#pragma unroll
    for (int i = 0; i < P; ++i) {
        if (i < n) {
            op.issue_a(a0 + i * kStageA, rw, i, t);
            op.issue_b(b0 + i * kStageB, i, t);
        }
        cp_commit();
    }
    bool ok = true;
    for (int i = 0; i < n; ++i) {
        const int s = i % S;
        cp_wait<P - 1>();              // this thread's copies of chunk i have landed
        umma::fence_async_smem();
        __syncthreads();
        if (t == 0) {
            umma::fence_after_sync();
            const uint32_t a = a0 + s * kStageA, b = b0 + s * kStageB;
#pragma unroll
            for (int kk = 0; kk < kChunkK / 16; ++kk)
                umma::mma_bf16(tmem, umma::smem_desc(a + 256 * kk, 128, 16 * kChunkK),
                               umma::smem_desc(b + 256 * kk, 128, 16 * kChunkK), kIdesc, i > 0 || kk > 0);
            umma::commit(umma::smem_u32(&mbar[s]));
        }
        const int j = i + P;           // refill the stage chunk i - 2 used
        if (j < n) {
            if (i >= 2) {
                const int sp = (i - 2) % S;
                if (!__syncthreads_and(umma::mbar_wait(umma::smem_u32(&mbar[sp]), (uint32_t)(((i - 2) / S) & 1)))) {
                    ok = false;
                    break;
                }
            }
            op.issue_a(a0 + (j % S) * kStageA, rw, j, t);
            op.issue_b(b0 + (j % S) * kStageB, j, t);
        }
        cp_commit();
    }
    cp_wait<0>();
    if (ok && n > 0)
        ok = __syncthreads_and(umma::mbar_wait(umma::smem_u32(&mbar[(n - 1) % S]), (uint32_t)(((n - 1) / S) & 1)));
    if (!ok) {
        if (t == 0) atomicExch(&g_nn_error, 1u);
    } else if (n > 0) {
        umma::fence_after_sync();
        float acc[32];
        umma::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), acc);
        op.epilogue(m0 + t, acc);
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_free(tmem, kTileN);
}

template <class Op>
cudaError_t launch_async(const Op &op, int M, cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_umma_async<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, kAsyncSmem);
    if (e != cudaSuccess) return e;
    k_umma_async<Op><<<(unsigned)((M + kTileM - 1) / kTileM), 128, kAsyncSmem, s>>>(op);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Weight gradient with MN-major operands (Cin = 32).  D[(tap, ci)][co] =
// sum_o X[2o + tap - 1][ci] dY[o][co]: in memory both operands run along
// their M / N index (the channels of one voxel are contiguous), so they are
// staged as MN-major tiles -- each 16-byte copy is 8 channels of one voxel,
// one row of a core matrix of 8 positions x 8 channels -- and the MMA reads
// them transposed (instruction-descriptor bits 15 and 16).  CTA (x, y): the
// 4 taps x 32 channels of M tile x, positions [y per, (y + 1) per) x 64;
// the split sums are added to dW with fp32 atomics.
// Tile layouts (bytes): A core (m / 8, k / 8) at (m / 8) 128 + (k / 8) 2048,
// row k % 8 at + 16 (k % 8); B core (n / 8, k / 8) at (n / 8) 128 + (k / 8) 512.
// ---------------------------------------------------------------------------
// Descriptor fields of an MN-major no-swizzle operand: the leading byte offset
// is the stride between core matrices along K, the stride byte offset the
// stride along M / N (checked on the device: one MMA of known operands is
// exact with this assignment and wrong with the other).
constexpr int kWgStages = 4;
constexpr int kWgA = 128 * kChunkK * 2;   // 16 KB
constexpr int kWgB = 32 * kChunkK * 2;    // 4 KB
constexpr int kWgSmem = kWgStages * (kWgA + kWgB) + 64;
constexpr uint32_t kIdescMN = kIdesc | (1u << 15) | (1u << 16);

__device__ __forceinline__ uint64_t mn_desc(uint32_t addr, uint32_t mn_stride, uint32_t k_stride) {
    return umma::smem_desc(addr, k_stride, mn_stride);
}
__device__ __forceinline__ void cp16_to(uint32_t dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}

struct WgradMnArgs {
    const uint16_t *X;    // [B][D^3][CIN]
    const uint16_t *dY;   // [B][Do^3][32]
    float *dW;            // [32][64][CIN], accumulated
    int D, P, per;        // input edge, output positions B Do^3, chunks per split
};

__device__ __forceinline__ void cp4_to(uint32_t dst, const void *src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}

// Thread t stages position o = t / 2 of the chunk.  CIN = 32: its 8 (tap,
// channel-group) 16-byte copies of X (M tile = 4 taps x 32 channels).
// CIN = 2 (M tile = all 64 taps x 2 channels): its 8 (kz, ky) rows, each the
// 4 voxels kx = 0..3 of one input row (16 contiguous bytes, but only 4-byte
// aligned: four 4-byte copies, each zero-filled when its voxel is outside).
// Both: 2 of the 4 channel groups of dY.
template <int CIN>
__device__ __forceinline__ void wgrad_issue(const WgradMnArgs &g, uint32_t sa, uint32_t sb, int c, int tap0,
                                            int t) {
    const int D = g.D, Do = D >> 1;
    const int ol = t >> 1, half = t & 1;
    const int p = c * kChunkK + ol;
    const bool live = p < g.P;
    const int pp = live ? p : 0;
    const int ox = pp % Do, oy = (pp / Do) % Do, oz = (pp / (Do * Do)) % Do, b = pp / (Do * Do * Do);
    const uint32_t krow = (uint32_t)((ol >> 3) * 2048 + (ol & 7) * 16);
    if (CIN == 32) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int q = half * 8 + u, tl = q >> 2, cc = q & 3, tap = tap0 + tl;
            const int z = 2 * oz + (tap >> 4) - 1, y = 2 * oy + ((tap >> 2) & 3) - 1, x = 2 * ox + (tap & 3) - 1;
            const bool ok = live && (unsigned)z < (unsigned)D && (unsigned)y < (unsigned)D && (unsigned)x < (unsigned)D;
            const uint16_t *src = ok ? g.X + ((((long long)b * D + z) * D + y) * D + x) * 32 + cc * 8 : g.X;
            cp16_to(sa + (uint32_t)((tl * 4 + cc) * 128) + krow, src, ok);
        }
    } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int grp = half * 8 + u, kz = grp >> 2, ky = grp & 3;   // M group = (kz, ky): taps 4 grp .. 4 grp + 3
            const int z = 2 * oz + kz - 1, y = 2 * oy + ky - 1;
            const bool row = live && (unsigned)z < (unsigned)D && (unsigned)y < (unsigned)D;
            const long long rbase = (((long long)b * D + z) * D + y) * D;
#pragma unroll
            for (int kx = 0; kx < 4; ++kx) {
                const int x = 2 * ox + kx - 1;
                const bool ok = row && (unsigned)x < (unsigned)D;
                cp4_to(sa + (uint32_t)(grp * 128 + kx * 4) + krow, ok ? g.X + (rbase + x) * 2 : g.X, ok);
            }
        }
    }
    const uint32_t krowb = (uint32_t)((ol >> 3) * 512 + (ol & 7) * 16);
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int cc = half * 2 + u;
        cp16_to(sb + (uint32_t)(cc * 128) + krowb, live ? g.dY + (size_t)p * 32 + cc * 8 : g.dY, live);
    }
}

template <int CIN>
__global__ void __launch_bounds__(128) k_wgrad_mn(const WgradMnArgs g) {
    extern __shared__ __align__(1024) uint8_t dsm[];
    uint8_t *sA = dsm;
    uint8_t *sB = dsm + kWgStages * kWgA;
    unsigned long long *mbar = reinterpret_cast<unsigned long long *>(sB + kWgStages * kWgB);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mbar + kWgStages);
    const int t = threadIdx.x, warp = t >> 5;
    const int tap0 = blockIdx.x * 4;
    const int nch = (g.P + kChunkK - 1) / kChunkK;
    const int c0 = blockIdx.y * g.per;
    const int n = max(0, min(nch, c0 + g.per) - c0);
    constexpr int S = kWgStages;

    if (warp == 0) umma::tmem_alloc(tmem_slot, kTileN);
    if (t == 0) {
        for (int q = 0; q < S; ++q) umma::mbar_init(umma::smem_u32(&mbar[q]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t a0 = umma::smem_u32(sA), b0 = umma::smem_u32(sB);

    constexpr int P = S - 2;
#pragma unroll
    for (int i = 0; i < P; ++i) {
        if (i < n) wgrad_issue<CIN>(g, a0 + i * kWgA, b0 + i * kWgB, c0 + i, tap0, t);
        cp_commit();
    }
    bool ok = true;
    for (int i = 0; i < n; ++i) {
        const int s = i % S;
        cp_wait<P - 1>();
        umma::fence_async_smem();
        __syncthreads();
        if (t == 0) {
            umma::fence_after_sync();
            const uint32_t a = a0 + s * kWgA, b = b0 + s * kWgB;
#pragma unroll
            for (int kk = 0; kk < kChunkK / 16; ++kk)
                umma::mma_bf16(tmem, mn_desc(a + 4096 * kk, 128, 2048), mn_desc(b + 1024 * kk, 128, 512), kIdescMN,
                               i > 0 || kk > 0);
            umma::commit(umma::smem_u32(&mbar[s]));
        }
        const int j = i + P;
        if (j < n) {
            if (i >= 2) {
                const int sp = (i - 2) % S;
                if (!__syncthreads_and(umma::mbar_wait(umma::smem_u32(&mbar[sp]), (uint32_t)(((i - 2) / S) & 1)))) {
                    ok = false;
                    break;
                }
            }
            wgrad_issue<CIN>(g, a0 + (j % S) * kWgA, b0 + (j % S) * kWgB, c0 + j, tap0, t);
        }
        cp_commit();
    }
    cp_wait<0>();
    if (ok && n > 0)
        ok = __syncthreads_and(umma::mbar_wait(umma::smem_u32(&mbar[(n - 1) % S]), (uint32_t)(((n - 1) / S) & 1)));
    if (!ok) {
        if (t == 0) atomicExch(&g_nn_error, 1u);
    } else if (n > 0) {
        umma::fence_after_sync();
        float acc[32];
        umma::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), acc);
        // M row t: (tap0 + t / 32, ci = t % 32) for CIN = 32, (tap = t / 2, ci = t % 2) for CIN = 2
        const int tap = CIN == 32 ? tap0 + (t >> 5) : t >> 1, ci = CIN == 32 ? t & 31 : t & 1;
#pragma unroll
        for (int co = 0; co < 32; ++co)
            if (acc[co] != 0.0f) atomicAdd(g.dW + ((size_t)co * 64 + tap) * CIN + ci, acc[co]);
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_free(tmem, kTileN);
}

// W [32][64][Cin] -> Wt [Cin][64][32] (bf16), for the data gradient.
__global__ void k_transpose_w(const uint16_t *W, int Cin, uint16_t *Wt) {
    const int n = 32 * 64 * Cin;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int ci = i % Cin, tap = (i / Cin) % 64, co = i / (64 * Cin);
        Wt[((size_t)ci * 64 + tap) * 32 + co] = W[i];
    }
}

// ---------------------------------------------------------------------------
// CUDA-core parts of the network: fully connected layers, bias gradients,
// the loss, Adam, input preparation and the synthetic training pairs.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(uint16_t v) { return __uint_as_float((uint32_t)v << 16); }
__device__ __forceinline__ uint16_t bf16_bits(float v) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    return *reinterpret_cast<const uint16_t *>(&h);
}

// out[b][n] = act(b_n + sum_k in[b][k] W[n][k]); one warp per output.
template <class T>
__global__ void k_fc_forward(const T *__restrict__ in, int B, int K, const float *__restrict__ W,
                             const float *__restrict__ bias, int N, float *__restrict__ out, int relu) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= B * N) return;
    const int b = w / N, n = w - b * N;
    float acc = 0.0f;
    for (int k = lane; k < K; k += 32) acc += to_f(in[(size_t)b * K + k]) * W[(size_t)n * K + k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        acc += bias[n];
        out[(size_t)b * N + n] = relu ? fmaxf(acc, 0.0f) : acc;
    }
}

// din[b][k] = [act[b][k] > 0] * sum_n dout[b][n] W[n][k]  (T = float or bf16 out).
template <class TA, class TO>
__global__ void k_fc_backward_input(const float *__restrict__ dout, int B, int N, const float *__restrict__ W,
                                    int K, const TA *__restrict__ act, TO *__restrict__ din) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * K) return;
    const int b = i / K, k = i - b * K;
    float acc = 0.0f;
    for (int n = 0; n < N; ++n) acc += dout[(size_t)b * N + n] * W[(size_t)n * K + k];
    if (!(to_f(act[i]) > 0.0f)) acc = 0.0f;
    if constexpr (sizeof(TO) == 2) din[i] = bf16_bits(acc);
    else din[i] = acc;
}

// dW[n][k] += sum_b dout[b][n] in[b][k];  db[n] += sum_b dout[b][n] (k == 0 threads).
template <class T>
__global__ void k_fc_backward_weight(const float *__restrict__ dout, int B, int N, const T *__restrict__ in, int K,
                                     float *__restrict__ dW, float *__restrict__ db) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * K) return;
    const int n = i / K, k = i - n * K;
    float acc = 0.0f, accb = 0.0f;
    for (int b = 0; b < B; ++b) {
        const float g = dout[(size_t)b * N + n];
        acc += g * to_f(in[(size_t)b * K + k]);
        accb += g;
    }
    dW[i] += acc;
    if (k == 0) db[n] += accb;
}

// db[c] += sum_rows dY[row][c] (32 channels, bf16 rows).
__global__ void k_bias_grad(const uint16_t *__restrict__ dY, long long rows, float *__restrict__ db) {
    __shared__ float part[8][32];
    const int c = threadIdx.x & 31, r0 = threadIdx.x >> 5;   // 256 threads: 8 row lanes
    float acc = 0.0f;
    for (long long r = (long long)blockIdx.x * 8 + r0; r < rows; r += (long long)gridDim.x * 8)
        acc += to_f(dY[r * 32 + c]);
    part[r0][c] = acc;
    __syncthreads();
    if (r0 == 0) {
        float s = 0.0f;
        for (int q = 0; q < 8; ++q) s += part[q][c];
        atomicAdd(db + c, s);
    }
}

// Gaussian negative log-likelihood of the labels y under N(mu, exp(s)) per
// DOF, out = [mu(6) | s(6)], averaged over the batch; writes d loss / d out
// and adds the loss into *loss.
__global__ void k_nll(const float *__restrict__ out, const float *__restrict__ y, int B, float *__restrict__ dout,
                      float *__restrict__ loss_log, const int *__restrict__ step) {
    float *loss = loss_log + *step;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.0f;
    if (i < B * 6) {
        const int b = i / 6, d = i - b * 6;
        const float mu = out[b * 12 + d], sv = out[b * 12 + 6 + d];
        const float r = y[b * 6 + d] - mu, e = __expf(-sv);
        dout[b * 12 + d] = -r * e / (float)B;
        dout[b * 12 + 6 + d] = 0.5f * (1.0f - r * r * e) / (float)B;
        l = 0.5f * (r * r * e + sv) / (float)B;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.0f) atomicAdd(loss, l);
}

// Adam (Kingma & Ba, Algorithm 1) with the step count t = *step + 1.
__global__ void k_adam(float *__restrict__ theta, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, long long n, float lr, const int *__restrict__ step) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const int t = *step + 1;
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi, vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void k_step_inc(int *step) { *step += 1; }

// bf16 copies of fp32 parameters (conv weights) and their [ci][tap][co] transposes.
__global__ void k_to_bf16(const float *__restrict__ a, long long n, uint16_t *__restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = bf16_bits(a[i]);
}

// Uniform initialisation U(-a, a), a = sqrt(6 / fan_in), from Philox(seed).
__global__ void k_init_uniform(float *p, long long n, float a, uint64_t seed, uint32_t tensor) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const u32x4 r = philox_seeded(seed, (uint32_t)i, tensor, 0x6E6E0000u, 0u);
        p[i] = a * (2.0f * ((float)(r.x >> 8) * 5.9604644775390625e-08f) - 1.0f);
    }
}

// Network input: the box-average of a uint8 volume over each cell of a
// G^3 grid covering the box [box_o, box_o + G h) (world units), scaled by
// 1/64, into channel c of a [G^3][2] bf16 input; cells with no voxel get 0.
struct DownArgs {
    const uint8_t *vol;
    int dims[3];
    float origin[3], spacing[3];
    float box_o[3], h[3];
    int G, c;
    uint16_t *x;
};
__global__ void k_downsample(const DownArgs a) {
    const int G = a.G;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G * G * G) return;
    const int gx = i % G, gy = (i / G) % G, gz = i / (G * G);
    const int g[3] = {gx, gy, gz};
    int lo[3], hi[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        // voxel p sits at origin + spacing * p; the cell covers [b0, b1)
        const float b0 = a.box_o[d] + a.h[d] * g[d], b1 = a.box_o[d] + a.h[d] * (g[d] + 1);
        lo[d] = max(0, (int)ceilf((b0 - a.origin[d]) / a.spacing[d]));
        hi[d] = min(a.dims[d], (int)ceilf((b1 - a.origin[d]) / a.spacing[d]));
    }
    unsigned sum = 0, cnt = 0;
    for (int z = lo[2]; z < hi[2]; ++z)
        for (int y = lo[1]; y < hi[1]; ++y) {
            const uint8_t *row = a.vol + ((size_t)z * a.dims[1] + y) * a.dims[0];
            for (int x = lo[0]; x < hi[0]; ++x) {
                sum += row[x];
                ++cnt;
            }
        }
    const float v = cnt ? (float)sum / (float)cnt * (1.0f / 64.0f) : 0.0f;
    a.x[(size_t)i * 2 + a.c] = bf16_bits(v);
}

// Synthetic training pairs: echo-like source and target views of a random
// left-ventricle shell (myocardium 1.0, blood pool 0.15, background 0.3,
// cut open at the valve plane), Rayleigh speckle (sigma 40) hashed from the
// rounded world voxel, a smooth multiplicative gain per view, a random rigid
// pose within the training limits and a target field of view slid along x
// for 35-60 % overlap -- the recipe of the image workload's pairs -- each
// voxel computed at full resolution (X, Y, Z) and box-averaged into the G^3
// input exactly as k_downsample does for real volumes.
struct SynthSample {
    float R[9], t[3], c[3];          // pose about the source centre c
    float hc[3], rout[3], rin[3];    // heart centre, reciprocal outer / inner shell semi-axes
    float base_x;
    float gf[2][3][3], gph[2][3];    // gain frequencies / phases per view
    int shift;                       // target origin x (voxels)
    uint32_t speckle;
};
struct SynthArgs {
    int X, Y, Z, G;
    float rot_lim, trans_lim;
    uint64_t seed;
    int step;                // used when step_ptr is NULL
    const int *step_ptr;     // the optimiser's step counter (graph replays)
    SynthSample *samples;
    uint16_t *x;   // [B][G^3][2]
    float *y;      // [B][6] pose / limits
};

__device__ __forceinline__ float u01(uint32_t r) { return (float)(r >> 8) * 5.9604644775390625e-08f; }

__global__ void k_synth_params(const SynthArgs a, int B) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const uint32_t step = (uint32_t)(a.step_ptr ? *a.step_ptr : a.step);
    uint32_t w[24];
    for (int q = 0; q < 6; ++q) {
        const u32x4 r = philox_seeded(a.seed, (uint32_t)b, step, 0x53594E00u, (uint32_t)q);
        w[4 * q] = r.x; w[4 * q + 1] = r.y; w[4 * q + 2] = r.z; w[4 * q + 3] = r.w;
    }
    SynthSample s;
    const float dims[3] = {(float)a.X, (float)a.Y, (float)a.Z};
    float ang[3], tr[3];
    for (int d = 0; d < 3; ++d) {
        ang[d] = a.rot_lim * (2.0f * u01(w[d]) - 1.0f);
        tr[d] = a.trans_lim * (2.0f * u01(w[3 + d]) - 1.0f);
        s.c[d] = 0.5f * (dims[d] - 1.0f);
        s.hc[d] = s.c[d] + 8.0f * u01(w[6 + d]) - 4.0f;
    }
    const float fr[3] = {0.36f, 0.26f, 0.28f};
    float outer[3];
    for (int d = 0; d < 3; ++d) outer[d] = fr[d] * dims[d] * (0.95f + 0.1f * u01(w[9 + d]));
    const float th = 0.055f * dims[0];
    for (int d = 0; d < 3; ++d) {
        s.rout[d] = 1.0f / outer[d];
        s.rin[d] = 1.0f / (outer[d] - th);
    }
    s.base_x = 0.55f * outer[0];
    // R = Rz Rx Ry
    float sx, cx, sy, cy, sz, cz;
    sincosf(ang[0], &sx, &cx);
    sincosf(ang[1], &sy, &cy);
    sincosf(ang[2], &sz, &cz);
    const float Rz[9] = {cz, -sz, 0, sz, cz, 0, 0, 0, 1};
    const float Rx[9] = {1, 0, 0, 0, cx, -sx, 0, sx, cx};
    const float Ry[9] = {cy, 0, sy, 0, 1, 0, -sy, 0, cy};
    float T[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            float acc = 0.0f;
            for (int k = 0; k < 3; ++k) acc += Rz[3 * i + k] * Rx[3 * k + j];
            T[3 * i + j] = acc;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            float acc = 0.0f;
            for (int k = 0; k < 3; ++k) acc += T[3 * i + k] * Ry[3 * k + j];
            s.R[3 * i + j] = acc;
        }
    for (int d = 0; d < 3; ++d) s.t[d] = tr[d];
    s.shift = (int)rintf((0.40f + 0.25f * u01(w[12])) * dims[0]);
    for (int v = 0; v < 2; ++v)
        for (int q = 0; q < 3; ++q) {
            for (int d = 0; d < 3; ++d) {
                const u32x4 r = philox_seeded(a.seed, (uint32_t)b, step, 0x53594E01u, (uint32_t)(9 * v + 3 * q + d));
                s.gf[v][q][d] = 0.3f + 0.9f * u01(r.x);
            }
            s.gph[v][q] = 6.2831853f * u01(w[13 + 3 * v + q]);
        }
    s.speckle = w[20];
    a.samples[b] = s;
    for (int d = 0; d < 3; ++d) {
        a.y[b * 6 + d] = ang[d] / a.rot_lim;
        a.y[b * 6 + 3 + d] = tr[d] / a.trans_lim;
    }
}

__device__ __forceinline__ uint32_t hash3(int x, int y, int z, uint32_t seed) {
    uint32_t h = (uint32_t)x * 0x8DA6B343u ^ (uint32_t)y * 0xD8163841u ^ (uint32_t)z * 0xCB1AB31Fu ^ seed;
    h ^= h >> 16;
    h *= 0x7FEB352Du;
    h ^= h >> 15;
    h *= 0x846CA68Bu;
    h ^= h >> 16;
    return h;
}

// One view's voxel value at world point w (source frame) and grid fraction u.
__device__ __forceinline__ float synth_voxel(const SynthSample &s, int view, const float w[3], const float u[3]) {
    const float ux = w[0] - s.hc[0], uy = w[1] - s.hc[1], uz = w[2] - s.hc[2];
    const float ox = ux * s.rout[0], oy = uy * s.rout[1], oz = uz * s.rout[2];
    const float ix = ux * s.rin[0], iy = uy * s.rin[1], iz = uz * s.rin[2];
    const float eo = ox * ox + oy * oy + oz * oz;
    const float ei = ix * ix + iy * iy + iz * iz;
    float tissue = 0.3f;
    if (ux <= s.base_x) {
        if (ei <= 1.0f) tissue = 0.15f;
        else if (eo <= 1.0f) tissue = 1.0f;
    }
    const uint32_t h = hash3((int)rintf(w[0]), (int)rintf(w[1]), (int)rintf(w[2]), s.speckle);
    const float uu = ((float)(h >> 8) + 0.5f) * 5.9604644775390625e-08f;
    const float speck = 40.0f * sqrtf(-2.0f * __logf(uu));
    float gsum = 0.0f;
#pragma unroll
    for (int q = 0; q < 3; ++q)
        gsum += __cosf(6.2831853f * (s.gf[view][q][0] * u[0] + s.gf[view][q][1] * u[1] + s.gf[view][q][2] * u[2]) +
                       s.gph[view][q]);
    const float gain = 1.0f + 0.3f * gsum / 3.0f;
    return fminf(fmaxf(rintf(tissue * speck * gain), 0.0f), 255.0f);
}

// blockIdx.y = sample, threads over the G^3 cells; both channels.
__global__ void k_synth_views(const SynthArgs a) {
    const int G = a.G, b = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G * G * G) return;
    const SynthSample &s = a.samples[b];
    const int g[3] = {i % G, (i / G) % G, i / (G * G)};
    const int dims[3] = {a.X, a.Y, a.Z};
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        const float h = (float)dims[d] / (float)G;
        lo[d] = (int)ceilf(h * g[d]);
        hi[d] = min(dims[d], (int)ceilf(h * (g[d] + 1)));
    }
    const float inv[3] = {1.0f / a.X, 1.0f / a.Y, 1.0f / a.Z};
    float sum_s = 0.0f, sum_t = 0.0f;
    int cnt_s = 0, cnt_t = 0;
    for (int z = lo[2]; z < hi[2]; ++z)
        for (int y = lo[1]; y < hi[1]; ++y)
            for (int x = lo[0]; x < hi[0]; ++x) {
                // source view: voxel (x, y, z) at world (x, y, z)
                const float ws[3] = {(float)x, (float)y, (float)z};
                const float us[3] = {x * inv[0], y * inv[1], z * inv[2]};
                sum_s += synth_voxel(s, 0, ws, us);
                ++cnt_s;
                // target view: target voxel p = (x - shift, y, z) sits here at identity;
                // its tissue is at R (p + o_T - c) + c + t
                const int px = x - s.shift;
                if (px >= 0 && px < a.X) {
                    const float q[3] = {(float)x - s.c[0], (float)y - s.c[1], (float)z - s.c[2]};
                    float wt[3];
                    for (int r = 0; r < 3; ++r)
                        wt[r] = s.R[3 * r] * q[0] + s.R[3 * r + 1] * q[1] + s.R[3 * r + 2] * q[2] + s.c[r] + s.t[r];
                    const float ut[3] = {px * inv[0], y * inv[1], z * inv[2]};
                    sum_t += synth_voxel(s, 1, wt, ut);
                    ++cnt_t;
                }
            }
    uint16_t *xo = a.x + ((size_t)b * G * G * G + i) * 2;
    xo[0] = bf16_bits(cnt_s ? sum_s / cnt_s * (1.0f / 64.0f) : 0.0f);
    xo[1] = bf16_bits(cnt_t ? sum_t / cnt_t * (1.0f / 64.0f) : 0.0f);
}

}  // namespace nn

namespace nn {
// Failure-detection self-test: one thread waits on an mbarrier that nothing
// arrives on, with a short bounded wait; when it gives up it sets the error
// flag the host reads (pf_nn_status), exactly as the tensor-core kernels do.
__global__ void k_wait_timeout_selftest(uint32_t polls) {
    __shared__ __align__(8) unsigned long long mbar;
    const uint32_t a = umma::smem_u32(&mbar);
    umma::mbar_init(a, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    bool done = false;
    for (uint32_t i = 0; i < polls && !done; ++i) {
        uint32_t r;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(r)
            : "r"(a), "r"(0u)
            : "memory");
        done = r != 0;
    }
    if (!done) atomicExch(&g_nn_error, 1u);
}
}  // namespace nn

cudaError_t nn_wait_selftest(cudaStream_t s) {
    nn::k_wait_timeout_selftest<<<1, 1, 0, s>>>(1u << 16);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t nn_error_flag(unsigned int *out, bool clear) {
    unsigned int conv = 0, dg = 0;
    cudaError_t e = conv_planes_error_flag(&conv, clear);
    if (e == cudaSuccess) e = dgrad_planes_error_flag(&dg, clear);
    conv |= dg;
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(out, nn::g_nn_error, sizeof(unsigned int));
    if (e != cudaSuccess) return e;
    *out |= conv;
    if (!clear) return e;
    const unsigned int z = 0;
    return cudaMemcpyToSymbol(nn::g_nn_error, &z, sizeof(z));
}

cudaError_t nn_gemm(const uint16_t *A, const uint16_t *B, float *C, int M, int K, cudaStream_t s) {
    nn::GemmOp op{A, B, C, M, K};
#if PF_NN_ASYNC
    return nn::launch_async(op, M, s);
#else
    return nn::launch_tile(op, M, (K + nn::kChunkK - 1) / nn::kChunkK, 1, s);
#endif
}

cudaError_t nn_conv_fwd(const uint16_t *X, int batch, int D, int Cin, const uint16_t *W, const float *bias,
                        uint16_t *Y, cudaStream_t s) {
#if PF_CONV_PLANES
    if (conv_planes_applies(D, Cin)) return conv_planes_forward(X, batch, D, W, bias, Y, s);
    if (conv_c2_applies(D, Cin)) return conv_c2_forward(X, batch, D, W, bias, Y, s);
#endif
    nn::ConvFwdOp op{{batch, D, Cin}, X, W, bias, Y};
    const int Do = D / 2;
#if PF_NN_ASYNC
    return nn::launch_async(op, batch * Do * Do * Do, s);
#else
    return nn::launch_tile(op, batch * Do * Do * Do, (64 * Cin + nn::kChunkK - 1) / nn::kChunkK, 1, s);
#endif
}

cudaError_t nn_conv_dgrad(const uint16_t *dY, int batch, int D, const uint16_t *Wt, const uint16_t *act,
                          uint16_t *dX, cudaStream_t s) {
#if PF_DGRAD_PLANES
    if (dgrad_planes_applies(D)) return dgrad_planes(dY, batch, D, Wt, act, dX, s);
#endif
#if PF_NN_ASYNC && PF_DGRAD_PHASES
    {
        const int Do = D / 2;
        const long long R = (long long)batch * Do * Do * Do;
        const long long Rp = (R + nn::kTileM - 1) / nn::kTileM * nn::kTileM;
        if (8 * Rp > 0x7fffffffLL) return cudaErrorInvalidValue;
        nn::ConvDgradPhaseOp op{{batch, D, 32}, dY, Wt, act, dX, (int)R, (int)Rp};
        return nn::launch_async(op, (int)(8 * Rp), s);
    }
#endif
    nn::ConvDgradOp op{{batch, D, 32}, dY, Wt, act, dX};
#if PF_NN_ASYNC
    return nn::launch_async(op, batch * D * D * D, s);
#else
    return nn::launch_tile(op, batch * D * D * D, 2048 / nn::kChunkK, 1, s);
#endif
}

cudaError_t nn_transpose_w(const uint16_t *W, int Cin, uint16_t *Wt, cudaStream_t s) {
    nn::k_transpose_w<<<64, 256, 0, s>>>(W, Cin, Wt);
    count_launches(1);
    return cudaGetLastError();
}

// SMs of the current device (the K splits of the weight gradient are sized by it).
static int current_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || sms < 1)
        sms = 1;
    return sms;
}

cudaError_t nn_conv_wgrad(const uint16_t *X, int batch, int D, int Cin, const uint16_t *dY, float *dW,
                          cudaStream_t s) {
    const int Do = D / 2;
    const int P = batch * Do * Do * Do;
    const int chunks = (P + nn::kChunkK - 1) / nn::kChunkK;
    const int mtiles = (64 * Cin + nn::kTileM - 1) / nn::kTileM;
    const int sms = current_sms();
    int splits = (4 * sms + mtiles - 1) / mtiles;   // about four CTAs per SM in all
#if PF_WGRAD_PLANES
    if (conv_planes_applies(D, Cin)) return conv_planes_wgrad(X, batch, D, dY, dW, s);
#endif
#if PF_WGRAD_MN
    if (Cin == 32 || Cin == 2) {
        // 32 channels: 16 M tiles of 4 taps; 2 channels: one M tile of all
        // 64 taps; K split for about two CTAs per SM (80 KB of stages each)
        const int mt = Cin == 32 ? 16 : 1;
        int sp = (2 * sms + mt - 1) / mt;
        if (sp > chunks) sp = chunks;
        const int per = (chunks + sp - 1) / sp;
        sp = (chunks + per - 1) / per;
        auto kern = Cin == 32 ? nn::k_wgrad_mn<32> : nn::k_wgrad_mn<2>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, nn::kWgSmem);
        if (e != cudaSuccess) return e;
        const nn::WgradMnArgs g{X, dY, dW, D, P, per};
        kern<<<dim3(mt, (unsigned)sp), 128, nn::kWgSmem, s>>>(g);
        count_launches(1);
        return cudaGetLastError();
    }
#endif
    nn::ConvWgradOp op{{batch, D, Cin}, X, dY, dW, 0};
    return nn::launch_tile(op, 64 * Cin, chunks, splits, s);
}

}  // namespace pfreg

namespace pfreg {

namespace {
unsigned grid_for(long long n, int threads, long long cap = 4096) {
    long long g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}
}  // namespace

#define NNCK(call)                             \
    do {                                       \
        cudaError_t e_ = (call);               \
        if (e_ != cudaSuccess) return e_;      \
    } while (0)
#define NNLAUNCH(n) (count_launches(n), cudaGetLastError())

cudaError_t net_forward(const NetPtrs &n, int B, cudaStream_t s) {
    const uint16_t *in = n.x;
    for (int l = 0; l < 4; ++l) {
        NNCK(nn_conv_fwd(in, B, net_din(l), net_cin(l), n.wbf[l], n.theta + n.L.cb[l], n.a[l], s));
        in = n.a[l];
    }
    const int t = 256;
    nn::k_fc_forward<uint16_t><<<grid_for((long long)B * kNetHidden * 32, t, 1 << 20), t, 0, s>>>(
        n.a[3], B, kNetFlat, n.theta + n.L.f1w, n.theta + n.L.f1b, kNetHidden, n.h, 1);
    NNCK(NNLAUNCH(1));
    nn::k_fc_forward<float><<<grid_for((long long)B * kNetOut * 32, t, 1 << 20), t, 0, s>>>(
        n.h, B, kNetHidden, n.theta + n.L.f2w, n.theta + n.L.f2b, kNetOut, n.out, 0);
    return NNLAUNCH(1);
}

// Gradients of the mean loss over the batch into n.grad (zeroed here) and the
// loss into n.loss[*n.step].
cudaError_t net_backward(const NetPtrs &n, int B, cudaStream_t s) {
    NNCK(cudaMemsetAsync(n.grad, 0, sizeof(float) * n.L.total, s));
    float *g = n.grad;
    const int t = 256;
    nn::k_nll<<<grid_for((long long)B * 6, t), t, 0, s>>>(n.out, n.y, B, n.dout, n.loss, n.step);
    NNCK(NNLAUNCH(1));
    nn::k_fc_backward_weight<float><<<grid_for((long long)kNetOut * kNetHidden, t), t, 0, s>>>(
        n.dout, B, kNetOut, n.h, kNetHidden, g + n.L.f2w, g + n.L.f2b);
    NNCK(NNLAUNCH(1));
    nn::k_fc_backward_input<float, float><<<grid_for((long long)B * kNetHidden, t), t, 0, s>>>(
        n.dout, B, kNetOut, n.theta + n.L.f2w, kNetHidden, n.h, n.dh);
    NNCK(NNLAUNCH(1));
    nn::k_fc_backward_weight<uint16_t><<<grid_for((long long)kNetHidden * kNetFlat, t, 1 << 20), t, 0, s>>>(
        n.dh, B, kNetHidden, n.a[3], kNetFlat, g + n.L.f1w, g + n.L.f1b);
    NNCK(NNLAUNCH(1));
    nn::k_fc_backward_input<uint16_t, uint16_t><<<grid_for((long long)B * kNetFlat, t, 1 << 20), t, 0, s>>>(
        n.dh, B, kNetHidden, n.theta + n.L.f1w, kNetFlat, n.a[3], n.d[3]);
    NNCK(NNLAUNCH(1));
    for (int l = 3; l >= 0; --l) {
        const int D = net_din(l), Do = D / 2;
        const uint16_t *X = l == 0 ? n.x : n.a[l - 1];
        NNCK(nn_conv_wgrad(X, B, D, net_cin(l), n.d[l], g + n.L.cw[l], s));
        const long long rows = (long long)B * Do * Do * Do;
        nn::k_bias_grad<<<grid_for(rows, 8, 1024), 256, 0, s>>>(n.d[l], rows, g + n.L.cb[l]);
        NNCK(NNLAUNCH(1));
        if (l > 0) NNCK(nn_conv_dgrad(n.d[l], B, D, n.wt[l], n.a[l - 1], n.d[l - 1], s));
    }
    return cudaSuccess;
}

cudaError_t net_refresh_bf16(const NetPtrs &n, cudaStream_t s) {
    for (int l = 0; l < 4; ++l) {
        const long long cnt = 32LL * 64 * net_cin(l);
        nn::k_to_bf16<<<grid_for(cnt, 256), 256, 0, s>>>(n.theta + n.L.cw[l], cnt, n.wbf[l]);
        NNCK(NNLAUNCH(1));
        if (l > 0) NNCK(nn_transpose_w(n.wbf[l], net_cin(l), n.wt[l], s));
    }
    return cudaSuccess;
}

cudaError_t net_adam(const NetPtrs &n, float lr, cudaStream_t s) {
    nn::k_adam<<<grid_for(n.L.total, 256, 2048), 256, 0, s>>>(n.theta, n.m, n.v, n.grad, n.L.total, lr, n.step);
    NNCK(NNLAUNCH(1));
    nn::k_step_inc<<<1, 1, 0, s>>>(n.step);
    NNCK(NNLAUNCH(1));
    return net_refresh_bf16(n, s);
}

cudaError_t net_init(const NetPtrs &n, uint64_t seed, cudaStream_t s) {
    NNCK(cudaMemsetAsync(n.theta, 0, sizeof(float) * n.L.total, s));
    NNCK(cudaMemsetAsync(n.m, 0, sizeof(float) * n.L.total, s));
    NNCK(cudaMemsetAsync(n.v, 0, sizeof(float) * n.L.total, s));
    NNCK(cudaMemsetAsync(n.step, 0, sizeof(int), s));
    struct T {
        long long off, cnt;
        int fan_in;
    } ts[6] = {{n.L.cw[0], 32LL * 64 * 2, 64 * 2},      {n.L.cw[1], 32LL * 64 * 32, 64 * 32},
               {n.L.cw[2], 32LL * 64 * 32, 64 * 32},    {n.L.cw[3], 32LL * 64 * 32, 64 * 32},
               {n.L.f1w, (long long)kNetHidden * kNetFlat, kNetFlat}, {n.L.f2w, (long long)kNetOut * kNetHidden, kNetHidden}};
    for (int i = 0; i < 6; ++i) {
        const float a = sqrtf(6.0f / (float)ts[i].fan_in) * (i == 5 ? 0.1f : 1.0f);   // small output layer
        nn::k_init_uniform<<<grid_for(ts[i].cnt, 256), 256, 0, s>>>(n.theta + ts[i].off, ts[i].cnt, a, seed, (uint32_t)i);
        NNCK(NNLAUNCH(1));
    }
    return net_refresh_bf16(n, s);
}

cudaError_t net_synth(const NetPtrs &n, int B, uint64_t seed, int step, float rot_lim, float trans_lim,
                      const int dims[3], bool step_from_counter, cudaStream_t s) {
    nn::SynthArgs a{};
    a.X = dims[0];
    a.Y = dims[1];
    a.Z = dims[2];
    a.G = kNetG;
    a.rot_lim = rot_lim;
    a.trans_lim = trans_lim;
    a.seed = seed;
    a.step = step;
    a.step_ptr = step_from_counter ? n.step : nullptr;
    a.samples = static_cast<nn::SynthSample *>(n.samples);
    a.x = n.x;
    a.y = n.y;
    nn::k_synth_params<<<grid_for(B, 64), 64, 0, s>>>(a, B);
    NNCK(NNLAUNCH(1));
    const int cells = kNetG * kNetG * kNetG;
    nn::k_synth_views<<<dim3((unsigned)((cells + 127) / 128), (unsigned)B), 128, 0, s>>>(a);
    return NNLAUNCH(1);
}

size_t net_sample_bytes() { return sizeof(nn::SynthSample); }

cudaError_t net_downsample(const NetPtrs &n, const uint8_t *vol, const int dims[3], const float origin[3],
                           const float spacing[3], const float box_o[3], const float box_h[3], int channel,
                           cudaStream_t s) {
    nn::DownArgs a{};
    a.vol = vol;
    for (int d = 0; d < 3; ++d) {
        a.dims[d] = dims[d];
        a.origin[d] = origin[d];
        a.spacing[d] = spacing[d];
        a.box_o[d] = box_o[d];
        a.h[d] = box_h[d];
    }
    a.G = kNetG;
    a.c = channel;
    a.x = n.x;
    const int cells = kNetG * kNetG * kNetG;
    nn::k_downsample<<<(cells + 255) / 256, 256, 0, s>>>(a);
    return NNLAUNCH(1);
}

#undef NNCK
#undef NNLAUNCH

}  // namespace pfreg
