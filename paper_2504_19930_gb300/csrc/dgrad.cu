// dgrad.cu -- the data gradient of the proposal network's 32-channel strided
// convolution (kernel 4^3, stride 2, padding 1; the learned proposal of the
// future work named in Sec. 6) on the tcgen05 tensor cores, with each plane
// of the output gradient dY staged once in shared memory.
//
// With stride 2, input voxel i = 2 j + p (p its parity per axis) receives
// dX[i][ci] = sum over t in {0,1}^3 and co of dY[j + p - t][co] W[co][k][ci],
// k = 1 - p + 2 t: per parity class p a stride-1 convolution of dY with
// 2 x 2 x 2 taps.  An output tile is 128 voxels of one class: 8 consecutive
// jx by 16 consecutive jy of one plane jz.  The dY window it reads in a dY
// plane is 9 x 17 voxels (entries (jx + 1 - tx, jy + 1 - ty) for the taps
// (ty, tx)), staged once; a tap is then a view of the window shifted by
// (1 - tx, 1 - ty) entries -- rows = 8 consecutive jx (one core matrix of
// 16-byte rows), row groups = consecutive jy -- which the tensor core reads
// in place through a shared-memory descriptor.  dY plane oz feeds the two
// output planes jz = oz - pz (tz = 0) and oz - pz + 1 (tz = 1) through the
// same views, so one N = 64 MMA against the weight pair (tz = 0, tz = 1)
// updates both.
//
// Shared-memory layouts (no swizzle, K-major, 8-row x 16-byte core matrices):
//   a dY plane, channel chunk c (co 8c .. 8c+7): [wy 17][wx 9][8 co], every
//     2576 bytes (an odd multiple of 16: the producers' stores spread over
//     the banks); the MMA descriptor: LBO (next chunk) = 2576, SBO (next
//     wy) = 144; kBufs plane buffers;
//   the 8 taps of the CTA's class: slot 2 (2 ty + tx) + tz at 2048 bytes
//     each, element (ci, co) at (ci / 8) * 512 + (co / 8) * 128 + (ci % 8) *
//     16 + (co % 8) * 2 (LBO 128, SBO 512), from the transposed weights
//     Wt[ci][tap][co].
//
// One CTA takes kZ consecutive output planes of one (batch, class, tile)
// pencil; their fp32 accumulators live in tensor memory (32 columns each,
// zeroed first).  Warp roles as in the forward kernel: warps 2-5 stage the
// planes and run the epilogue (the ReLU mask of the layer below, bf16),
// warp 1 lane 0 issues the MMAs.  Every mbarrier wait is bounded: when one
// gives up the kernel sets the error flag the host reads (pf_nn_status) and
// leaves cleanly.
#include <cuda_bf16.h>

#include "kernels.h"
#include "nn.h"
#include "umma.cuh"

namespace pfreg {
namespace dgradp {

constexpr int kTileX = 8, kTileY = 16;              // output voxels of a tile (M = 128)
constexpr int kZ = 8;                               // output planes per CTA
constexpr int kWinX = kTileX + 1, kWinY = kTileY + 1;   // dY window: 9 x 17 voxels
constexpr int kChunkPitch = 2576;                   // one channel chunk of the window (2448 bytes used)
constexpr int kPlaneBytes = 4 * kChunkPitch;
constexpr int kBufs = 3;
constexpr int kPieces = kWinX * kWinY * 4;          // 16-byte pieces of one window
constexpr int kProducers = 128;                     // warps 2-5
constexpr int kPerThread = (kPieces + kProducers - 1) / kProducers;   // 5
constexpr int kWeightBytes = 8 * 2048;              // the 8 taps of one class
constexpr int kSmemWeights = 0;
constexpr int kSmemPlanes = kWeightBytes;
constexpr int kSmemBar = kSmemPlanes + kBufs * kPlaneBytes;
constexpr int kSmemTotal = kSmemBar + 128;
constexpr int kThreads = 192;
static_assert(kChunkPitch % 16 == 0 && kPlaneBytes % 16 == 0, "descriptor offsets are in 16-byte units");
static_assert(kSmemTotal < (1 << 18), "shared addresses fit the descriptor's 14-bit field (x 16 bytes)");
constexpr uint32_t kIdesc32 = umma::idesc_bf16_f32(128, 32);
constexpr uint32_t kIdesc64 = umma::idesc_bf16_f32(128, 64);

__device__ unsigned int g_dgrad_error;   // a bounded wait of this kernel gave up

struct Args {
    const uint16_t *dY;    // [batch][Do^3][32 co] bf16
    const uint16_t *Wt;    // [32 ci][64 taps][32 co] bf16
    const uint16_t *act;   // [batch][D^3][32] this layer's input (ReLU output below), or nullptr
    uint16_t *dX;          // [batch][D^3][32 ci] bf16
    int D;
};

// The 8 taps of class (pz, py, px): slot 2 (2 ty + tx) + tz holds tap
// (1 - pz + 2 tz, 1 - py + 2 ty, 1 - px + 2 tx); 16-byte asynchronous copies
// of the groups (ci, tap, 8 co), all in flight.
__device__ __forceinline__ void copy_weights(uint32_t wbase, const uint16_t *__restrict__ Wt, int pz, int py,
                                             int px, int first, int step) {
    for (int g = first; g < 8 * 32 * 4; g += step) {   // g = (slot * 32 + ci) * 4 + cc
        const int cc = g & 3, ci = (g >> 2) & 31, slot = g >> 7;
        const int tz = slot & 1, ty = (slot >> 2) & 1, tx = (slot >> 1) & 1;
        const int tap = ((1 - pz + 2 * tz) * 4 + (1 - py + 2 * ty)) * 4 + (1 - px + 2 * tx);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                         wbase + slot * 2048 + (ci >> 3) * 512 + cc * 128 + (ci & 7) * 16),
                     "l"(reinterpret_cast<const uint4 *>(Wt) + ((size_t)ci * 64 + tap) * 4 + cc)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void tmem_zero32(uint32_t taddr) {
    const uint32_t z = 0u;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
        "r"(z)
        : "memory");
}

// One dY plane oz of the tile's window, by the 128 producer threads: the
// window's 9 x 17 voxels of 64 bytes as 16-byte pieces (four lanes per
// voxel, consecutive voxels along x), piece g = u + 128 k in v[k]; voxels
// outside the grid are zeros.
__device__ __forceinline__ void load_plane(uint4 (&v)[kPerThread], const uint16_t *__restrict__ dY, int Do, int b,
                                           int oz, int ox_lo, int oy_lo, int u) {
    const size_t plane = (((size_t)b * Do + oz) * Do) * Do;
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        const int g = u + k * kProducers;
        v[k] = make_uint4(0u, 0u, 0u, 0u);
        if (g < kPieces) {
            const int vox = g >> 2, c = g & 3;
            const int wy = vox / kWinX, wx = vox - wy * kWinX;
            const int x = ox_lo + wx, y = oy_lo + wy;
            if ((unsigned)x < (unsigned)Do && (unsigned)y < (unsigned)Do)
                v[k] = __ldg(reinterpret_cast<const uint4 *>(dY + (plane + (size_t)y * Do + x) * 32) + c);
        }
    }
}
__device__ __forceinline__ void store_plane(uint8_t *buf, const uint4 (&v)[kPerThread], int u) {
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        const int g = u + k * kProducers;
        if (g < kPieces) {
            const int vox = g >> 2, c = g & 3;
            const int wy = vox / kWinX, wx = vox - wy * kWinX;
            *reinterpret_cast<uint4 *>(buf + c * kChunkPitch + (wy * kWinX + wx) * 16) = v[k];
        }
    }
}

__global__ void __launch_bounds__(kThreads, 1) k_dgrad_planes(const Args p) {
    extern __shared__ __align__(1024) uint8_t sm[];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int D = p.D, Do = D >> 1;
    const int tiles_x = Do / kTileX, tiles_y = Do / kTileY, halves = Do / kZ;
    // this CTA: planes j0 .. j0 + kZ - 1 of pencil (b, class, tile x, tile y)
    int r = blockIdx.x;
    const int j0 = (r % halves) * kZ;
    r /= halves;
    const int ty_t = r % tiles_y;
    r /= tiles_y;
    const int tx_t = r % tiles_x;
    r /= tiles_x;
    const int cls = r % 8, b = r / 8;
    const int px = cls & 1, py = (cls >> 1) & 1, pz = cls >> 2;
    const int jx0 = tx_t * kTileX, jy0 = ty_t * kTileY;
    const int ox_lo = jx0 + px - 1, oy_lo = jy0 + py - 1;
    const int zl = max(j0 + pz - 1, 0), zh = min(j0 + kZ - 1 + pz, Do - 1);
    const int nplanes = zh - zl + 1;
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(sm + kSmemBar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + kSmemBar + 8 * (2 * kBufs + 1));
    const uint32_t full0 = umma::smem_u32(&bars[0]), empty0 = umma::smem_u32(&bars[kBufs]);
    const uint32_t done = umma::smem_u32(&bars[2 * kBufs]);
    const uint32_t planes = umma::smem_u32(sm + kSmemPlanes), wbase = umma::smem_u32(sm + kSmemWeights);

    if (warp == 0) umma::tmem_alloc(tmem_slot, 32 * kZ);
    if (t == 0) {
        for (int i = 0; i < 2 * kBufs + 1; ++i)
            umma::mbar_init(umma::smem_u32(&bars[i]), i < kBufs ? (uint32_t)kProducers : 1u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    copy_weights(wbase, p.Wt, pz, py, px, t, kThreads);
    const int u = t - 64;
    uint4 v[kPerThread];
    if (warp >= 2 && nplanes > 0) load_plane(v, p.dY, Do, b, zl, ox_lo, oy_lo, u);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    umma::fence_async_smem();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    if (warp >= 2) {   // every accumulator starts at zero, so that each MMA accumulates
        for (int q = 0; q < kZ; ++q) tmem_zero32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(32 * q));
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();

    bool ok = true;
    if (warp >= 2) {
        // producers: plane i into buffer i % kBufs once the MMAs of plane
        // i - kBufs are done; make the stores visible to the tensor core,
        // arrive on the buffer's "full" barrier, load plane i + 1
        for (int i = 0; i < nplanes; ++i) {
            const int s = i % kBufs;
            if (i >= kBufs && !umma::mbar_wait(empty0 + 8 * s, (uint32_t)(((i - kBufs) / kBufs) & 1))) {
                ok = false;
                break;
            }
            store_plane(sm + kSmemPlanes + s * kPlaneBytes, v, u);
            umma::fence_async_smem();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(full0 + 8 * s) : "memory");
            if (i + 1 < nplanes) load_plane(v, p.dY, Do, b, zl + i + 1, ox_lo, oy_lo, u);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: descriptors built once (constant offsets below 2^18
        // bytes only add to the 14-bit address field)
        const uint64_t adesc0 = umma::smem_desc(planes, kChunkPitch, kWinX * 16);
        const uint64_t bdesc0 = umma::smem_desc(wbase, 128, 512);
        for (int i = 0; i < nplanes; ++i) {
            const int s = i % kBufs;
            if (!umma::mbar_wait(full0 + 8 * s, (uint32_t)((i / kBufs) & 1))) {
                ok = false;
                break;
            }
            umma::fence_after_sync();
            const int oz = zl + i;
            // dY plane oz feeds output plane qa (tz = 0) and qa + 1 (tz = 1);
            // the weight pair (tz = 0, tz = 1) is one N = 64 operand whose
            // rows 0-31 go to accumulator qa, rows 32-63 to qa + 1
            const int qa = oz - pz - j0, qb = qa + 1;
            const bool va = qa >= 0 && qa < kZ, vb = qb >= 0 && qb < kZ;
            const uint64_t ab = adesc0 + (uint64_t)((s * kPlaneBytes) >> 4);
            const uint32_t dt = tmem + 32 * (va ? qa : qb);
            const uint32_t idesc = (va && vb) ? kIdesc64 : kIdesc32;
            const uint32_t bsel = va ? 0u : 2048u >> 4;   // the tz = 1 tap alone for an edge plane
#pragma unroll
            for (int tq = 0; tq < 4; ++tq) {
                const int tyy = tq >> 1, txx = tq & 1;
                const uint32_t aoff = (((1 - tyy) * kWinX + (1 - txx)) * 16) >> 4;
                const uint64_t bt = bdesc0 + bsel + (uint32_t)((2 * tq * 2048) >> 4);
                umma::mma_bf16(dt, ab + aoff, bt, idesc, true);
                umma::mma_bf16(dt, ab + aoff + (uint32_t)((2 * kChunkPitch) >> 4), bt + (256u >> 4), idesc, true);
            }
            umma::commit(empty0 + 8 * s);
        }
        if (ok) umma::commit(done);
    }
    bool waited = true;
    if (warp >= 2 && ok) waited = umma::mbar_wait(done, 0u);
    const bool all_ok = __syncthreads_and(ok && waited);
    if (all_ok && warp >= 2) {
        umma::fence_after_sync();
        const int wq = warp & 3;
        const int rr = 32 * wq + lane;   // tile row: 8 jx per jy
        const int ix = 2 * (jx0 + (rr & 7)) + px, iy = 2 * (jy0 + (rr >> 3)) + py;
        for (int q = 0; q < kZ; ++q) {
            float acc[32];
            umma::tmem_ld32(tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)(32 * q), acc);
            const int iz = 2 * (j0 + q) + pz;
            const size_t vi = (((size_t)b * D + iz) * D + iy) * D + ix;
            uint32_t mask[16];
            if (p.act) {
                const uint4 *a4 = reinterpret_cast<const uint4 *>(p.act + vi * 32);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint4 w4 = a4[i];
                    mask[4 * i] = w4.x; mask[4 * i + 1] = w4.y; mask[4 * i + 2] = w4.z; mask[4 * i + 3] = w4.w;
                }
            }
            uint32_t packed[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                float a = acc[2 * i], c = acc[2 * i + 1];
                if (p.act) {   // bf16 activations are >= 0 (ReLU): positive iff a nonzero bit pattern
                    a = (mask[i] & 0xFFFFu) ? a : 0.0f;
                    c = (mask[i] >> 16) ? c : 0.0f;
                }
                const __nv_bfloat162 h = __floats2bfloat162_rn(a, c);
                packed[i] = *reinterpret_cast<const uint32_t *>(&h);
            }
            uint4 *dst = reinterpret_cast<uint4 *>(p.dX + vi * 32);
#pragma unroll
            for (int i = 0; i < 4; ++i)
                dst[i] = make_uint4(packed[4 * i], packed[4 * i + 1], packed[4 * i + 2], packed[4 * i + 3]);
        }
    }
    if (!all_ok && t == 0) atomicExch(&g_dgrad_error, 1u);
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_free(tmem, 32 * kZ);
}

}  // namespace dgradp
}  // namespace pfreg

namespace pfreg {

// The plane-staged data gradient applies to inputs whose output edge D / 2 is
// a multiple of 16 (tile 8 x 16, 8 planes per CTA).
bool dgrad_planes_applies(int D) { return D >= 32 && D % 32 == 0 && D <= 512; }

// dX = (conv^T dY) masked by act > 0 for 32 -> 32 channels (see the top of
// this file); dY [batch][(D/2)^3][32], Wt [32][64][32], act / dX
// [batch][D^3][32], bf16; act may be null (no mask).
cudaError_t dgrad_planes(const uint16_t *dY, int batch, int D, const uint16_t *Wt, const uint16_t *act,
                         uint16_t *dX, cudaStream_t s) {
    using namespace dgradp;
    if (!dgrad_planes_applies(D) || batch < 1) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_dgrad_planes, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTotal);
    if (e != cudaSuccess) return e;
    const int Do = D / 2;
    const long long grid = (long long)batch * 8 * (Do / kTileX) * (Do / kTileY) * (Do / kZ);
    if (grid > 0x7FFFFFFF) return cudaErrorInvalidValue;
    const Args a{dY, Wt, act, dX, D};
    k_dgrad_planes<<<(unsigned)grid, kThreads, kSmemTotal, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

// The error flag of the plane-staged data gradient (a bounded wait gave up).
cudaError_t dgrad_planes_error_flag(unsigned int *out, bool clear) {
    cudaError_t e = cudaMemcpyFromSymbol(out, dgradp::g_dgrad_error, sizeof(unsigned int));
    if (e != cudaSuccess || !clear) return e;
    const unsigned int z = 0;
    return cudaMemcpyToSymbol(dgradp::g_dgrad_error, &z, sizeof(z));
}

}  // namespace pfreg
