// conv.cu -- the proposal network's 32-channel strided convolution (kernel
// 4^3, stride 2, padding 1, 32 -> 32 channels; the learned proposal of the
// future work named in Sec. 6) on the tcgen05 tensor cores, with each input
// plane staged once in shared memory instead of re-gathered per tap.
//
// An output tile is 128 output voxels: 8 consecutive ox by 16 consecutive oy
// of one output plane oz.  Output voxel o reads input 2o + k - 1 per axis for
// taps k = 0..3, so per axis the taps fall into two parity classes: input
// index 2(o + j) - 1 + s with s = k & 1 and j = k >> 1.  Each input plane z
// of the tile's window is therefore staged as four "parity sub-planes"
// (sy, sx) of 17 x 9 voxels -- entry (jy, jx) = input (2 oy0 + 2 jy - 1 + sy,
// 2 ox0 + 2 jx - 1 + sx), zeros outside the volume.  A tap (ky, kx) is then a
// plain view of one sub-plane shifted by (ky >> 1, kx >> 1) entries: rows =
// 8 consecutive jx (one 8-row core matrix of 16-byte rows), row groups =
// consecutive jy, so the tensor core reads the operand in place through a
// shared-memory descriptor and nothing is re-staged per tap.  An input plane
// feeds two output planes (taps kz and kz + 2) through the same views, so
// one N = 64 MMA against the weight pair (kz + 2, kz) updates both.
//
// Shared-memory layouts (no swizzle, K-major, 8-row x 16-byte core matrices):
//   sub-plane chunk c (channels 8c .. 8c+7): [jy 17][jx 9][8 ch], 2448 bytes,
//     every 2576 bytes (an odd multiple of 16: the producers' stores spread
//     over the banks); the MMA descriptor: LBO (next channel chunk) = 2576,
//     SBO (next jy) = 144;
//   a plane buffer: 4 sub-planes x 4 chunks, two buffers;
//   the weights of all 64 taps, resident for the CTA's lifetime, in pairs
//     (see weight_slot): slot s at 2048 s, element (co, ci) at (co / 8) * 512
//     + (ci / 8) * 128 + (co % 8) * 16 + (ci % 8) * 2 (LBO 128, SBO 512).
//
// One CTA per SM takes a contiguous range of output plane-tiles (at most kZC,
// split into at most two segments where it crosses from one tile's pencil of
// planes to the next), whose fp32 accumulators live in tensor memory (32
// columns each, zeroed first).  Warp roles: warps 2-5 stage the planes
// (coalesced 16-byte loads into registers, stores into the parity layout, a
// proxy fence, an mbarrier arrive; the next plane's loads go out as soon as
// the current one is stored) and run the epilogue (bias, ReLU, bf16) once
// the last MMA has committed; warp 1 lane 0 issues the MMAs from descriptors
// built once.  Every mbarrier wait is bounded: when one gives up the kernel
// sets the error flag the host reads (pf_nn_status) and leaves cleanly.
#include <cuda_bf16.h>

#include "kernels.h"
#include "nn.h"
#include "umma.cuh"

namespace pfreg {
namespace convp {

constexpr int kTileX = 8, kTileY = 16;         // output voxels per tile in x and y (M = 128)
#ifndef PF_CONV_ZC
#define PF_CONV_ZC 8
#endif
constexpr int kZC = PF_CONV_ZC;                 // output planes per CTA (1, 2, 4 or 8)
constexpr int kSubX = kTileX + 1, kSubY = kTileY + 1;   // parity sub-plane extent (entries)
constexpr int kChunkPitch = 2576;                       // its slot (odd multiple of 16: conflict-free stores)
constexpr int kPlaneBytes = 4 * 4 * kChunkPitch;        // 4 sub-planes x 4 chunks
constexpr int kBufs = 2;                                // plane buffers
constexpr int kWinX = 2 * kSubX, kWinY = 2 * kSubY;     // the plane's input window: 18 x 34 voxels
constexpr int kPieces = kWinX * kWinY * 4;              // 16-byte pieces of one plane window
constexpr int kProducers = 128;                         // warps 2-5
constexpr int kWeightBytes = 64 * 32 * 32 * 2;          // all 64 taps, 32 x 32 bf16 each
constexpr int kSmemWeights = 0;
constexpr int kSmemPlanes = kWeightBytes;
constexpr int kSmemBar = kSmemPlanes + kBufs * kPlaneBytes;
constexpr int kSmemTotal = kSmemBar + 128;
constexpr int kThreads = 192;                           // 6 warps
static_assert(kChunkPitch % 16 == 0 && kPlaneBytes % 16 == 0, "descriptor offsets are in 16-byte units");
static_assert(kSmemTotal < (1 << 18), "shared addresses fit the descriptor's 14-bit field (x 16 bytes)");
constexpr uint32_t kIdesc32 = umma::idesc_bf16_f32(128, 32);   // one output plane
constexpr uint32_t kIdesc64 = umma::idesc_bf16_f32(128, 64);   // two output planes at once

__device__ unsigned int g_conv_error;   // a bounded wait of this kernel gave up

struct ConvPlaneArgs {
    const uint16_t *W;   // [32 co][64 taps][32 ci] bf16
    const float *bias;   // [32]
    uint16_t *Y;         // [batch][Do][Do][Do][32] bf16
    int batch, D;
    long long tiles;     // output plane-tiles (b, tile x, tile y, oz), in that order
};

// A CTA's work: a contiguous range of output plane-tiles, at most kZC, split
// where it crosses from one pencil (b, tile x, tile y) to the next into at
// most two segments; segment k covers output planes o0 .. o1 - 1 of its
// pencil, accumulators (tensor-memory slots) sb .. sb + o1 - o0 - 1, and the
// input planes zl .. zh (those of its window inside the volume).
struct Segment {
    int b, ox0, oy0, o0, o1, sb, zl, zh;
};

// All 64 taps' weights into shared memory, in pairs: for the kz parity par
// and the in-plane tap tq = ky * 4 + kx, slot 2 (16 par + tq) holds tap
// (par + 2, tq) and the next slot tap (par, tq), so one N = 64 operand covers
// both output planes an input plane feeds.  Slot s at 2048 s, element
// (co, ci) at (co / 8) * 512 + (ci / 8) * 128 + (co % 8) * 16 + (ci % 8) * 2;
// 16-byte asynchronous copies of the groups (co, tap, 8 ci), all in flight
// (the caller waits for them and fences before the tensor core reads).
__device__ __forceinline__ int weight_slot(int kz, int tq) { return 2 * (16 * (kz & 1) + tq) + 1 - (kz >> 1); }
__device__ __forceinline__ void copy_weights(uint32_t wbase, const uint16_t *__restrict__ W, int first, int step) {
    constexpr int kGroups = 32 * 64 * 4;
    for (int g = first; g < kGroups; g += step) {   // g = (co * 64 + tap) * 4 + cc
        const int cc = g & 3, tap = (g >> 2) & 63, co = g >> 8;
        const int slot = weight_slot(tap >> 4, tap & 15);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                         wbase + slot * 2048 + (co >> 3) * 512 + cc * 128 + (co & 7) * 16),
                     "l"(reinterpret_cast<const uint4 *>(W) + g)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// 32 zero columns into this warp's 32 tensor-memory lanes.
__device__ __forceinline__ void tmem_zero32(uint32_t taddr) {
    const uint32_t z = 0u;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
        "r"(z)
        : "memory");
}

// One input plane z of the tile's window, by the 128 producer threads
// (u = 0..127): the window's 18 x 34 voxels of 64 bytes as 16-byte pieces
// (four lanes per voxel, consecutive voxels along x: coalesced reads), piece
// g = u + 128 k in v[k]; voxels outside the volume are zeros (the padding).
// The producers load the next plane as soon as they have stored the current
// one, so a plane's round trip to L2 overlaps the tensor core's work.
constexpr int kPerThread = (kPieces + kProducers - 1) / kProducers;   // 20
__device__ __forceinline__ void load_plane(uint4 (&v)[kPerThread], const uint16_t *__restrict__ X, int D, int b,
                                           int z, int ox0, int oy0, int u) {
    const int x_lo = 2 * ox0 - 1, y_lo = 2 * oy0 - 1;
    const size_t plane = (((size_t)b * D + z) * D) * D;   // voxel index of (b, z, 0, 0)
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        const int g = u + k * kProducers;
        v[k] = make_uint4(0u, 0u, 0u, 0u);
        if (g < kPieces) {
            const int vox = g >> 2, c = g & 3;
            const int wy = vox / kWinX, wx = vox - wy * kWinX;
            const int x = x_lo + wx, y = y_lo + wy;
            if ((unsigned)x < (unsigned)D && (unsigned)y < (unsigned)D)
                v[k] = __ldg(reinterpret_cast<const uint4 *>(X + (plane + (size_t)y * D + x) * 32) + c);
        }
    }
}
// ... each piece stored at its parity sub-plane, entry and channel chunk.
__device__ __forceinline__ void store_plane(uint8_t *buf, const uint4 (&v)[kPerThread], int u) {
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        const int g = u + k * kProducers;
        if (g < kPieces) {
            const int vox = g >> 2, c = g & 3;
            const int wy = vox / kWinX, wx = vox - wy * kWinX;
            const int sub = (wy & 1) * 2 + (wx & 1);
            *reinterpret_cast<uint4 *>(buf + (sub * 4 + c) * kChunkPitch + ((wy >> 1) * kSubX + (wx >> 1)) * 16) = v[k];
        }
    }
}

__device__ __forceinline__ Segment make_segment(int D, long long t0, long long t1, int sb) {
    const int Do = D >> 1, tiles_x = Do / kTileX, tiles_y = Do / kTileY;
    Segment g;
    const long long pencil = t0 / Do;
    g.o0 = (int)(t0 - pencil * Do);
    g.o1 = g.o0 + (int)(t1 - t0);
    const int ty = (int)(pencil % tiles_y), tx = (int)((pencil / tiles_y) % tiles_x);
    g.b = (int)(pencil / ((long long)tiles_y * tiles_x));
    g.ox0 = tx * kTileX;
    g.oy0 = ty * kTileY;
    g.sb = sb;
    g.zl = max(2 * g.o0 - 1, 0);
    g.zh = min(2 * (g.o1 - 1) + 2, D - 1);
    return g;
}

__global__ void __launch_bounds__(kThreads, 1)
    k_conv_planes(const uint16_t *__restrict__ X, const ConvPlaneArgs p) {
    extern __shared__ __align__(1024) uint8_t sm[];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int D = p.D, Do = D >> 1;
    // this CTA's range of plane-tiles and its (at most two) segments
    const long long t0 = p.tiles * blockIdx.x / gridDim.x, t1 = p.tiles * (blockIdx.x + 1) / gridDim.x;
    const long long cut = min(t1, (t0 / Do + 1) * Do);   // the end of t0's pencil
    Segment sg[2];
    sg[0] = make_segment(p.D, t0, cut, 0);
    const int nseg = cut < t1 ? 2 : 1;
    sg[1] = nseg == 2 ? make_segment(p.D, cut, t1, (int)(cut - t0)) : sg[0];
    const int np0 = sg[0].zh - sg[0].zl + 1;
    const int nplanes = np0 + (nseg == 2 ? sg[1].zh - sg[1].zl + 1 : 0);
    // barriers: full[kBufs] (128 producer arrivals), empty[kBufs], all MMAs done
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(sm + kSmemBar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + kSmemBar + 8 * (2 * kBufs + 1));
    const uint32_t full0 = umma::smem_u32(&bars[0]), empty0 = umma::smem_u32(&bars[kBufs]);
    const uint32_t done = umma::smem_u32(&bars[2 * kBufs]);
    const uint32_t planes = umma::smem_u32(sm + kSmemPlanes), wbase = umma::smem_u32(sm + kSmemWeights);
    // plane i of the CTA's sequence: its segment and z
    auto seg_of = [&](int i) -> const Segment & { return i < np0 ? sg[0] : sg[1]; };
    auto z_of = [&](int i) { return i < np0 ? sg[0].zl + i : sg[1].zl + (i - np0); };
    auto load_i = [&](uint4 (&v)[kPerThread], int i, int u) {
        const Segment &g = seg_of(i);
        load_plane(v, X, D, g.b, z_of(i), g.ox0, g.oy0, u);
    };

    if (warp == 0) umma::tmem_alloc(tmem_slot, 32 * kZC);
    if (t == 0) {
        for (int i = 0; i < 2 * kBufs + 1; ++i)
            umma::mbar_init(umma::smem_u32(&bars[i]), i < kBufs ? (uint32_t)kProducers : 1u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    copy_weights(wbase, p.W, t, kThreads);
    // the producers' first plane loads overlap the weights' copies
    const int u = t - 64;
    uint4 v[kPerThread];
    if (warp >= 2 && nplanes > 0) load_i(v, 0, u);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    umma::fence_async_smem();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    // every accumulator starts at zero, so that each MMA accumulates (a fused
    // MMA updates two output planes, one of which may be fresh)
    if (warp >= 2) {
        for (int q = 0; q < kZC; ++q) tmem_zero32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(32 * q));
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();

    bool ok = true;
    if (warp >= 2) {
        // producers: plane i into buffer i % kBufs once the MMAs of plane
        // i - kBufs are done; then make the stores visible to the tensor core,
        // arrive on the buffer's "full" barrier and load plane i + 1
        for (int i = 0; i < nplanes; ++i) {
            const int s = i % kBufs;
            if (i >= kBufs && !umma::mbar_wait(empty0 + 8 * s, (uint32_t)(((i - kBufs) / kBufs) & 1))) {
                ok = false;
                break;
            }
            store_plane(sm + kSmemPlanes + s * kPlaneBytes, v, u);
            umma::fence_async_smem();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(full0 + 8 * s) : "memory");
            if (i + 1 < nplanes) load_i(v, i + 1, u);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer.  Descriptors are built once: every operand lies at a
        // constant byte offset from buffer 0 / slot 0, and an offset below
        // 2^18 bytes only adds to the descriptor's 14-bit address field
        // (addresses stay below 256 KB, so the field never carries).
        const uint64_t adesc0 = umma::smem_desc(planes, kChunkPitch, kSubX * 16);
        const uint64_t bdesc0 = umma::smem_desc(wbase, 128, 512);
        for (int i = 0; i < nplanes; ++i) {
            const int s = i % kBufs;
            if (!umma::mbar_wait(full0 + 8 * s, (uint32_t)((i / kBufs) & 1))) {
                ok = false;
                break;
            }
            umma::fence_after_sync();
            const Segment &g = seg_of(i);
            const int z = z_of(i), n = g.o1 - g.o0;
            const uint64_t ab = adesc0 + (uint64_t)((s * kPlaneBytes) >> 4);
            // plane z feeds output plane qa through tap kz = par and qa - 1
            // through kz = par + 2: the weight pair (par + 2, par) is one N = 64
            // operand whose rows 0-31 go to accumulator qa - 1, rows 32-63 to qa
            const int par = (z + 1) & 1;
            const int qa = ((z + 1 - par) >> 1) - g.o0, qb = qa - 1;
            const bool va = qa >= 0 && qa < n, vb = qb >= 0 && qb < n;
            const uint64_t bpair = bdesc0 + (uint64_t)((32 * par * 2048) >> 4);
            const uint32_t dt = tmem + 32 * (g.sb + (vb ? qb : qa));
            const uint32_t idesc = (va && vb) ? kIdesc64 : kIdesc32;
            const uint32_t bsel = (va && vb) ? 0u : (va ? 2048u >> 4 : 0u);   // the one tap of an edge plane
#pragma unroll
            for (int tq = 0; tq < 16; ++tq) {
                const int ky = tq >> 2, kx = tq & 3;
                // sub-plane (ky & 1, kx & 1), shifted by (ky >> 1, kx >> 1) entries
                const uint32_t aoff = (((ky & 1) * 2 + (kx & 1)) * 4 * kChunkPitch +
                                       ((ky >> 1) * kSubX + (kx >> 1)) * 16) >> 4;
                const uint64_t bt = bpair + bsel + (uint32_t)((2 * tq * 2048) >> 4);
                umma::mma_bf16(dt, ab + aoff, bt, idesc, true);
                umma::mma_bf16(dt, ab + aoff + (uint32_t)((2 * kChunkPitch) >> 4), bt + (256u >> 4), idesc, true);
            }
            umma::commit(empty0 + 8 * s);   // the buffer is free once these MMAs have read it
        }
        if (ok) umma::commit(done);
    }
    bool waited = true;
    if (warp >= 2 && ok) waited = umma::mbar_wait(done, 0u);
    const bool all_ok = __syncthreads_and(ok && waited);
    if (all_ok && warp >= 2) {
        umma::fence_after_sync();
        const int wq = warp & 3;                 // this warp's tensor-memory lanes 32 wq .. 32 wq + 31
        const int r = 32 * wq + lane;            // tile row: 8 ox per oy
        for (int k = 0; k < nseg; ++k) {
            const Segment &g = sg[k];
            const int ox = g.ox0 + (r & 7), oy = g.oy0 + (r >> 3);
            for (int q = 0; q < g.o1 - g.o0; ++q) {
                float acc[32];
                umma::tmem_ld32(tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)(32 * (g.sb + q)), acc);
                uint32_t packed[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float a = fmaxf(acc[2 * i] + p.bias[2 * i], 0.0f);
                    const float c = fmaxf(acc[2 * i + 1] + p.bias[2 * i + 1], 0.0f);
                    const __nv_bfloat162 hv = __floats2bfloat162_rn(a, c);
                    packed[i] = *reinterpret_cast<const uint32_t *>(&hv);
                }
                const size_t row = (((size_t)g.b * Do + (g.o0 + q)) * Do + oy) * Do + ox;
                uint4 *dst = reinterpret_cast<uint4 *>(p.Y + row * 32);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    dst[i] = make_uint4(packed[4 * i], packed[4 * i + 1], packed[4 * i + 2], packed[4 * i + 3]);
            }
        }
    }
    if (!all_ok && t == 0) atomicExch(&g_conv_error, 1u);
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_free(tmem, 32 * kZC);
}

// ---------------------------------------------------------------------------
// Weight gradient of the same convolution, dW[co][tap][ci] += sum over the
// output positions o of X[2 o + k - 1][ci] dY[o][co], on the same staged
// input planes.  Contracted over positions, both operands are MN-major: in a
// staged sub-plane the 16 bytes of an entry are 8 channels and consecutive
// entries (8 consecutive output x) are 16 bytes apart -- a core matrix of 8
// positions x 8 channels -- and the four parity sub-planes x four channel
// chunks are 16 such groups at the uniform stride 2576: one A operand of
// M = 128 rows (sub-plane, ci) = the four taps (ky, kx) with one in-plane
// shift (ky >> 1, kx >> 1), K = 16 positions (two tile rows, stride 144).
// The dY tiles of the CTA's output plane-tiles are staged once at the start
// as B operands ([co chunk][oy 16][ox 8][8 co], 8 KB each, consecutive), so
// an input plane's two output planes (taps kz = par and par + 2) are one
// N = 64 operand [dY of qa - 1 ; dY of qa].  The accumulators -- 16 blocks
// of 32 columns, one per (shift, kz), all of tensor memory -- sum over every
// position the CTA covers and are added to dW with fp32 atomics at the end.
// ---------------------------------------------------------------------------
constexpr int kWgTile = 4 * kTileY * kTileX * 16;     // one dY tile: 4 chunks x 128 positions x 16 B (8 KB)
constexpr int kWgSmemTiles = 0;
constexpr int kWgSmemPlanes = kZC * kWgTile;           // 64 KB of dY tiles
constexpr int kWgSmemBar = kWgSmemPlanes + kBufs * kPlaneBytes;
constexpr int kWgSmemTotal = kWgSmemBar + 128;
static_assert(kWgSmemTotal <= 232448, "fits the opt-in shared memory of one CTA");
// instruction descriptors: bf16 -> fp32, both operands MN-major (bits 15, 16)
constexpr uint32_t kIdescMN32 = kIdesc32 | (1u << 15) | (1u << 16);
constexpr uint32_t kIdescMN64 = kIdesc64 | (1u << 15) | (1u << 16);

__device__ unsigned int g_wgrad_error;   // a bounded wait of the weight-gradient kernel gave up

struct WgradPlaneArgs {
    const uint16_t *dY;   // [batch][Do][Do][Do][32] bf16
    float *dW;            // [32 co][64 taps][32 ci] fp32, accumulated
    int batch, D;
    long long tiles;      // output plane-tiles (b, tile x, tile y, oz), in that order
};

// Accumulator block of (in-plane shift sh = 2 (ky >> 1) + (kx >> 1), kz):
// the pair (kz = par + 2, kz = par) of one shift is adjacent, in that order,
// so the N = 64 MMA [dY of qa - 1 ; dY of qa] writes both.
__device__ __forceinline__ int wg_block(int sh, int kz) { return (sh * 2 + (kz & 1)) * 2 + 1 - (kz >> 1); }

// The dY tile of output plane-tile (b, oz, ox0, oy0) into slot q: position
// (oy, ox) of chunk c at q * 8 KB + c * 2048 + (oy * 8 + ox) * 16, by 16-byte
// asynchronous copies (thread first, stride step).
__device__ __forceinline__ void copy_dy_tile(uint32_t base, const uint16_t *__restrict__ dY, int Do, int b, int oz,
                                             int ox0, int oy0, int q, int first, int step) {
    for (int g = first; g < 4 * kTileY * kTileX; g += step) {   // g = (oy * 8 + ox) * 4 + c
        const int c = g & 3, pos = g >> 2, ox = pos & 7, oy = pos >> 3;
        const size_t vox = (((size_t)b * Do + oz) * Do + (oy0 + oy)) * Do + (ox0 + ox);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                         base + (uint32_t)(q * kWgTile + c * 2048 + pos * 16)),
                     "l"(reinterpret_cast<const uint4 *>(dY + vox * 32) + c)
                     : "memory");
    }
}

__global__ void __launch_bounds__(kThreads, 1)
    k_wgrad_planes(const uint16_t *__restrict__ X, const WgradPlaneArgs p) {
    extern __shared__ __align__(1024) uint8_t sm[];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int D = p.D, Do = D >> 1;
    const long long t0 = p.tiles * blockIdx.x / gridDim.x, t1 = p.tiles * (blockIdx.x + 1) / gridDim.x;
    const long long cut = min(t1, (t0 / Do + 1) * Do);
    Segment sg[2];
    sg[0] = make_segment(D, t0, cut, 0);
    const int nseg = cut < t1 ? 2 : 1;
    sg[1] = nseg == 2 ? make_segment(D, cut, t1, (int)(cut - t0)) : sg[0];
    const int np0 = sg[0].zh - sg[0].zl + 1;
    const int nplanes = np0 + (nseg == 2 ? sg[1].zh - sg[1].zl + 1 : 0);
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(sm + kWgSmemBar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + kWgSmemBar + 8 * (2 * kBufs + 1));
    const uint32_t full0 = umma::smem_u32(&bars[0]), empty0 = umma::smem_u32(&bars[kBufs]);
    const uint32_t done = umma::smem_u32(&bars[2 * kBufs]);
    const uint32_t planes = umma::smem_u32(sm + kWgSmemPlanes), tiles = umma::smem_u32(sm + kWgSmemTiles);
    auto seg_of = [&](int i) -> const Segment & { return i < np0 ? sg[0] : sg[1]; };
    auto z_of = [&](int i) { return i < np0 ? sg[0].zl + i : sg[1].zl + (i - np0); };

    if (warp == 0) umma::tmem_alloc(tmem_slot, 512);
    if (t == 0) {
        for (int i = 0; i < 2 * kBufs + 1; ++i)
            umma::mbar_init(umma::smem_u32(&bars[i]), i < kBufs ? (uint32_t)kProducers : 1u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the dY tiles of the CTA's plane-tiles, all in flight
    for (int k = 0; k < nseg; ++k) {
        const Segment &g = k ? sg[1] : sg[0];
        for (int q = 0; q < g.o1 - g.o0; ++q)
            copy_dy_tile(tiles, p.dY, Do, g.b, g.o0 + q, g.ox0, g.oy0, g.sb + q, t, kThreads);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    const int u = t - 64;
    uint4 v[kPerThread];
    if (warp >= 2 && nplanes > 0) {
        const Segment &g = seg_of(0);
        load_plane(v, X, D, g.b, z_of(0), g.ox0, g.oy0, u);
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    umma::fence_async_smem();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    if (warp >= 2) {
        for (int q = 0; q < 16; ++q) tmem_zero32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(32 * q));
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();

    bool ok = true;
    if (warp >= 2) {
        for (int i = 0; i < nplanes; ++i) {
            const int s = i % kBufs;
            if (i >= kBufs && !umma::mbar_wait(empty0 + 8 * s, (uint32_t)(((i - kBufs) / kBufs) & 1))) {
                ok = false;
                break;
            }
            store_plane(sm + kWgSmemPlanes + s * kPlaneBytes, v, u);
            umma::fence_async_smem();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(full0 + 8 * s) : "memory");
            if (i + 1 < nplanes) {
                const Segment &g = seg_of(i + 1);
                load_plane(v, X, D, g.b, z_of(i + 1), g.ox0, g.oy0, u);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MN-major descriptors: leading offset = the stride along K
        // (positions: the next tile row), stride offset = the stride along
        // M / N (the next 8 channels)
        const uint64_t adesc0 = umma::smem_desc(planes, kSubX * 16, kChunkPitch);
        const uint64_t bdesc0 = umma::smem_desc(tiles, kTileX * 16, 2048);
        for (int i = 0; i < nplanes; ++i) {
            const int s = i % kBufs;
            if (!umma::mbar_wait(full0 + 8 * s, (uint32_t)((i / kBufs) & 1))) {
                ok = false;
                break;
            }
            umma::fence_after_sync();
            const Segment &g = seg_of(i);
            const int z = z_of(i), n = g.o1 - g.o0;
            // plane z feeds output plane qa through kz = par and qa - 1 through
            // kz = par + 2; dY tiles qa - 1 and qa are consecutive slots
            const int par = (z + 1) & 1;
            const int qa = ((z + 1 - par) >> 1) - g.o0, qb = qa - 1;
            const bool va = qa >= 0 && qa < n, vb = qb >= 0 && qb < n;
            const uint64_t ab = adesc0 + (uint64_t)((s * kPlaneBytes) >> 4);
            const uint64_t bb = bdesc0 + (uint64_t)(((g.sb + (vb ? qb : qa)) * kWgTile) >> 4);
            const uint32_t idesc = (va && vb) ? kIdescMN64 : kIdescMN32;
            const int kz0 = vb ? par + 2 : par;   // the block of the first 32 columns
#pragma unroll
            for (int sh = 0; sh < 4; ++sh) {
                const uint32_t dt = tmem + 32 * wg_block(sh, kz0);
                const uint32_t aoff = (((sh >> 1) * kSubX + (sh & 1)) * 16) >> 4;
#pragma unroll
                for (int ks = 0; ks < 8; ++ks)
                    umma::mma_bf16(dt, ab + aoff + (uint32_t)((2 * ks * kSubX * 16) >> 4),
                                   bb + (uint32_t)((2 * ks * kTileX * 16) >> 4), idesc, true);
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
        const int wq = warp & 3;   // this warp's tensor-memory lanes: rows (sub-plane wq, ci = lane)
        for (int blk = 0; blk < 16; ++blk) {
            float acc[32];
            umma::tmem_ld32(tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)(32 * blk), acc);
            const int sh = blk >> 2, kz = ((blk >> 1) & 1) + 2 * (1 - (blk & 1));
            const int ky = 2 * (sh >> 1) + (wq >> 1), kx = 2 * (sh & 1) + (wq & 1);
            const int tap = (kz * 4 + ky) * 4 + kx;
#pragma unroll
            for (int co = 0; co < 32; ++co)
                if (acc[co] != 0.0f) atomicAdd(p.dW + ((size_t)co * 64 + tap) * 32 + lane, acc[co]);
        }
    }
    if (!all_ok && t == 0) atomicExch(&g_wgrad_error, 1u);
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_free(tmem, 512);
}

// ---------------------------------------------------------------------------
// Forward convolution of the 2-channel first layer.  With two channels the
// four taps kx = 0..3 of one (kz, ky) read four consecutive input voxels,
// 16 contiguous bytes = one 8-element K group.  For each input row y of the
// tile's window an input plane is staged as 8 entries (one per output x of
// the tile), entry ox = the 16 bytes of voxels 2 ox - 1 .. 2 ox + 2 (4-byte
// loads: the run is only 4-byte aligned; voxels outside are zeros): [row
// 34][ox 8][16 B], rows 128 bytes apart.  The A operand of output rows
// (ox, oy) and tap row ky is then entry (2 oy + ky, ox): rows 16 bytes apart
// (a core matrix of 8 ox), row groups (next oy) 256 bytes, K groups (next
// ky) 128 bytes -- one MMA of K = 16 takes the ky pair (2 m, 2 m + 1).  An
// input plane feeds two output planes (kz = par and par + 2): one N = 64
// MMA against the weight pair, as in the 32-channel kernel.
// ---------------------------------------------------------------------------
constexpr int kC2Rows = 2 * kTileY + 2;                 // 34 input rows of the window
constexpr int kC2Plane = kC2Rows * kTileX * 16;         // 4352 bytes
constexpr int kC2Bufs = 4;
constexpr int kC2Pieces = kC2Rows * kTileX * 4;         // 4-byte pieces of one staged plane
constexpr int kC2PerThread = (kC2Pieces + kProducers - 1) / kProducers;   // 9
constexpr int kC2Weights = 4 * 2048;                    // 4 kz slots of 32 co x 32 (ky, kx, ci)
constexpr int kC2SmemWeights = 0;
constexpr int kC2SmemPlanes = kC2Weights;
constexpr int kC2SmemBar = kC2SmemPlanes + kC2Bufs * kC2Plane;
constexpr int kC2SmemTotal = kC2SmemBar + 128;

__device__ unsigned int g_c2_error;   // a bounded wait of the first-layer kernel gave up

struct C2Args {
    const uint16_t *W;   // [32 co][64 taps][2 ci] bf16
    const float *bias;   // [32]
    uint16_t *Y;         // [batch][Do][Do][Do][32] bf16
    int batch, D;
    long long tiles;     // output plane-tiles (b, tile x, tile y, oz), in that order
};

// kz slot: the pair (kz = par + 2, kz = par) at slots 2 par, 2 par + 1;
// element (co, k = (ky 4 + kx) 2 + ci) at slot 2048 + (co / 8) 512 + (k / 8)
// 128 + (co % 8) 16 + (k % 8) 2 (LBO 128, SBO 512).
__device__ __forceinline__ int c2_slot(int kz) { return 2 * (kz & 1) + 1 - (kz >> 1); }
__device__ __forceinline__ void c2_copy_weights(uint32_t wbase, const uint16_t *__restrict__ W, int first,
                                                int step) {
    for (int g = first; g < 32 * 4 * 4; g += step) {   // g = (co * 4 + kz) * 4 + kg
        const int kg = g & 3, kz = (g >> 2) & 3, co = g >> 4;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                         wbase + c2_slot(kz) * 2048 + (co >> 3) * 512 + kg * 128 + (co & 7) * 16),
                     "l"(W + ((size_t)co * 64 + kz * 16) * 2 + kg * 8)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// One input plane z of the window by the 128 producers: piece g = u + 128 k
// = (row, ox, kx) -> voxel (2 ox0 - 1 + 2 ox + kx, 2 oy0 - 1 + row), a
// warp's 32 pieces being one row's 8 entries (coalesced, 72 bytes).
__device__ __forceinline__ void c2_load_plane(uint32_t (&v)[kC2PerThread], const uint16_t *__restrict__ X, int D,
                                              int b, int z, int ox0, int oy0, int u) {
    const size_t plane = (((size_t)b * D + z) * D) * D;
#pragma unroll
    for (int k = 0; k < kC2PerThread; ++k) {
        const int g = u + k * kProducers;
        v[k] = 0u;
        if (g < kC2Pieces) {
            const int kx = g & 3, ox = (g >> 2) & 7, row = g >> 5;
            const int x = 2 * (ox0 + ox) - 1 + kx, y = 2 * oy0 - 1 + row;
            if ((unsigned)x < (unsigned)D && (unsigned)y < (unsigned)D)
                v[k] = __ldg(reinterpret_cast<const uint32_t *>(X + (plane + (size_t)y * D + x) * 2));
        }
    }
}
__device__ __forceinline__ void c2_store_plane(uint8_t *buf, const uint32_t (&v)[kC2PerThread], int u) {
#pragma unroll
    for (int k = 0; k < kC2PerThread; ++k) {
        const int g = u + k * kProducers;
        if (g < kC2Pieces) *reinterpret_cast<uint32_t *>(buf + g * 4) = v[k];   // (row, ox, kx) -> row 128 + ox 16 + kx 4
    }
}

__global__ void __launch_bounds__(kThreads, 1) k_conv_c2(const uint16_t *__restrict__ X, const C2Args p) {
    extern __shared__ __align__(1024) uint8_t sm[];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int D = p.D, Do = D >> 1;
    const long long t0 = p.tiles * blockIdx.x / gridDim.x, t1 = p.tiles * (blockIdx.x + 1) / gridDim.x;
    const long long cut = min(t1, (t0 / Do + 1) * Do);
    Segment sg[2];
    sg[0] = make_segment(D, t0, cut, 0);
    const int nseg = cut < t1 ? 2 : 1;
    sg[1] = nseg == 2 ? make_segment(D, cut, t1, (int)(cut - t0)) : sg[0];
    const int np0 = sg[0].zh - sg[0].zl + 1;
    const int nplanes = np0 + (nseg == 2 ? sg[1].zh - sg[1].zl + 1 : 0);
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(sm + kC2SmemBar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + kC2SmemBar + 8 * (2 * kC2Bufs + 1));
    const uint32_t full0 = umma::smem_u32(&bars[0]), empty0 = umma::smem_u32(&bars[kC2Bufs]);
    const uint32_t done = umma::smem_u32(&bars[2 * kC2Bufs]);
    const uint32_t planes = umma::smem_u32(sm + kC2SmemPlanes), wbase = umma::smem_u32(sm + kC2SmemWeights);
    auto seg_of = [&](int i) -> const Segment & { return i < np0 ? sg[0] : sg[1]; };
    auto z_of = [&](int i) { return i < np0 ? sg[0].zl + i : sg[1].zl + (i - np0); };

    if (warp == 0) umma::tmem_alloc(tmem_slot, 32 * kZC);
    if (t == 0) {
        for (int i = 0; i < 2 * kC2Bufs + 1; ++i)
            umma::mbar_init(umma::smem_u32(&bars[i]), i < kC2Bufs ? (uint32_t)kProducers : 1u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    c2_copy_weights(wbase, p.W, t, kThreads);
    const int u = t - 64;
    uint32_t v[kC2PerThread];
    if (warp >= 2 && nplanes > 0) {
        const Segment &g = seg_of(0);
        c2_load_plane(v, X, D, g.b, z_of(0), g.ox0, g.oy0, u);
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    umma::fence_async_smem();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    if (warp >= 2) {
        for (int q = 0; q < kZC; ++q) tmem_zero32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(32 * q));
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();

    bool ok = true;
    if (warp >= 2) {
        for (int i = 0; i < nplanes; ++i) {
            const int s = i % kC2Bufs;
            if (i >= kC2Bufs && !umma::mbar_wait(empty0 + 8 * s, (uint32_t)(((i - kC2Bufs) / kC2Bufs) & 1))) {
                ok = false;
                break;
            }
            c2_store_plane(sm + kC2SmemPlanes + s * kC2Plane, v, u);
            umma::fence_async_smem();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(full0 + 8 * s) : "memory");
            if (i + 1 < nplanes) {
                const Segment &g = seg_of(i + 1);
                c2_load_plane(v, X, D, g.b, z_of(i + 1), g.ox0, g.oy0, u);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // K-major descriptors: A rows (ox) 16 B apart, LBO 128 (next ky row),
        // SBO 256 (next oy: two input rows); B as in the 32-channel kernel
        const uint64_t adesc0 = umma::smem_desc(planes, kTileX * 16, 2 * kTileX * 16);
        const uint64_t bdesc0 = umma::smem_desc(wbase, 128, 512);
        for (int i = 0; i < nplanes; ++i) {
            const int s = i % kC2Bufs;
            if (!umma::mbar_wait(full0 + 8 * s, (uint32_t)((i / kC2Bufs) & 1))) {
                ok = false;
                break;
            }
            umma::fence_after_sync();
            const Segment &g = seg_of(i);
            const int z = z_of(i), n = g.o1 - g.o0;
            const int par = (z + 1) & 1;
            const int qa = ((z + 1 - par) >> 1) - g.o0, qb = qa - 1;
            const bool va = qa >= 0 && qa < n, vb = qb >= 0 && qb < n;
            const uint64_t ab = adesc0 + (uint64_t)((s * kC2Plane) >> 4);
            const uint64_t bpair = bdesc0 + (uint64_t)((2 * par * 2048) >> 4);
            const uint32_t dt = tmem + 32 * (g.sb + (vb ? qb : qa));
            const uint32_t idesc = (va && vb) ? kIdesc64 : kIdesc32;
            const uint32_t bsel = (va && vb) ? 0u : (va ? 2048u >> 4 : 0u);
#pragma unroll
            for (int m = 0; m < 2; ++m)   // ky pair (2 m, 2 m + 1): rows 2 m .. of the window, K groups 2 m ..
                umma::mma_bf16(dt, ab + (uint32_t)((2 * m * kTileX * 16) >> 4), bpair + bsel + (uint32_t)((2 * m * 128) >> 4),
                               idesc, true);
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
        const int r = 32 * wq + lane;
        for (int k = 0; k < nseg; ++k) {
            const Segment &g = k ? sg[1] : sg[0];
            const int ox = g.ox0 + (r & 7), oy = g.oy0 + (r >> 3);
            for (int q = 0; q < g.o1 - g.o0; ++q) {
                float acc[32];
                umma::tmem_ld32(tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)(32 * (g.sb + q)), acc);
                uint32_t packed[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float a = fmaxf(acc[2 * i] + p.bias[2 * i], 0.0f);
                    const float c = fmaxf(acc[2 * i + 1] + p.bias[2 * i + 1], 0.0f);
                    const __nv_bfloat162 hv = __floats2bfloat162_rn(a, c);
                    packed[i] = *reinterpret_cast<const uint32_t *>(&hv);
                }
                const size_t row = (((size_t)g.b * Do + (g.o0 + q)) * Do + oy) * Do + ox;
                uint4 *dst = reinterpret_cast<uint4 *>(p.Y + row * 32);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    dst[i] = make_uint4(packed[4 * i], packed[4 * i + 1], packed[4 * i + 2], packed[4 * i + 3]);
            }
        }
    }
    if (!all_ok && t == 0) atomicExch(&g_c2_error, 1u);
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_free(tmem, 32 * kZC);
}

}  // namespace convp
}  // namespace pfreg

namespace pfreg {

// The plane-staged forward convolution applies to 32 input channels and
// inputs whose output edge D / 2 is a multiple of 16 (tile 8 x 16, 4 planes
// per CTA).
bool conv_planes_applies(int D, int Cin) { return Cin == 32 && D >= 32 && D % 32 == 0 && D <= 512; }

// y = relu(conv(x, w) + bias) for 32 -> 32 channels (see the top of this
// file); x [batch][D^3][32], w [32][64][32], y [batch][(D/2)^3][32], bf16.
cudaError_t conv_planes_forward(const uint16_t *X, int batch, int D, const uint16_t *W, const float *bias,
                                uint16_t *Y, cudaStream_t s) {
    using namespace convp;
    if (!conv_planes_applies(D, 32) || batch < 1) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_conv_planes, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTotal);
    if (e != cudaSuccess) return e;
    const int Do = D / 2;
    const long long tiles = (long long)batch * (Do / kTileX) * (Do / kTileY) * Do;
    // one CTA per SM, each a contiguous range of plane-tiles (more CTAs only
    // when a range would exceed the kZC accumulators)
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
            sms = 1;
    }
    long long grid = tiles < sms ? tiles : sms;
    if ((tiles + grid - 1) / grid > kZC) grid = (tiles + kZC - 1) / kZC;
    if (grid > 0x7FFFFFFF) return cudaErrorInvalidValue;
    ConvPlaneArgs a{W, bias, Y, batch, D, tiles};
    k_conv_planes<<<(unsigned)grid, kThreads, kSmemTotal, s>>>(X, a);
    count_launches(1);
    return cudaGetLastError();
}

// dW[co][tap][ci] += sum_o X[2 o + k - 1][ci] dY[o][co] for 32 -> 32
// channels (the weight-gradient kernel above); x [batch][D^3][32], dy
// [batch][(D/2)^3][32] bf16, dw [32][64][32] fp32 (accumulated).
cudaError_t conv_planes_wgrad(const uint16_t *X, int batch, int D, const uint16_t *dY, float *dW, cudaStream_t s) {
    using namespace convp;
    if (!conv_planes_applies(D, 32) || batch < 1) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_wgrad_planes, cudaFuncAttributeMaxDynamicSharedMemorySize, kWgSmemTotal);
    if (e != cudaSuccess) return e;
    const int Do = D / 2;
    const long long tiles = (long long)batch * (Do / kTileX) * (Do / kTileY) * Do;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        sms = 1;
    long long grid = tiles < sms ? tiles : sms;
    if ((tiles + grid - 1) / grid > kZC) grid = (tiles + kZC - 1) / kZC;
    if (grid > 0x7FFFFFFF) return cudaErrorInvalidValue;
    const WgradPlaneArgs a{dY, dW, batch, D, tiles};
    k_wgrad_planes<<<(unsigned)grid, kThreads, kWgSmemTotal, s>>>(X, a);
    count_launches(1);
    return cudaGetLastError();
}

// The first layer's forward convolution (2 -> 32 channels; the kernel
// above) applies to inputs whose output edge is a multiple of 16.
bool conv_c2_applies(int D, int Cin) { return Cin == 2 && D >= 32 && D % 32 == 0 && D <= 512; }

// y = relu(conv(x, w) + bias) for 2 -> 32 channels; x [batch][D^3][2],
// w [32][64][2], y [batch][(D/2)^3][32], bf16.
cudaError_t conv_c2_forward(const uint16_t *X, int batch, int D, const uint16_t *W, const float *bias, uint16_t *Y,
                            cudaStream_t s) {
    using namespace convp;
    if (!conv_c2_applies(D, 2) || batch < 1) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_conv_c2, cudaFuncAttributeMaxDynamicSharedMemorySize, kC2SmemTotal);
    if (e != cudaSuccess) return e;
    const int Do = D / 2;
    const long long tiles = (long long)batch * (Do / kTileX) * (Do / kTileY) * Do;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        sms = 1;
    // two CTAs per SM (256 tensor-memory columns each), ranges of at most kZC plane-tiles
    long long grid = tiles < 2LL * sms ? tiles : 2LL * sms;
    if ((tiles + grid - 1) / grid > kZC) grid = (tiles + kZC - 1) / kZC;
    if (grid > 0x7FFFFFFF) return cudaErrorInvalidValue;
    const C2Args a{W, bias, Y, batch, D, tiles};
    k_conv_c2<<<(unsigned)grid, kThreads, kC2SmemTotal, s>>>(X, a);
    count_launches(1);
    return cudaGetLastError();
}

// The error flags of the plane-staged kernels (a bounded wait gave up).
cudaError_t conv_planes_error_flag(unsigned int *out, bool clear) {
    unsigned int f = 0, w = 0, c2 = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&f, convp::g_conv_error, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&w, convp::g_wgrad_error, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&c2, convp::g_c2_error, sizeof(unsigned int));
    if (e != cudaSuccess) return e;
    *out = f | w | c2;
    if (!clear) return e;
    const unsigned int z = 0;
    e = cudaMemcpyToSymbol(convp::g_conv_error, &z, sizeof(z));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(convp::g_wgrad_error, &z, sizeof(z));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(convp::g_c2_error, &z, sizeof(z));
    return e;
}

}  // namespace pfreg
