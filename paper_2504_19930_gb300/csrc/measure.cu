// measure.cu -- the measurement step (Fig. 1 caption: the similarity of the
// source warped by each particle's transform is the particle's measurement).
//
// One work item = (particle p, 32 consecutive target rows), one warp; a warp
// takes a few consecutive items (one particle) and the grid covers all items
// in several waves.  Lane l first finds the exact inside interval of row
// first + l (each coordinate is monotone along a row, so the interval where
// all six bounds hold is found by probing and bisection on the same fp32
// coordinates the samples use); then the warp sweeps the 32 intervals as one
// sequence, lane = x offset, so its gathers follow the rotated row through
// the L2-resident source.  No voxel is tested for inside-ness and the result
// equals the full sweep of the target grid.
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
//
// Debug build (-DPF_DEBUG=1): every gather index is checked against its
// buffer before the load; an index outside sets a device flag, records the
// first bad index and skips the load (the value reads 0) -- nothing traps.
#include "kernels.h"

#ifndef PF_DEBUG
#define PF_DEBUG 0
#endif

namespace pfreg {

namespace {

#if PF_DEBUG
__device__ unsigned long long g_dbg_hits;
__device__ long long g_dbg_first;
// true when idx < limit; otherwise counts the hit, keeps the first bad index
__device__ __forceinline__ bool dbg_ok(unsigned long long idx, unsigned long long limit) {
    if (idx < limit) return true;
    if (atomicAdd(&g_dbg_hits, 1ull) == 0ull) g_dbg_first = (long long)idx;
    return false;
}
#endif

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr float kTwo23 = 8388608.0f;
constexpr uint32_t kTwo23Bits = 0x4B000000u;   // bits of 2^23
constexpr uint32_t k256Bits = 0x43800000u;     // bits of 256.0f

// Per-mode forms of the sweep (each gives the same bits; each mode takes the
// form that timed faster for it):
// paired table (image only): the x-product table holds the products of x and
// x + 32 side by side, so a pass inside one row reads both voxels' products
// as ready-made pairs (the combined kernel, which also gathers mask bits
// through L1, was slower with the larger table);
// crossing without clamp (combined only): the per-row clamp flag is kept
// across passes and a row-crossing pass whose two rows need no y/z clamp
// skips it (the image kernel was slower with it).
#ifndef PF_MEASURE_NNPACK
#define PF_MEASURE_NNPACK 1
#endif
template <bool IMG, bool MASK> __host__ __device__ constexpr bool paired_tab() { return IMG && !MASK; }
template <bool IMG, bool MASK> __host__ __device__ constexpr bool crossing_noclamp() { return IMG && MASK; }
// per-CTA x-product tables (mask and combined modes; see k_measure): the
// combined kernel, whose mask-bit gathers use L1, ran 6.6 % faster with them,
// the image-only kernel 1 % slower
template <bool IMG, bool MASK> __host__ __device__ constexpr bool cta_tab_mode() { return MASK; }

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// 2^23 + byte k of w, as a float (exact).
__device__ __forceinline__ float byte_biased(uint32_t w, uint32_t k) {
    return __uint_as_float(__byte_perm(w, kTwo23Bits, 0x7540u | k));
}


// x as a float for 0 <= x < 2^23 (exact), by an integer add and an fp32
// subtract instead of a conversion instruction.
__device__ __forceinline__ float float_of(int x) {
    return __fsub_rn(__uint_as_float(kTwo23Bits + (uint32_t)x), kTwo23);
}

// Integer value of an integral float v in [0, 2^22).
__device__ __forceinline__ uint32_t int_of(float v) {
    return __float_as_uint(__fadd_rn(v, kTwo23)) - kTwo23Bits;
}

// Packed fp32 pairs (Blackwell f32x2): two independent IEEE round-to-nearest
// operations per instruction, lane-wise identical to __fadd_rn / __fsub_rn /
// __fmaf_rn.  Packed adds and subtracts are used only where no separately
// rounded product feeds them: ptxas fuses a single-use packed multiply into a
// following packed add (one rounding instead of two) even under .rn, so the
// coordinate products (which the arithmetic reading keeps unfused) and the
// adds that consume them stay scalar __fmul_rn / __fadd_rn, which are never
// contracted.  The trilinear lerps are fused by definition (fma2).
struct f2 {
    float x, y;
};
__device__ __forceinline__ f2 pair(float a, float b) { return f2{a, b}; }
__device__ __forceinline__ f2 splat(float a) { return f2{a, a}; }
#ifndef PF_USE_F32X2
#define PF_USE_F32X2 1
#endif
#if PF_USE_F32X2
#define PF_F32X2(NAME, OP)                                                                         \
    __device__ __forceinline__ f2 NAME(f2 a, f2 b) {                                               \
        f2 d;                                                                                      \
        asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2,%3};\n\tmov.b64 rb, {%4,%5};\n\t" OP        \
            ".rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0,%1}, rd;}"                                       \
            : "=f"(d.x), "=f"(d.y)                                                                 \
            : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                                             \
        return d;                                                                                  \
    }
PF_F32X2(add2, "add")
PF_F32X2(sub2, "sub")
#undef PF_F32X2
// a + b rounded toward -infinity, per lane.  With b = 2^23 and 0 <= a < 2^23
// the exact sum lies in [2^23, 2^24), where the floats are the integers, so
// the result is 2^23 + floor(a) exactly.
__device__ __forceinline__ f2 addrm2(f2 a, f2 b) {
    f2 d;
    asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2,%3};\n\tmov.b64 rb, {%4,%5};\n\t"
        "add.rm.f32x2 rd, ra, rb;\n\tmov.b64 {%0,%1}, rd;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
// a*b + c with one rounding per lane (fused, lane-wise identical to
// __fmaf_rn): the trilinear lerps, and the index arithmetic on integer-valued
// operands whose products and sums stay below 2^24 (every rounding exact).
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("{.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2,%3};\n\tmov.b64 rb, {%4,%5};\n\tmov.b64 rc, {%6,%7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0,%1}, rd;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
#else
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return f2{__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)}; }
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return f2{__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y)}; }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    return f2{__fmaf_rn(a.x, b.x, c.x), __fmaf_rn(a.y, b.y, c.y)};
}
__device__ __forceinline__ f2 addrm2(f2 a, f2 b) { return f2{__fadd_rd(a.x, b.x), __fadd_rd(a.y, b.y)}; }
#endif

// a + f*(b - a) for two voxels: the difference rounded, then one fused
// multiply-add (a single rounding of a + f*d).
__device__ __forceinline__ f2 lerp2(f2 a, f2 b, f2 f) { return fma2(f, sub2(b, a), a); }
// the same with biased end points A = 2^23 + a, B = 2^23 + b (a, b bytes, so
// both differences are exact).
__device__ __forceinline__ f2 lerp2_biased(f2 A, f2 B, f2 f) {
    return fma2(f, sub2(B, A), sub2(A, splat(kTwo23)));
}
// q = r*dx + K for two voxels (scalar: a product feeds the add).
__device__ __forceinline__ f2 coord2(float r, f2 dx, f2 K) {
    return f2{__fadd_rn(__fmul_rn(r, dx.x), K.x), __fadd_rn(__fmul_rn(r, dx.y), K.y)};
}

struct ImgAcc {
    uint32_t n = 0, T1 = 0, T2 = 0, S1row = 0;
    unsigned long long S1 = 0, S2 = 0, ST = 0;
};
struct MaskAcc {
    uint32_t n = 0, A = 0, B = 0, C = 0;
};

// Two voxels handed to eval_pair: their x (as floats and as integers, the
// latter indexing the x-product table), the row offsets K of each voxel's
// row and their target indices (in bounds even for a voxel that is not
// taken).
struct PairIn {
    f2 xf;
    int x0, x1;
    f2 K0, K1, K2;
    uint32_t t0, t1;
    // FULL: address of the first voxel's target byte (the second is 32
    // further): image target, or mask target in the mask modes; tpm: the
    // mask target in the combined mode
    const uint8_t *tp, *tpm;
};

// Nearest-neighbour mask sample of one voxel the caller has placed inside
// the source grid (valid: the voxel is taken).
__device__ __forceinline__ void mask_voxel(const MeasureArgs &a, const uint32_t *__restrict__ bits, float qx,
                                           float qy, float qz, const uint8_t *tptr, bool valid, MaskAcc &ma) {
    const int SX = a.g.sd[0], SY = a.g.sd[1];
    const uint32_t SXY = (uint32_t)SX * (uint32_t)SY;
    if (valid) {
        const float hx = __fadd_rn(qx, 0.5f), hy = __fadd_rn(qy, 0.5f), hz = __fadd_rn(qz, 0.5f);
        const uint32_t si = int_of(floorf(hx)) + (uint32_t)SX * int_of(floorf(hy)) + SXY * int_of(floorf(hz));
#if PF_DEBUG
        const bool ok = dbg_ok(si, (unsigned long long)SXY * a.g.sd[2]);
        const uint32_t sb = ok ? (bits[si >> 5] >> (si & 31)) & 1u : 0u;
#else
        const uint32_t sb = (bits[si >> 5] >> (si & 31)) & 1u;
#endif
        const uint32_t tb = __ldg(tptr);
        ma.A += sb;
        ma.B += tb;
        ma.C += sb & tb;
    }
}

// Two voxels of the exact inside intervals the caller visits (no voxel is
// tested here; the overlap counts are added per row by the caller).  valid0 /
// valid1: the voxel is taken (for the mask, and for the image unless
// ivalid0 / ivalid1 say otherwise in the combined mode, whose image interval
// lies inside the mask's).  FULL: both voxels taken for every score, no
// predicates; IFULL: both taken for the image.
// The x base corner is floor(q) unclamped: at q = D-1 it reads the packed
// neighbour byte 0 with fraction 0, a + 0*(0 - a) = a, which equals the
// clamped a' + 1*(b' - a') = b' exactly since the end points are integers
// (y and z keep the clamp: their end points are interpolated values).
// NOCLAMP: the caller knows q_y < D_y - 1 and q_z < D_z - 1 for both voxels,
// where min(floor q, D - 2) = floor q.  FIDX: the source has at most 2^23
// voxels and the quad index is formed in fp32 (exact integers below 2^24)
// as 2^23 + index, read through a base address lowered by 2^23 words.
// XTAB: the products r_i0 * (x - a0) of the particle's matrix come from the
// warp's shared-memory table (the same fp32 roundings, computed once per
// particle), so q = product + K is one packed add per axis.
template <bool IMG, bool MASK, bool FULL, bool IFULL, bool NOCLAMP, bool FIDX, bool XTAB>
__device__ __forceinline__ void eval_pair(const MeasureArgs &a, const uint32_t *__restrict__ bits,
                                          const float4 *__restrict__ tab, const float2 *__restrict__ tabz,
                                          const float r0x, const float r0y, const float r0z, const PairIn &v,
                                          bool valid0, bool valid1, bool ivalid0, bool ivalid1, ImgAcc &ia,
                                          MaskAcc &ma) {
    if (FULL) valid0 = valid1 = true;
    f2 qx, qy, qz;
    if (XTAB) {
        if (paired_tab<IMG, MASK>() && FULL) {
            // entry x holds the products of x and x + 32 (= x1) side by side
            const float4 P = tab[v.x0];
            const float2 Z = tabz[v.x0];
            qx = add2(pair(P.x, P.y), v.K0);
            qy = add2(pair(P.z, P.w), v.K1);
            qz = add2(pair(Z.x, Z.y), v.K2);
        } else if (paired_tab<IMG, MASK>()) {
            const float4 P0 = tab[v.x0], P1 = tab[v.x1];
            const float Z0 = tabz[v.x0].x, Z1 = tabz[v.x1].x;
            qx = add2(pair(P0.x, P1.x), v.K0);
            qy = add2(pair(P0.z, P1.z), v.K1);
            qz = add2(pair(Z0, Z1), v.K2);
        } else {
            const float4 P0 = tab[v.x0], P1 = tab[v.x1];
            qx = add2(pair(P0.x, P1.x), v.K0);
            qy = add2(pair(P0.y, P1.y), v.K1);
            qz = add2(pair(P0.z, P1.z), v.K2);
        }
    } else {
        const f2 dx = sub2(v.xf, splat(a.g.a[0]));
        qx = coord2(r0x, dx, v.K0);
        qy = coord2(r0y, dx, v.K1);
        qz = coord2(r0z, dx, v.K2);
    }
    if (IMG) {
        const int SX = a.g.sd[0], SY = a.g.sd[1], SZ = a.g.sd[2];
        const uint32_t SXY = (uint32_t)SX * (uint32_t)SY;
        const bool in0 = IFULL || (MASK ? ivalid0 : valid0);
        const bool in1 = IFULL || (MASK ? ivalid1 : valid1);
        // base corner min(floor q, D-2) and fraction q - base
        const float Dm2y = a.fdims[2], Dm2z = a.fdims[3];
        // floors by rounding 2^23 + q down, two voxels per instruction (every
        // voxel taken has q >= 0; the others get their index replaced below);
        // bx = 2^23 + floor(qx) is also the biased x term of the quad index
        const f2 bx = addrm2(qx, splat(kTwo23));
        const f2 flx = sub2(bx, splat(kTwo23));
        const f2 fly0 = sub2(addrm2(qy, splat(kTwo23)), splat(kTwo23));
        const f2 flz0 = sub2(addrm2(qz, splat(kTwo23)), splat(kTwo23));
        const f2 fly = NOCLAMP ? fly0 : pair(fminf(fly0.x, Dm2y), fminf(fly0.y, Dm2y));
        const f2 flz = NOCLAMP ? flz0 : pair(fminf(flz0.x, Dm2z), fminf(flz0.y, Dm2z));
        const f2 fx = sub2(qx, flx), fy = sub2(qy, fly), fz = sub2(qz, flz);
        const uint32_t *qbase;
        uint32_t i0, i1;
        if (FIDX) {
            const f2 w = fma2(splat(a.fdims[1]), flz, fma2(splat(a.fdims[0]), fly, bx));
            i0 = __float_as_uint(w.x);
            i1 = __float_as_uint(w.y);
            qbase = reinterpret_cast<const uint32_t *>(reinterpret_cast<uintptr_t>(a.src_quad) -
                                                       (uintptr_t)kTwo23Bits * 4u);
            if (!IFULL) {
                i0 = in0 ? i0 : kTwo23Bits;   // voxels not taken read word 0 and are not accumulated
                i1 = in1 ? i1 : kTwo23Bits;
            }
        } else {
            const uint32_t bias = 0u - kTwo23Bits * (1u + (uint32_t)SX + SXY);   // folds the three int_of
            const f2 bxv = bx, byv = add2(fly, splat(kTwo23)), bzv = add2(flz, splat(kTwo23));
            i0 = __float_as_uint(bxv.x) + (uint32_t)SX * __float_as_uint(byv.x) + SXY * __float_as_uint(bzv.x) + bias;
            i1 = __float_as_uint(bxv.y) + (uint32_t)SX * __float_as_uint(byv.y) + SXY * __float_as_uint(bzv.y) + bias;
            qbase = a.src_quad;
            if (!IFULL) {
                i0 = in0 ? i0 : 0u;   // voxels not taken read word 0 and are not accumulated
                i1 = in1 ? i1 : 0u;
            }
        }
#if PF_DEBUG
        const unsigned long long nq = (unsigned long long)SXY * SZ;
        const unsigned long long ntgt = (unsigned long long)a.g.td[0] * a.g.td[1] * a.g.td[2];
        const uint32_t ioff = FIDX ? kTwo23Bits : 0u;   // the fp32 index is biased by 2^23
        const bool ok0 = dbg_ok((unsigned long long)(uint32_t)(i0 - ioff) + SXY, nq);
        const bool ok1 = dbg_ok((unsigned long long)(uint32_t)(i1 - ioff) + SXY, nq);
        const uint8_t *tp0 = FULL ? v.tp : a.tgt_img + v.t0;
        const uint8_t *tp1 = FULL ? v.tp + 32 : a.tgt_img + v.t1;
        const bool okt0 = dbg_ok((unsigned long long)(tp0 - a.tgt_img), ntgt);
        const bool okt1 = dbg_ok((unsigned long long)(tp1 - a.tgt_img), ntgt);
        const uint32_t w00 = ok0 ? __ldg(qbase + i0) : 0u, w01 = ok0 ? __ldg(qbase + i0 + SXY) : 0u;
        const uint32_t w10 = ok1 ? __ldg(qbase + i1) : 0u, w11 = ok1 ? __ldg(qbase + i1 + SXY) : 0u;
        const uint32_t t0 = okt0 ? __ldg(tp0) : 0u;
        const uint32_t t1 = okt1 ? __ldg(tp1) : 0u;
#else
        const uint32_t w00 = __ldg(qbase + i0), w01 = __ldg(qbase + i0 + SXY);
        const uint32_t w10 = __ldg(qbase + i1), w11 = __ldg(qbase + i1 + SXY);
        const uint32_t t0 = FULL ? __ldg(v.tp) : __ldg(a.tgt_img + v.t0);
        const uint32_t t1 = FULL ? __ldg(v.tp + 32) : __ldg(a.tgt_img + v.t1);
#endif
        const f2 c00 = lerp2_biased(pair(byte_biased(w00, 0), byte_biased(w10, 0)),
                                    pair(byte_biased(w00, 1), byte_biased(w10, 1)), fx);
        const f2 c10 = lerp2_biased(pair(byte_biased(w00, 2), byte_biased(w10, 2)),
                                    pair(byte_biased(w00, 3), byte_biased(w10, 3)), fx);
        const f2 c01 = lerp2_biased(pair(byte_biased(w01, 0), byte_biased(w11, 0)),
                                    pair(byte_biased(w01, 1), byte_biased(w11, 1)), fx);
        const f2 c11 = lerp2_biased(pair(byte_biased(w01, 2), byte_biased(w11, 2)),
                                    pair(byte_biased(w01, 3), byte_biased(w11, 3)), fx);
        const f2 c0 = lerp2(c00, c10, fy), c1 = lerp2(c01, c11, fy);
        const f2 s = add2(lerp2(c0, c1, fz), splat(256.0f));
        const uint32_t sq0 = __float_as_uint(s.x) - k256Bits;   // rint(2^15 s)
        const uint32_t sq1 = __float_as_uint(s.y) - k256Bits;
        if (in0) {
            ia.S1row += sq0;
            ia.S2 += (unsigned long long)sq0 * sq0;
            ia.ST += (unsigned long long)sq0 * t0;
            ia.T1 += t0;
            ia.T2 += t0 * t0;
        }
        if (in1) {
            ia.S1row += sq1;
            ia.S2 += (unsigned long long)sq1 * sq1;
            ia.ST += (unsigned long long)sq1 * t1;
            ia.T1 += t1;
            ia.T2 += t1 * t1;
        }
    }
    if (MASK) {
        const uint8_t *tm = IMG ? v.tpm : v.tp;   // FULL: the mask target's address
#if PF_MEASURE_NNPACK
        // nearest-neighbour voxel floor(q + 0.5) for both voxels at once:
        // h = q + 0.5 (rounded), then 2^23 + floor(h) by a rounding-down add
        // (every voxel taken has h >= 0); the three biases fold into one
        // constant of the integer index
        const int SX = a.g.sd[0], SY = a.g.sd[1];
        const uint32_t SXY = (uint32_t)SX * (uint32_t)SY;
        const f2 bxn = addrm2(add2(qx, splat(0.5f)), splat(kTwo23));
        const f2 byn = addrm2(add2(qy, splat(0.5f)), splat(kTwo23));
        const f2 bzn = addrm2(add2(qz, splat(0.5f)), splat(kTwo23));
        const uint32_t bias = 0u - kTwo23Bits * (1u + (uint32_t)SX + SXY);
#if PF_DEBUG
        const unsigned long long nvx = (unsigned long long)SXY * a.g.sd[2];
        const unsigned long long ntm = (unsigned long long)a.g.td[0] * a.g.td[1] * a.g.td[2];
#endif
        if (valid0) {
            const uint32_t si = __float_as_uint(bxn.x) + (uint32_t)SX * __float_as_uint(byn.x) +
                                SXY * __float_as_uint(bzn.x) + bias;
#if PF_DEBUG
            const uint8_t *tq = FULL ? tm : a.tgt_mask + v.t0;
            const uint32_t sb = dbg_ok(si, nvx) ? (bits[si >> 5] >> (si & 31)) & 1u : 0u;
            const uint32_t tb = dbg_ok((unsigned long long)(tq - a.tgt_mask), ntm) ? __ldg(tq) : 0u;
#else
            const uint32_t sb = (bits[si >> 5] >> (si & 31)) & 1u;
            const uint32_t tb = __ldg(FULL ? tm : a.tgt_mask + v.t0);
#endif
            ma.A += sb;
            ma.B += tb;
            ma.C += sb & tb;
        }
        if (valid1) {
            const uint32_t si = __float_as_uint(bxn.y) + (uint32_t)SX * __float_as_uint(byn.y) +
                                SXY * __float_as_uint(bzn.y) + bias;
#if PF_DEBUG
            const uint8_t *tq = FULL ? tm + 32 : a.tgt_mask + v.t1;
            const uint32_t sb = dbg_ok(si, nvx) ? (bits[si >> 5] >> (si & 31)) & 1u : 0u;
            const uint32_t tb = dbg_ok((unsigned long long)(tq - a.tgt_mask), ntm) ? __ldg(tq) : 0u;
#else
            const uint32_t sb = (bits[si >> 5] >> (si & 31)) & 1u;
            const uint32_t tb = __ldg(FULL ? tm + 32 : a.tgt_mask + v.t1);
#endif
            ma.A += sb;
            ma.B += tb;
            ma.C += sb & tb;
        }
#else
        mask_voxel(a, bits, qx.x, qy.x, qz.x, FULL ? tm : a.tgt_mask + v.t0, valid0, ma);
        mask_voxel(a, bits, qx.y, qy.y, qz.y, FULL ? tm + 32 : a.tgt_mask + v.t1, valid1, ma);
#endif
    }
}

constexpr int kRowsPerWarp = 32;
// consecutive items per warp (one particle, adjacent row blocks): the tile
// shape the autotuner picks; this is the default
constexpr int kItemsPerWarp = kDefaultItemsPerWarp;
__host__ __device__ __forceinline__ int ipw_of(int v) { return v > 0 ? v : kItemsPerWarp; }

// Coordinate q_d(x) of target voxel x of a row (fixed order, no FMA).
__device__ __forceinline__ float coord1(float r, float K, float a0, int x) {
    return __fadd_rn(__fmul_rn(r, __fsub_rn(__int2float_rn(x), a0)), K);
}

// Exact inside interval [xl, xr] of one row, searched within the conservative
// range [xb, xe) that contains it.  Each q_d(x) is monotone in x (rounding is
// monotone), so of the two conditions per axis (lower bound, upper bound) one
// can only turn true as x grows and the other only turn false.  "inc" is the
// conjunction of the first kind, "dec" of the second; the inside set is
// [first x with inc, last x with dec], found by a few linear probes from
// each end and, when those do not reach it, a binary search.  TRI: 0 <= q <= D-1 (trilinear);
// otherwise 0 <= q + 0.5 < D (nearest neighbour).
template <bool TRI>
__device__ __forceinline__ void axis_conds(float q, float D, bool &lower, bool &upper) {
    if (TRI) {
        lower = q >= 0.0f;
        upper = q <= D - 1.0f;
    } else {
        const float h = __fadd_rn(q, 0.5f);
        lower = h >= 0.0f;
        upper = h < D;
    }
}

template <bool TRI>
__device__ __forceinline__ void exact_interval(const float r0[3], const float K[3], float a0, const float D[3],
                                               int xb, int xe, int &xl, int &xr) {
    bool constant_ok = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (r0[d] == 0.0f) {   // q_d does not depend on x
            bool lo, up;
            axis_conds<TRI>(coord1(r0[d], K[d], a0, xb), D[d], lo, up);
            constant_ok &= lo & up;
        }
    }
    auto inc = [&](int x) {
        bool ok = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            bool lo, up;
            axis_conds<TRI>(coord1(r0[d], K[d], a0, x), D[d], lo, up);
            ok &= r0[d] > 0.0f ? lo : (r0[d] < 0.0f ? up : true);
        }
        return ok;
    };
    auto dec = [&](int x) {
        bool ok = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            bool lo, up;
            axis_conds<TRI>(coord1(r0[d], K[d], a0, x), D[d], lo, up);
            ok &= r0[d] > 0.0f ? up : (r0[d] < 0.0f ? lo : true);
        }
        return ok;
    };
    // the conservative ends are usually within a few voxels of the exact
    // ones: probe up to four voxels inward, then fall back to binary search
    int l = xb, cnt = 0;
    while (l < xe && !inc(l)) {
        ++l;
        if (++cnt == 4) break;
    }
    if (cnt == 4 && l < xe) {   // inc(l - 1) is false
        int pl = l - 1;
#pragma unroll 1
        for (int step = 2048; step > 0; step >>= 1)
            if (pl + step < xe && !inc(pl + step)) pl += step;
        l = pl + 1;
    }
    int r = xe - 1;
    cnt = 0;
    while (r >= xb && !dec(r)) {
        --r;
        if (++cnt == 4) break;
    }
    if (cnt == 4 && r >= xb) {  // dec(r + 1) is false
        int pr = xb - 1;
#pragma unroll 1
        for (int step = 2048; step > 0; step >>= 1)
            if (pr + step <= r && dec(pr + step)) pr += step;
        r = pr;
    }
    xl = l;
    xr = constant_ok ? r : xl - 1;
}

// One work item = (particle p, 32 target rows), processed by one warp: lane l
// prepares row (first + l) -- hoisted K, the exact inside interval [vb, ve)
// the row is visited over (nearest-neighbour for the mask modes, trilinear
// for the image mode) and, combined, the trilinear interval [ib, ie) inside
// it -- then the warp sweeps the intervals, reduces the moments and adds
// them to mom[p] with one integer atomic each (S2 is 128-bit).
template <bool IMG, bool MASK, bool FIDX, bool XTAB>
__device__ __forceinline__ void measure_item(const MeasureArgs &a, const uint32_t *__restrict__ bits,
                                             const float4 *__restrict__ tab, const float2 *__restrict__ tabz,
                                             long long item, int lane) {
    constexpr bool BOTH = IMG && MASK;
    const int SX = a.g.sd[0], SY = a.g.sd[1], SZ = a.g.sd[2];
    const int TX = a.g.td[0], TY = a.g.td[1];
    const int rows = a.g.td[1] * a.g.td[2];
    float lo[3], hi[3];
    lo[0] = lo[1] = lo[2] = MASK ? -0.5f : 0.0f;
    hi[0] = MASK ? (float)SX - 0.5f : (float)(SX - 1);
    hi[1] = MASK ? (float)SY - 0.5f : (float)(SY - 1);
    hi[2] = MASK ? (float)SZ - 0.5f : (float)(SZ - 1);
    const float D[3] = {(float)SX, (float)SY, (float)SZ};
    const int nblocks = (rows + kRowsPerWarp - 1) / kRowsPerWarp;

    const int p = (int)(item / nblocks);
    const int rb = (int)(item - (long long)p * nblocks);
    const float *Mp = a.mats + 12 * (size_t)p;
    float M[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) M[i] = __ldg(Mp + i);
    const float r0[3] = {M[0], M[4], M[8]};
    ImgAcc ia;
    MaskAcc ma;

    const int first = rb * kRowsPerWarp;
    const int my_row = first + lane;
    float myK0 = 0.0f, myK1 = 0.0f, myK2 = 0.0f;
    int my_vb = 0, my_ve = 0, my_ib = 0, my_ie = 0;
    bool my_noclamp = false;
    if (my_row < rows) {
        const int y = my_row % TY, z = my_row / TY;
        const float dy = __fsub_rn((float)y, a.g.a[1]);
        const float dz = __fsub_rn((float)z, a.g.a[2]);
        myK0 = row_K(M[1], M[2], M[3], dy, dz);
        myK1 = row_K(M[5], M[6], M[7], dy, dz);
        myK2 = row_K(M[9], M[10], M[11], dy, dz);
        const float K[3] = {myK0, myK1, myK2};
        int xb, xe;
        row_interval(r0, K, a.g.a[0], lo, hi, TX, xb, xe);
        if (xb < xe) {
            int xl, xr;
            exact_interval<!MASK>(r0, K, a.g.a[0], D, xb, xe, xl, xr);
            my_vb = xl;
            my_ve = xr + 1 > xl ? xr + 1 : xl;
            if (BOTH && my_vb < my_ve) {
                // the trilinear inside set lies within the nearest-neighbour one
                exact_interval<true>(r0, K, a.g.a[0], D, my_vb, my_ve, xl, xr);
                my_ib = xl;
                my_ie = xr + 1 > xl ? xr + 1 : xl;
            } else {
                my_ib = my_vb;
                my_ie = my_ve;
            }
            if (IMG && my_ib < my_ie) {
                // q_y, q_z are monotone along the row: below D - 1 at both
                // image interval ends means below it on the whole row
                const int l = my_ib, r = my_ie - 1;
                const float yl = coord1(r0[1], K[1], a.g.a[0], l), yr = coord1(r0[1], K[1], a.g.a[0], r);
                const float zl = coord1(r0[2], K[2], a.g.a[0], l), zr = coord1(r0[2], K[2], a.g.a[0], r);
                my_noclamp = fmaxf(yl, yr) < (float)(SY - 1) && fmaxf(zl, zr) < (float)(SZ - 1);
            }
        }
    }
    // Overlap counts: each lane holds its own row's interval lengths; the warp
    // sums below give the item's counts.
    if (IMG) ia.n = (uint32_t)(my_ie - my_ib);
    if (MASK) ma.n = (uint32_t)(my_ve - my_vb);

    // The rows' visit intervals are swept as one sequence in passes of 64
    // voxels (lane l takes entries l and l + 32): a pass inside one row has
    // no validity predicates; a pass across a row end takes the rest of that
    // row and the start of the next non-empty row.
    uint32_t live = __ballot_sync(0xffffffffu, my_ve > my_vb);
    const uint32_t noclamp = __ballot_sync(0xffffffffu, my_noclamp);
    const uint8_t *tgt = IMG ? a.tgt_img : a.tgt_mask;
    if (live) {
        int j0 = __ffs(live) - 1;
        live &= live - 1;
        int pos = __shfl_sync(0xffffffffu, my_vb, j0), end0 = __shfl_sync(0xffffffffu, my_ve, j0);
        int ib0 = __shfl_sync(0xffffffffu, my_ib, j0), ie0 = __shfl_sync(0xffffffffu, my_ie, j0);
        float K0 = __shfl_sync(0xffffffffu, myK0, j0), K1 = __shfl_sync(0xffffffffu, myK1, j0),
              K2 = __shfl_sync(0xffffffffu, myK2, j0);
        uint32_t trow0 = (uint32_t)(first + j0) * (uint32_t)TX;
        float xf = float_of(pos + lane);
        uint32_t toff = trow0 + (uint32_t)(pos + lane);
        bool nc0 = IMG && ((noclamp >> j0) & 1u);   // row j0 needs no y/z clamp
        for (;;) {
            const int len0 = end0 - pos;
            if (len0 >= 64) {
                const PairIn v{pair(xf, __fadd_rn(xf, 32.0f)), pos + lane, pos + lane + 32, splat(K0), splat(K1),
                               splat(K2), 0u, 0u, tgt + toff, a.tgt_mask + toff};
                const bool nc = crossing_noclamp<IMG, MASK>() ? nc0 : IMG && ((noclamp >> j0) & 1u);
                if (BOTH && !(pos >= ib0 && pos + 64 <= ie0)) {   // the image interval ends in this pass
                    const int x = pos + lane;
                    const bool iv0 = x >= ib0 && x < ie0, iv1 = x + 32 >= ib0 && x + 32 < ie0;
                    if (nc)
                        eval_pair<IMG, MASK, true, false, true, FIDX, XTAB>(a, bits, tab, tabz, r0[0], r0[1], r0[2], v, true, true,
                                                                      iv0, iv1, ia, ma);
                    else
                        eval_pair<IMG, MASK, true, false, false, FIDX, XTAB>(a, bits, tab, tabz, r0[0], r0[1], r0[2], v, true,
                                                                       true, iv0, iv1, ia, ma);
                } else if (nc) {
                    eval_pair<IMG, MASK, true, true, true, FIDX, XTAB>(a, bits, tab, tabz, r0[0], r0[1], r0[2], v, true, true, true,
                                                                 true, ia, ma);
                } else {
                    eval_pair<IMG, MASK, true, true, false, FIDX, XTAB>(a, bits, tab, tabz, r0[0], r0[1], r0[2], v, true, true,
                                                                  true, true, ia, ma);
                }
                pos += 64;
                xf = __fadd_rn(xf, 64.0f);
                toff += 64u;
                continue;
            }
            const bool has1 = live != 0u;
            if (len0 == 0 && !has1) break;
            const int j1 = has1 ? __ffs(live) - 1 : j0;
            const int xb1 = __shfl_sync(0xffffffffu, my_vb, j1), xe1 = __shfl_sync(0xffffffffu, my_ve, j1);
            const int ib1 = __shfl_sync(0xffffffffu, my_ib, j1), ie1 = __shfl_sync(0xffffffffu, my_ie, j1);
            const float L0 = __shfl_sync(0xffffffffu, myK0, j1), L1 = __shfl_sync(0xffffffffu, myK1, j1),
                        L2 = __shfl_sync(0xffffffffu, myK2, j1);
            const int len1 = has1 ? xe1 - xb1 : 0;
            const uint32_t trow1 = (uint32_t)(first + j1) * (uint32_t)TX;
            const int e0 = lane, e1 = lane + 32;          // entries of this pass
            const bool in0a = e0 < len0, in1a = e1 < len0;
            const bool ok0 = in0a || e0 - len0 < len1, ok1 = in1a || e1 - len0 < len1;
            // entries past both rows read voxel 0 of row j0 and are not taken
            const int x0 = in0a ? pos + e0 : (ok0 ? xb1 + e0 - len0 : 0);
            const int x1 = in1a ? pos + e1 : (ok1 ? xb1 + e1 - len0 : 0);
            const bool iv0 = ok0 && (in0a ? x0 >= ib0 && x0 < ie0 : x0 >= ib1 && x0 < ie1);
            const bool iv1 = ok1 && (in1a ? x1 >= ib0 && x1 < ie0 : x1 >= ib1 && x1 < ie1);
            const PairIn v{pair(float_of(x0), float_of(x1)), x0, x1, pair(in0a ? K0 : L0, in1a ? K0 : L0),
                           pair(in0a ? K1 : L1, in1a ? K1 : L1), pair(in0a ? K2 : L2, in1a ? K2 : L2),
                           (in0a || !ok0 ? trow0 : trow1) + (uint32_t)x0,
                           (in1a || !ok1 ? trow0 : trow1) + (uint32_t)x1, nullptr, nullptr};
            // with j1 = j0 when no row follows
            const bool nc1 = IMG && ((noclamp >> j1) & 1u);
            if (crossing_noclamp<IMG, MASK>() && nc0 && nc1)   // both rows' taken voxels need no y/z clamp
                eval_pair<IMG, MASK, false, false, true, FIDX, XTAB>(a, bits, tab, tabz, r0[0], r0[1], r0[2], v, ok0, ok1,
                                                                   iv0, iv1, ia, ma);
            else
                eval_pair<IMG, MASK, false, false, false, FIDX, XTAB>(a, bits, tab, tabz, r0[0], r0[1], r0[2], v, ok0, ok1,
                                                                    iv0, iv1, ia, ma);
            if (IMG) {
                ia.S1 += ia.S1row;
                ia.S1row = 0;
            }
            if (!has1) break;
            live &= live - 1;
            const int used1 = 64 - len0;                  // entries taken from row j1
            if (len1 > used1) {
                j0 = j1;
                pos = xb1 + used1;
                end0 = xe1;
                ib0 = ib1;
                ie0 = ie1;
                K0 = L0;
                K1 = L1;
                K2 = L2;
                trow0 = trow1;
                nc0 = nc1;
            } else {
                if (!live) break;
                j0 = __ffs(live) - 1;
                live &= live - 1;
                pos = __shfl_sync(0xffffffffu, my_vb, j0);
                end0 = __shfl_sync(0xffffffffu, my_ve, j0);
                ib0 = __shfl_sync(0xffffffffu, my_ib, j0);
                ie0 = __shfl_sync(0xffffffffu, my_ie, j0);
                K0 = __shfl_sync(0xffffffffu, myK0, j0);
                K1 = __shfl_sync(0xffffffffu, myK1, j0);
                K2 = __shfl_sync(0xffffffffu, myK2, j0);
                trow0 = (uint32_t)(first + j0) * (uint32_t)TX;
                nc0 = IMG && ((noclamp >> j0) & 1u);
            }
            xf = float_of(pos + lane);
            toff = trow0 + (uint32_t)(pos + lane);
        }
        if (IMG) {
            ia.S1 += ia.S1row;
            ia.S1row = 0;
        }
    }

    // warp reduction and one integer atomic per moment (S2: 128-bit)
    unsigned long long *dst = a.mom + (size_t)p * kMomStride;
    if (IMG) {
        const unsigned long long n = __reduce_add_sync(0xffffffffu, ia.n);
        const unsigned long long S1 = warp_sum64(ia.S1), S2 = warp_sum64(ia.S2), ST = warp_sum64(ia.ST);
        const unsigned long long T1 = warp_sum64(ia.T1), T2 = warp_sum64(ia.T2);
        if (lane == 0 && n) {
            atomicAdd(dst + 0, n);
            atomicAdd(dst + 1, S1);
            const unsigned long long old = atomicAdd(dst + 2, S2);
            if (old + S2 < old) atomicAdd(dst + 3, 1ull);   // carry into S2's high word
            atomicAdd(dst + 4, ST);
            atomicAdd(dst + 5, T1);
            atomicAdd(dst + 6, T2);
        }
    }
    if (MASK) {
        const unsigned long long n = __reduce_add_sync(0xffffffffu, ma.n);
        const unsigned long long A = __reduce_add_sync(0xffffffffu, ma.A);
        const unsigned long long B = __reduce_add_sync(0xffffffffu, ma.B);
        const unsigned long long C = __reduce_add_sync(0xffffffffu, ma.C);
        if (lane == 0 && n) {
            atomicAdd(dst + 8, n);
            if (A) atomicAdd(dst + 9, A);
            if (B) atomicAdd(dst + 10, B);
            if (C) atomicAdd(dst + 11, C);
        }
    }
}

// Measurement kernel of one registration.  Each warp takes kItemsPerWarp
// consecutive items (spatially adjacent rows of one particle) and the grid
// covers all items in several waves, so no block barrier is needed after the
// optional shared-memory load of the mask and finished CTAs are replaced by
// fresh ones.
// Resident CTAs per SM the register allocation must allow: image-only and
// combined 3 (80 registers; 4 CTAs, 64 registers, measured no faster), mask 4.
#ifndef PF_MEASURE_MIN_BLOCKS_IMG
#define PF_MEASURE_MIN_BLOCKS_IMG 3
#endif
#ifndef PF_MEASURE_MIN_BLOCKS_COMBINED
#define PF_MEASURE_MIN_BLOCKS_COMBINED 3
#endif
// XTAB: the table of r_i0 * (x - a0), x = 0 .. X-1, of a particle sits in
// shared memory (X <= kTabMaxX), in front of the optional mask bits: one per
// warp for its current particle, or (CTAB) two per CTA for the particles of
// the CTA's items.  Paired layout: float4 {r_00 dx, r_00 dx', r_10 dx, r_10 dx'} per
// x, then float2 {r_20 dx, r_20 dx'} per x, with dx = x - a0, dx' = x + 32 - a0;
// otherwise float4 {r_00 dx, r_10 dx, r_20 dx, 0} per x.
constexpr int kTabMaxX = 512;
#ifndef PF_MEASURE_XTAB
#define PF_MEASURE_XTAB 1
#endif
// float4 slots of one warp's table (a multiple of 16 bytes)
__host__ __device__ __forceinline__ int tab_slots(int X, bool paired) { return paired ? X + (X + 1) / 2 : X; }

// Table of one particle, same roundings as the per-voxel form: fl(r_i0 * fl(x - a0)),
// entries x = first, first + step, ... written by the calling thread.
template <bool PAIRED>
__device__ __forceinline__ void fill_xtab(float4 *tab, float2 *tabz, int X, float a0, const float *Mp, int first,
                                          int step) {
    const float r0 = __ldg(Mp + 0), r1 = __ldg(Mp + 4), r2 = __ldg(Mp + 8);
    for (int x = first; x < X; x += step) {
        const float dx = __fsub_rn((float)x, a0);
        if (PAIRED) {
            const float dx2 = __fsub_rn((float)(x + 32), a0);
            tab[x] = make_float4(__fmul_rn(r0, dx), __fmul_rn(r0, dx2), __fmul_rn(r1, dx), __fmul_rn(r1, dx2));
            tabz[x] = make_float2(__fmul_rn(r2, dx), __fmul_rn(r2, dx2));
        } else {
            tab[x] = make_float4(__fmul_rn(r0, dx), __fmul_rn(r1, dx), __fmul_rn(r2, dx), 0.0f);
        }
    }
}
// A warp's own table, built by its 32 lanes.
template <bool PAIRED>
__device__ __forceinline__ void build_xtab(float4 *tab, float2 *tabz, int X, float a0, const float *Mp, int lane) {
    __syncwarp();
    fill_xtab<PAIRED>(tab, tabz, X, a0, Mp, lane, 32);
    __syncwarp();
}
// CTAB (with XTAB): the CTA's kWarps * ipw consecutive items are at most
// one particle's item count long (the launch checks it), so they belong to at
// most two particles; the CTA builds those two tables once, together, instead
// of one table per warp (8x less shared memory, which leaves that much more
// of the SM's L1 to the source gathers).
template <bool IMG, bool MASK, bool MASK_SMEM, bool FIDX, bool XTAB, bool CTAB>
__global__ void __launch_bounds__(kThreads, IMG && MASK ? PF_MEASURE_MIN_BLOCKS_COMBINED
                                                        : (IMG ? PF_MEASURE_MIN_BLOCKS_IMG : 4))
    k_measure(const MeasureArgs a) {
    extern __shared__ float4 smem_dyn[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int TX = a.g.td[0];
    constexpr bool PAIRED = paired_tab<IMG, MASK>();
    const int slots = tab_slots(TX, PAIRED);
    const int ntabs = XTAB ? (CTAB ? 2 : kWarps) : 0;
    float4 *tab = XTAB && !CTAB ? smem_dyn + (size_t)warp * slots : nullptr;
    float2 *tabz = XTAB && !CTAB ? reinterpret_cast<float2 *>(tab + TX) : nullptr;
    const int rows = a.g.td[1] * a.g.td[2];
    const int nblocks = (rows + kRowsPerWarp - 1) / kRowsPerWarp;
    const long long items = (long long)a.P * nblocks;
    const int ipw = ipw_of(a.items_per_warp);
    const uint32_t *bits = a.src_bits;
    if (MASK && MASK_SMEM) {
        uint32_t *sb = reinterpret_cast<uint32_t *>(smem_dyn + (size_t)ntabs * slots);
        const int nwords = (int)(((size_t)a.g.sd[0] * a.g.sd[1] * a.g.sd[2] + 31) / 32);
        for (int i = threadIdx.x; i < nwords; i += kThreads) sb[i] = a.src_bits[i];
        bits = sb;
    }
    int p_lo = 0;
    if (XTAB && CTAB) {
        const long long c0 = (long long)blockIdx.x * kWarps * ipw;
        const long long c1 = min(items, c0 + (long long)kWarps * ipw) - 1;
        p_lo = (int)(c0 / nblocks);
        const int p_hi = (int)(c1 / nblocks);
        for (int t = 0; t <= p_hi - p_lo; ++t) {
            float4 *T = smem_dyn + (size_t)t * slots;
            fill_xtab<PAIRED>(T, reinterpret_cast<float2 *>(T + TX), TX, a.g.a[0], a.mats + 12 * (size_t)(p_lo + t),
                              threadIdx.x, kThreads);
        }
    }
    if ((MASK && MASK_SMEM) || (XTAB && CTAB)) __syncthreads();
    const long long item0 = ((long long)blockIdx.x * kWarps + warp) * ipw;
    const long long item1 = min(items, item0 + ipw);
    int tab_p = -1;
    for (long long item = item0; item < item1; ++item) {
        if (XTAB) {
            const int p = (int)(item / nblocks);   // warp-uniform
            if (CTAB) {
                tab = smem_dyn + (size_t)(p - p_lo) * slots;
                tabz = reinterpret_cast<float2 *>(tab + TX);
            } else if (p != tab_p) {
                build_xtab<PAIRED>(tab, tabz, TX, a.g.a[0], a.mats + 12 * (size_t)p, lane);
                tab_p = p;
            }
        }
        measure_item<IMG, MASK, FIDX, XTAB>(a, bits, tab, tabz, item, lane);
    }
}

// Measurement of many registrations in one launch: the items of the listed
// registrations are concatenated (offs = prefix of their item counts); each
// item finds its registration by binary search, and registrations that have
// run all their iterations are skipped.  With tab_x > 0 (every listed
// registration's target rows are at most tab_x <= kTabMaxX long) each warp
// keeps the x-product table of its current (registration, particle) in
// shared memory, as the single-registration kernel does; image sources of at
// most 2^23 voxels take the fp32 quad index.  (A per-warp shared-memory copy
// of the current member's arguments measured slower than reading them
// through the read-only path of the registration table.)
// (The registration lookup costs registers: tighter bounds than these spill.)
template <bool IMG, bool MASK>
__global__ void __launch_bounds__(kThreads, IMG && !MASK ? 3 : 1) k_measure_batch(const BatchReg *__restrict__ regs,
                                                            const int32_t *__restrict__ list,
                                                            const long long *__restrict__ offs, int nlist,
                                                            int ipw, int tab_x) {
    extern __shared__ float4 smem_dyn[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr bool PAIRED = paired_tab<IMG, MASK>();
    float4 *tab = tab_x > 0 ? smem_dyn + (size_t)warp * tab_slots(tab_x, PAIRED) : nullptr;
    const long long total = offs[nlist];
    const long long item0 = ((long long)blockIdx.x * kWarps + warp) * ipw;
    const long long item1 = min(total, item0 + ipw);
    int tab_r = -1, tab_p = -1;
    for (long long item = item0; item < item1; ++item) {
        int lo = 0, hi = nlist - 1;                  // last r with offs[r] <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (offs[mid] <= item) lo = mid; else hi = mid - 1;
        }
        const BatchReg &R = regs[list[lo]];
        if (*R.B.k >= R.n_iters) continue;          // warp-uniform
        const MeasureArgs &A = R.ma;
        const long long local = item - offs[lo];
        const bool fidx = IMG && (size_t)A.g.sd[0] * A.g.sd[1] * A.g.sd[2] <= ((size_t)1 << 23);
        if (tab) {
            const int rows = A.g.td[1] * A.g.td[2];
            const int p = (int)(local / ((rows + kRowsPerWarp - 1) / kRowsPerWarp));   // warp-uniform
            // this member's table: its own row length, in the warp's tab_x slots
            float2 *tabz = reinterpret_cast<float2 *>(tab + A.g.td[0]);
            if (lo != tab_r || p != tab_p) {
                build_xtab<PAIRED>(tab, tabz, A.g.td[0], A.g.a[0], A.mats + 12 * (size_t)p, lane);
                tab_r = lo;
                tab_p = p;
            }
            if (fidx) measure_item<IMG, MASK, true, true>(A, A.src_bits, tab, tabz, local, lane);
            else measure_item<IMG, MASK, false, true>(A, A.src_bits, tab, tabz, local, lane);
        } else {
            if (fidx) measure_item<IMG, MASK, true, false>(A, A.src_bits, nullptr, nullptr, local, lane);
            else measure_item<IMG, MASK, false, false>(A, A.src_bits, nullptr, nullptr, local, lane);
        }
    }
}

template <bool IMG, bool MASK, bool SMEM, bool FIDX, bool XTAB, bool CTAB>
cudaError_t launch_variant(const MeasureArgs &a, size_t smem, cudaStream_t s) {
    auto kern = k_measure<IMG, MASK, SMEM, FIDX, XTAB, CTAB>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int rows = a.g.td[1] * a.g.td[2];
    const long long items = (long long)a.P * ((rows + kRowsPerWarp - 1) / kRowsPerWarp);
    const long long per_cta = (long long)kWarps * ipw_of(a.items_per_warp);
    long long grid = (items + per_cta - 1) / per_cta;
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

// Rows per work item (one warp, 32 rows).  A thread then visits at most
// 2 * ceil(32 X / 64) <= 2048 voxels of one particle per item (X <= 2048), so
// its 32-bit partial sums n, T1 < 2^20 and T2 < 2^27 stay exact; S1 is moved
// to 64 bits after every pass across a row end (in between, the passes of one
// row add < 32 * 2 * 2^23).
int rows_per_item_for(int) { return kRowsPerWarp; }

cudaError_t launch_pack_quads(const uint8_t *src, const int32_t dims[3], uint32_t *quad, cudaStream_t s) {
    const size_t n = (size_t)dims[0] * dims[1] * dims[2];
    unsigned g = (unsigned)((n + 255) / 256);
    if (g > 8192) g = 8192;
    k_pack_quads<<<g, 256, 0, s>>>(src, dims[0], dims[1], dims[2], quad);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_measure_batch(const BatchReg *regs, const int32_t *list, const long long *offs, int nlist,
                                 long long total_items, bool img, bool mask, int items_per_warp, int max_tx,
                                 cudaStream_t s) {
    if (nlist <= 0 || total_items <= 0) return cudaSuccess;
    const int ipw = ipw_of(items_per_warp);
    const long long per_cta = (long long)kWarps * ipw;
    const unsigned grid = (unsigned)((total_items + per_cta - 1) / per_cta);
    const int tab_x = (PF_MEASURE_XTAB && max_tx > 0 && max_tx <= kTabMaxX) ? max_tx : 0;
    const size_t smem = (size_t)kWarps * tab_slots(tab_x, img && !mask) * sizeof(float4);
    auto kern = img && mask ? k_measure_batch<true, true> : (img ? k_measure_batch<true, false> : k_measure_batch<false, true>);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, kThreads, smem, s>>>(regs, list, offs, nlist, ipw, tab_x);
    count_launches(1);
    return cudaGetLastError();
}

long long measure_items(const MeasureArgs &a) {
    const int rows = a.g.td[1] * a.g.td[2];
    return (long long)a.P * ((rows + kRowsPerWarp - 1) / kRowsPerWarp);
}

// The CTA's items span at most two particles when kWarps * items per warp is
// at most one particle's item count; then the CTA shares two tables.
#ifndef PF_MEASURE_CTAB
#define PF_MEASURE_CTAB 1
#endif
bool cta_tables(const MeasureArgs &a) {
    const int rows = a.g.td[1] * a.g.td[2];
    const long long nblocks = (rows + kRowsPerWarp - 1) / kRowsPerWarp;
    return PF_MEASURE_CTAB && (long long)kWarps * ipw_of(a.items_per_warp) <= nblocks;
}

template <bool IMG, bool MASK, bool SMEM, bool FIDX>
cudaError_t launch_tab(const MeasureArgs &a, bool xtab, bool ctab, size_t smem_bits, cudaStream_t s) {
    const size_t tab = (size_t)tab_slots(a.g.td[0], paired_tab<IMG, MASK>()) * sizeof(float4);
    const size_t bits = SMEM ? smem_bits : 0;
    if constexpr (cta_tab_mode<IMG, MASK>())
        if (xtab && ctab) return launch_variant<IMG, MASK, SMEM, FIDX, true, true>(a, 2 * tab + bits, s);
    if (xtab) return launch_variant<IMG, MASK, SMEM, FIDX, true, false>(a, kWarps * tab + bits, s);
    return launch_variant<IMG, MASK, SMEM, FIDX, false, false>(a, bits, s);
}

cudaError_t launch_measure(const MeasureArgs &a, bool img, bool mask, cudaStream_t s) {
    if (a.P <= 0) return cudaSuccess;
    const size_t nvox = (size_t)a.g.sd[0] * a.g.sd[1] * a.g.sd[2];
    const size_t smem_bits = ((nvox + 31) / 32) * 4;
    const bool smem = mask && smem_bits <= 160 * 1024;
    const bool fidx = nvox <= ((size_t)1 << 23);   // quad indices formed in fp32
    const bool ctab = cta_tables(a) && mask;   // cta_tab_mode<img, mask>()
    const size_t tab_bytes = (size_t)(ctab ? 2 : kWarps) * tab_slots(a.g.td[0], img && !mask) * sizeof(float4);
    const bool xtab = PF_MEASURE_XTAB && a.g.td[0] <= kTabMaxX &&
                      tab_bytes + (smem ? smem_bits : 0) <= 200 * 1024;
    if (img && mask) {
        if (smem) return fidx ? launch_tab<true, true, true, true>(a, xtab, ctab, smem_bits, s)
                              : launch_tab<true, true, true, false>(a, xtab, ctab, smem_bits, s);
        return fidx ? launch_tab<true, true, false, true>(a, xtab, ctab, smem_bits, s)
                    : launch_tab<true, true, false, false>(a, xtab, ctab, smem_bits, s);
    }
    if (img) return fidx ? launch_tab<true, false, false, true>(a, xtab, ctab, smem_bits, s)
                         : launch_tab<true, false, false, false>(a, xtab, ctab, smem_bits, s);
    return smem ? launch_tab<false, true, true, false>(a, xtab, ctab, smem_bits, s)
                : launch_tab<false, true, false, false>(a, xtab, ctab, smem_bits, s);
}

// Bounds-check counters of the debug build (all zero otherwise).
cudaError_t measure_debug_bounds(bool clear, unsigned long long *hits, long long *first, bool *on) {
#if PF_DEBUG
    *on = true;
    cudaError_t e = cudaMemcpyFromSymbol(hits, g_dbg_hits, sizeof *hits);
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(first, g_dbg_first, sizeof *first);
    if (e == cudaSuccess && clear) {
        const unsigned long long z = 0;
        const long long zf = 0;
        e = cudaMemcpyToSymbol(g_dbg_hits, &z, sizeof z);
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_dbg_first, &zf, sizeof zf);
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
