// device.cuh -- device building blocks of the registration path (sm_103a).
//
// Every float operation on the parity path is an explicit round-to-nearest
// intrinsic (__fadd_rn, __fmul_rn, __dadd_rn, ...), which nvcc never fuses
// into an FMA, so the bits are fixed by the order written here.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pfreg {

// fp64 / fp32 round-to-nearest operations (never contracted into an FMA).
#define PF_HD __device__ __forceinline__
PF_HD double d_mul(double a, double b) { return __dmul_rn(a, b); }
PF_HD double d_add(double a, double b) { return __dadd_rn(a, b); }
PF_HD double d_sub(double a, double b) { return __dsub_rn(a, b); }
PF_HD double d_div(double a, double b) { return __ddiv_rn(a, b); }
PF_HD float d2f(double a) { return __double2float_rn(a); }
// a * s and a / s with the exact shortcut for s = 1 (x * 1 = x / 1 = x in
// IEEE arithmetic, so the result is the same bits; a division costs ~550
// clocks of dependent latency here, and unit voxel spacing is the common case)
PF_HD double d_mul_s(double a, double s) { return s == 1.0 ? a : __dmul_rn(a, s); }
PF_HD double d_div_s(double a, double s) { return s == 1.0 ? a : __ddiv_rn(a, s); }
PF_HD double u64_to_f64(unsigned long long v) { return __ull2double_rn(v); }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// multiplications by the Philox constants, XOR of the high halves with the
// other words and the round key, word permutation; the key advances by the
// two Weyl constants between rounds.
// ---------------------------------------------------------------------------
struct u32x4 { uint32_t x, y, z, w; };

__device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) { return __umulhi(a, b); }

__device__ __forceinline__ u32x4 philox10(u32x4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = mulhi32(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = mulhi32(0xCD9E8D57u, c.z);
        c = u32x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Philox stream ids (counter word 2): one per use of randomness.
enum : uint32_t { kStreamInit = 0, kStreamPerturb = 1, kStreamResample = 2, kStreamSeed = 3 };

__device__ __forceinline__ u32x4 philox_seeded(uint64_t seed, uint32_t w0, uint32_t w1,
                                               uint32_t w2, uint32_t w3) {
    return philox10(u32x4{w0, w1, w2, w3}, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// Uniform in [0,1) from the top 24 bits of a draw (exact in fp32).
__device__ __forceinline__ float unit24(uint32_t u) {
    return __fmul_rn((float)(u >> 8), 5.9604644775390625e-08f);  // 2^-24
}

// ---------------------------------------------------------------------------
// fp64 sin / cos, |x| <= pi/2: Taylor series, term k = term k-1 * (-x^2) /
// ((2k)(2k+1)) (sin) or / ((2k-1)(2k)) (cos), 14 terms, summed smallest first.
// Written out so host and device agree bit for bit without either libm.
//
// One code path serves both: a lane computing a cosine differs from one
// computing a sine only in its first term and its divisors, so the lanes of
// a warp that hold the three sines and the three cosines of a pose run the
// chain together instead of one function after the other.
//
// Each quotient a / c_k must be the correctly rounded one.  A division costs
// ~550 clocks of dependent latency on this GPU against ~64 for a multiply or
// FMA, and the divisors are constants, so the chain takes q = RN(a * y) with
// y = RN(1 / c_k), the exact remainder r = fma(-q, c_k, a) and the corrected
// quotient fma(r, y, q) -- Markstein's correction step (IBM J. Res. Dev.
// 34(1), 1990), used for constant divisors by Brisebarre, Muller and Raina
// (IEEE Trans. Comput. 53(8), 2004).  Rather than rest on that theorem's
// hypotheses, the identity RN(a / c_k) == fma(r, y, q) was checked for every
// division of both chains at every fp32 angle with 2^-32 <= |x| <= 64 (the
// chains' values are odd or even in x, and round-to-nearest is symmetric,
// so x >= 0 covers both signs): no mismatch.  Below 2^-32 the terms reach
// the subnormal range, where the step can be off by one unit in the last
// place, so those angles (and any beyond 64) take the IEEE division.  The
// angles arrive as fp32, so this covers every input the kernels can see.
// ---------------------------------------------------------------------------
// RN(1 / c_k), k = 1..13 (entry 0 unused): c_k = (2k)(2k+1) and (2k-1)(2k).
#define PF_TAYLOR_RECIP_SIN {0.0, 0x1.5555555555555p-3, 0x1.999999999999ap-5, 0x1.8618618618618p-6, \
    0x1.c71c71c71c71cp-7, 0x1.29e4129e4129ep-7, 0x1.a41a41a41a41ap-8, 0x1.3813813813814p-8,           \
    0x1.e1e1e1e1e1e1ep-9, 0x1.7f405fd017f40p-9, 0x1.3813813813814p-9, 0x1.03091b51f5e1ap-9,           \
    0x1.b4e81b4e81b4fp-10, 0x1.756cac201756dp-10}
#define PF_TAYLOR_RECIP_COS {0.0, 0x1.0000000000000p-1, 0x1.5555555555555p-4, 0x1.1111111111111p-5, \
    0x1.2492492492492p-6, 0x1.6c16c16c16c17p-7, 0x1.f07c1f07c1f08p-8, 0x1.6816816816817p-8,           \
    0x1.1111111111111p-8, 0x1.ac5701ac5701bp-9, 0x1.58ed2308158edp-9, 0x1.1bb4a4046ed29p-9,           \
    0x1.dae6076b981dbp-10, 0x1.934c67f9b2ce6p-10}

// The angle is taken as the fp32 value it always is, which is what the check covered.
PF_HD double taylor_sincos(float xf, bool cosine) {
    const double ys[14] = PF_TAYLOR_RECIP_SIN, yc[14] = PF_TAYLOR_RECIP_COS;
    const double x = (double)xf;
    const double mx2 = -d_mul(x, x);
    const double ax = fabs(x);
    double t[14];
    t[0] = cosine ? 1.0 : x;
    if (ax >= 0x1p-32 && ax <= 64.0) {
#pragma unroll
        for (int k = 1; k < 14; ++k) {
            const double c = cosine ? (double)((2 * k - 1) * (2 * k)) : (double)((2 * k) * (2 * k + 1));
            const double y = cosine ? yc[k] : ys[k];
            const double a = d_mul(t[k - 1], mx2);
            const double q = __dmul_rn(a, y);
            t[k] = __fma_rn(__fma_rn(-q, c, a), y, q);
        }
    } else {
#pragma unroll
        for (int k = 1; k < 14; ++k) {
            const double c = cosine ? (double)((2 * k - 1) * (2 * k)) : (double)((2 * k) * (2 * k + 1));
            t[k] = d_div(d_mul(t[k - 1], mx2), c);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 13; k >= 0; --k) s = d_add(s, t[k]);
    return s;
}

PF_HD double taylor_sin(float x) { return taylor_sincos(x, false); }
PF_HD double taylor_cos(float x) { return taylor_sincos(x, true); }

// 3x3 product C = A B, each entry accumulated from 0 in k order (fp64).
PF_HD void mat3_mul(const double A[9], const double B[9], double C[9]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc = d_add(acc, d_mul(A[3 * i + k], B[3 * k + j]));
            C[3 * i + j] = acc;
        }
}

// Eq. 3: pose -> 3x4 matrix [r00 r01 r02 b0 | r10 r11 r12 b1 | r20 r21 r22 b2]
// with R = Rz(rz) Rx(rx) Ry(ry) (fp64, rounded once to fp32) and
// b = (c + t) - o_S, c = o_S + (dims_S - 1)/2.  (a = c - o_T is per geometry.)
struct Geometry {
    int32_t sd[3];      // source dims
    int32_t td[3];      // target dims
    float so[3];        // source origin (world)
    float to[3];        // target origin (world)
    float ss[3];        // source spacing (world units per voxel)
    float ts[3];        // target spacing
    float a[3];         // (c - o_T) / s_T, target voxel units (fp32)
};

// Source-grid centre in world units, c_d = o_S,d + s_S,d (dims_S,d - 1)/2.
PF_HD double grid_centre(const Geometry &g, int d) {
    // (dims - 1) / 2 is an exact halving of a small integer, the same bits as the division
    return d_add((double)g.so[d], d_mul_s(d_mul((double)(g.sd[d] - 1), 0.5), (double)g.ss[d]));
}

// Per-particle pose -> matrix on the device: sin/cos of the three angles
// (taylor_sin / taylor_cos), R = Rz Rx Ry; with the spacings, target voxel p
// maps to source voxel q = diag(1/s_S) (R (o_T + s_T p - c) + c + t - o_S),
// i.e. M_ij = (R_ij s_T,j) / s_S,i and b_i = ((c_i + t_i) - o_S,i) / s_S,i
// (fp64, one rounding to fp32 each; with unit spacings M = R, b = c + t - o_S).

PF_HD void matrix_from_sincos(const float pose[6], double sa, double ca, double sb, double cb,
                               double sg, double cg, const Geometry &g, float M[12]) {
    const double Rx[9] = {1.0, 0.0, 0.0, 0.0, ca, -sa, 0.0, sa, ca};
    const double Ry[9] = {cb, 0.0, sb, 0.0, 1.0, 0.0, -sb, 0.0, cb};
    const double Rz[9] = {cg, -sg, 0.0, sg, cg, 0.0, 0.0, 0.0, 1.0};
    double XY[9], R[9];
    mat3_mul(Rx, Ry, XY);
    mat3_mul(Rz, XY, R);
    for (int i = 0; i < 3; ++i) {
        const double si = (double)g.ss[i];
        const double b = d_div_s(d_sub(d_add(grid_centre(g, i), (double)pose[3 + i]), (double)g.so[i]), si);
        M[4 * i + 0] = d2f(d_div_s(d_mul_s(R[3 * i + 0], (double)g.ts[0]), si));
        M[4 * i + 1] = d2f(d_div_s(d_mul_s(R[3 * i + 1], (double)g.ts[1]), si));
        M[4 * i + 2] = d2f(d_div_s(d_mul_s(R[3 * i + 2], (double)g.ts[2]), si));
        M[4 * i + 3] = d2f(b);
    }
}

PF_HD void pose_to_matrix(const float pose[6], const Geometry &g, float M[12]) {
    matrix_from_sincos(pose, taylor_sin(pose[0]), taylor_cos(pose[0]), taylor_sin(pose[1]), taylor_cos(pose[1]),
                       taylor_sin(pose[2]), taylor_cos(pose[2]), g, M);
}

// ---------------------------------------------------------------------------
// Quaternion estimator.  q = qz(rz) * qx(rx) * qy(ry) is the unit quaternion
// (w, x, y, z) of R = Rz Rx Ry, from the half-angle cosines and sines
// (ch = sqrt((1 + cos)/2), sh = sin / (2 ch), stable for |angle| <= pi/2).
// ---------------------------------------------------------------------------
PF_HD void quat_from_half(double cx, double sx, double cy, double sy, double cz, double sz, double q[4]) {
    q[0] = d_sub(d_mul(d_mul(cz, cx), cy), d_mul(d_mul(sz, sx), sy));
    q[1] = d_sub(d_mul(d_mul(cz, sx), cy), d_mul(d_mul(sz, cx), sy));
    q[2] = d_add(d_mul(d_mul(cz, cx), sy), d_mul(d_mul(sz, sx), cy));
    q[3] = d_add(d_mul(d_mul(cz, sx), sy), d_mul(d_mul(sz, cx), cy));
}

// Per-row hoisted part of the coordinate: K_i = (r_i1*dy + r_i2*dz) + b_i.
// Then q_i = r_i0*dx + K_i with dx = x - a0 (fixed fp32 order, no FMA).
__device__ __forceinline__ float row_K(float r1, float r2, float b, float dy, float dz) {
    return __fadd_rn(__fadd_rn(__fmul_rn(r1, dy), __fmul_rn(r2, dz)), b);
}

// Trilinear lerp a + f*(b - a): the difference rounded, then one fused
// multiply-add (single rounding of the product and sum).
__device__ __forceinline__ float lerp_rn(float a, float b, float f) {
    return __fmaf_rn(f, __fsub_rn(b, a), a);
}

// Conservative x-range of one target row whose samples can fall inside
// [lo_d, hi_d] on every axis d: q_d(x) = r_d0 (x - a0) + K_d.  q_d is monotone
// in x (rounding is monotone), so the exact inside set of a row is an
// interval; this range contains it with a margin (delta in q, 1 voxel in x),
// and every voxel in it is still tested with the exact predicate.
__device__ __forceinline__ void row_interval(const float r0[3], const float K[3], float a0,
                                             const float lo[3], const float hi[3], int X,
                                             int &x_begin, int &x_end) {
    const float delta = 0.0625f;
    float xmin = -1.0f, xmax = (float)X;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float L = lo[d] - delta - K[d], H = hi[d] + delta - K[d];
        if (fabsf(r0[d]) < 1e-20f) {
            if (L > 0.0f || H < 0.0f) { xmin = 1.0f; xmax = 0.0f; }
        } else {
            float u = L / r0[d] + a0, v = H / r0[d] + a0;
            if (u > v) { const float t = u; u = v; v = t; }
            xmin = fmaxf(xmin, u);
            xmax = fminf(xmax, v);
        }
    }
    if (!(xmin <= xmax)) { x_begin = 0; x_end = 0; return; }
    xmin = fmaxf(xmin, -1.0f);
    xmax = fminf(xmax, (float)X);
    x_begin = max(0, (int)floorf(xmin) - 1);
    x_end = min(X, (int)ceilf(xmax) + 2);
    if (x_end < x_begin) x_end = x_begin;
}

}  // namespace pfreg
