/*
 * pf_oracle.c -- plain, slow, single-threaded CPU oracle for the particle
 * filter (sequential Monte Carlo) 3D-3D rigid registration hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA path; both follow the same written
 * readings of the paper (listed at each function).
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, so every
 * float expression below is the sequence of IEEE-754 round-to-nearest
 * operations it spells, evaluated left to right).
 *
 * What the paper fixes and what is a reading:
 *   - Eq. 1 (Sec. 3.1): registration = the rigid map that best matches the
 *     resampled source to the target.
 *   - Eq. 3 (Sec. 3.3): the rigid map is [R t; 0 1] from an Euler-3D
 *     rotation (rx, ry, rz) and a translation (tx, ty, tz).  Reading: R =
 *     Rz Rx Ry (the Euler-3D default order), about the source grid centre.
 *   - Eq. 2 (Sec. 3.3): NCC = squared correlation over the compared voxels.
 *   - Eq. 4 (Sec. 3.4): DSC = 2|S n T| / (|S| + |T|).
 *   - Fig. 1 caption: particles x^i, weights w^i, measurements z^i; the
 *     prediction / measurement / update / resampling / estimation cycle.  The
 *     particle count, likelihood, resampling scheme, noise and estimator are
 *     not printed; the readings used here are stated at each step.
 *   - Sec. 3.3: trilinear interpolation for images; masks use
 *     nearest-neighbour sampling (reading).
 *
 * Volumes are uint8, x fastest: index = x + X*(y + Y*z).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------ */
/* Counter-based RNG: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel   */
/* random numbers: as easy as 1, 2, 3", SC'11).  Ten rounds; each round      */
/* multiplies words 0 and 2 by the two Philox multipliers, XORs the high     */
/* halves with the other two words and the round key, and permutes; the key  */
/* advances by the two Weyl constants between rounds.                        */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Stream identifiers in counter word 2 (reading: one Philox stream per use). */
enum { ORC_STREAM_INIT = 0, ORC_STREAM_PERTURB = 1, ORC_STREAM_RESAMPLE = 2, ORC_STREAM_SEED = 3 };

static void philox_seeded(uint64_t seed, uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3,
                          uint32_t out[4])
{
    uint32_t ctr[4] = {w0, w1, w2, w3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* A uniform in [0, 1) from the top 24 bits of a 32-bit draw (exact in fp32). */
static float unit24(uint32_t u)
{
    return (float)(u >> 8) * 0x1p-24f;
}

/* ------------------------------------------------------------------------ */
/* sin / cos in fp64 by their Taylor series (|x| <= pi/2): term k is term     */
/* k-1 times -x^2 / ((2k)(2k+1)) for sin and / ((2k-1)(2k)) for cos; 14      */
/* terms (through x^27 / x^26) summed from the smallest up.  Written out so  */
/* the CPU and GPU produce the same bits without relying on either libm.     */
/* ------------------------------------------------------------------------ */
double orc_sin(double x)
{
    double x2 = x * x;
    double t[14];
    t[0] = x;
    for (int k = 1; k < 14; ++k)
        t[k] = (t[k - 1] * (-x2)) / (double)((2 * k) * (2 * k + 1));
    double s = 0.0;
    for (int k = 13; k >= 0; --k) s = s + t[k];
    return s;
}

double orc_cos(double x)
{
    double x2 = x * x;
    double t[14];
    t[0] = 1.0;
    for (int k = 1; k < 14; ++k)
        t[k] = (t[k - 1] * (-x2)) / (double)((2 * k - 1) * (2 * k));
    double s = 0.0;
    for (int k = 13; k >= 0; --k) s = s + t[k];
    return s;
}

/* ------------------------------------------------------------------------ */
/* Pose -> 3x4 matrix (Eq. 3).  R = Rz(rz) * Rx(rx) * Ry(ry) by two plain    */
/* 3x3 products in fp64.  World positions (the Euler transform of Sec. 3.3   */
/* acts in physical space; Table 1 gives the voxel sizes): target voxel p    */
/* sits at w = o_T + s_T p; it maps to R (w - c) + c + t, which is source    */
/* voxel q = (R (w - c) + c + t - o_S) / s_S, so                             */
/*     q = M3 (p - a) + b,   M3_ij = (R_ij s_T,j) / s_S,i,                   */
/*     a = (c - o_T) / s_T,  b = ((c + t) - o_S) / s_S,                      */
/* c = o_S + s_S (dims_S - 1)/2 the source grid centre (reading: the         */
/* rotation centre), each entry computed in fp64 and rounded once to fp32.   */
/* With unit spacings M3 = R, a = c - o_T, b = c + t - o_S.                  */
/* M holds [r00 r01 r02 b0 | r10 r11 r12 b1 | r20 r21 r22 b2].               */
/* ------------------------------------------------------------------------ */
static void matmul3(const double A[3][3], const double B[3][3], double C[3][3])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc = acc + A[i][k] * B[k][j];
            C[i][j] = acc;
        }
}

void orc_rotation(const float pose[6], double R[9])
{
    double ax = (double)pose[0], ay = (double)pose[1], az = (double)pose[2];
    double sa = orc_sin(ax), ca = orc_cos(ax);
    double sb = orc_sin(ay), cb = orc_cos(ay);
    double sg = orc_sin(az), cg = orc_cos(az);
    double Rx[3][3] = {{1.0, 0.0, 0.0}, {0.0, ca, -sa}, {0.0, sa, ca}};
    double Ry[3][3] = {{cb, 0.0, sb}, {0.0, 1.0, 0.0}, {-sb, 0.0, cb}};
    double Rz[3][3] = {{cg, -sg, 0.0}, {sg, cg, 0.0}, {0.0, 0.0, 1.0}};
    double XY[3][3], Rm[3][3];
    matmul3(Rx, Ry, XY);
    matmul3(Rz, XY, Rm);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) R[3 * i + j] = Rm[i][j];
}

/* sspacing / tspacing may be NULL (unit spacing). */
void orc_pose_matrix_sp(const float pose[6], const int32_t sdims[3], const float sorigin[3],
                        const float sspacing[3], const float torigin[3], const float tspacing[3],
                        float M[12], float a[3])
{
    double R[9], ss[3], ts[3];
    orc_rotation(pose, R);
    for (int d = 0; d < 3; ++d) {
        ss[d] = sspacing ? (double)sspacing[d] : 1.0;
        ts[d] = tspacing ? (double)tspacing[d] : 1.0;
    }
    for (int i = 0; i < 3; ++i) {
        double c = (double)sorigin[i] + ss[i] * ((double)(sdims[i] - 1) / 2.0);
        a[i] = (float)((c - (double)torigin[i]) / ts[i]);
        double b = ((c + (double)pose[3 + i]) - (double)sorigin[i]) / ss[i];
        for (int j = 0; j < 3; ++j) M[4 * i + j] = (float)((R[3 * i + j] * ts[j]) / ss[i]);
        M[4 * i + 3] = (float)b;
    }
}

void orc_pose_matrix(const float pose[6], const int32_t sdims[3], const float sorigin[3],
                     const float torigin[3], float M[12], float a[3])
{
    orc_pose_matrix_sp(pose, sdims, sorigin, NULL, torigin, NULL, M, a);
}

/* q for target voxel (x, y, z), in this fixed fp32 order (no FMA):          */
/*   dx = x - a0 (likewise dy, dz)                                           */
/*   q_i = r_i0*dx + ((r_i1*dy + r_i2*dz) + b_i)                             */
static void coord(const float *M, const float a[3], int x, int y, int z, float q[3])
{
    float dx = (float)x - a[0];
    float dy = (float)y - a[1];
    float dz = (float)z - a[2];
    for (int i = 0; i < 3; ++i) {
        float K = (M[4 * i + 1] * dy + M[4 * i + 2] * dz) + M[4 * i + 3];
        q[i] = M[4 * i + 0] * dx + K;
    }
}

/* Nearest-neighbour sample of a binary mask (reading for masks): the voxel   */
/* floor(q + 0.5) on every axis, inside iff 0 <= q + 0.5 < dims (fp32).      */
static int nn_inside(const float q[3], const int32_t sd[3], int64_t *index)
{
    float h0 = q[0] + 0.5f, h1 = q[1] + 0.5f, h2 = q[2] + 0.5f;
    if (!(h0 >= 0.0f && h0 < (float)sd[0])) return 0;
    if (!(h1 >= 0.0f && h1 < (float)sd[1])) return 0;
    if (!(h2 >= 0.0f && h2 < (float)sd[2])) return 0;
    int64_t i0 = (int64_t)floorf(h0), i1 = (int64_t)floorf(h1), i2 = (int64_t)floorf(h2);
    *index = i0 + (int64_t)sd[0] * (i1 + (int64_t)sd[1] * i2);
    return 1;
}

/* Trilinear sample (Sec. 3.3).  Inside iff 0 <= q <= dims-1 on every axis   */
/* (fp32).  Base corner i = min(floor(q), dims-2), fraction f = q - i; lerp  */
/* along x, then y, then z, each lerp a + f*(b - a) in fp32 with the         */
/* difference b - a rounded and then a + f*d rounded once (fused multiply-   */
/* add: C99 fmaf is correctly rounded on every host).                        */
static float lerp(float a, float b, float f)
{
    return fmaf(f, b - a, a);
}

static int tri_sample(const uint8_t *S, const int32_t sd[3], const float q[3], float *out)
{
    for (int d = 0; d < 3; ++d)
        if (!(q[d] >= 0.0f && q[d] <= (float)(sd[d] - 1))) return 0;
    int i[3];
    float f[3];
    for (int d = 0; d < 3; ++d) {
        int fl = (int)floorf(q[d]);
        if (fl > sd[d] - 2) fl = sd[d] - 2;
        i[d] = fl;
        f[d] = q[d] - (float)fl;
    }
    int64_t sx = sd[0], sxy = (int64_t)sd[0] * sd[1];
    int64_t base = i[0] + sx * i[1] + sxy * i[2];
    float v000 = S[base], v100 = S[base + 1];
    float v010 = S[base + sx], v110 = S[base + sx + 1];
    float v001 = S[base + sxy], v101 = S[base + sxy + 1];
    float v011 = S[base + sxy + sx], v111 = S[base + sxy + sx + 1];
    float c00 = lerp(v000, v100, f[0]);
    float c10 = lerp(v010, v110, f[0]);
    float c01 = lerp(v001, v101, f[0]);
    float c11 = lerp(v011, v111, f[0]);
    float c0 = lerp(c00, c10, f[1]);
    float c1 = lerp(c01, c11, f[1]);
    *out = lerp(c0, c1, f[2]);
    return 1;
}

/* One trilinear sample (Sec. 3.3) at q, as tri_sample; returns 1 when q is  */
/* inside, else 0 and *out untouched (test export).                          */
int orc_trilinear(const uint8_t *S, const int32_t sd[3], const float q[3], float *out)
{
    return tri_sample(S, sd, q, out);
}

/* ------------------------------------------------------------------------ */
/* Measurement z^i (Fig. 1), mask mode: per matrix the four counts over the   */
/* target grid  n = #inside, A = sum S(q), B = sum T(p)[inside],              */
/* C = sum S(q) T(p).  Masks are binary (nonzero = 1).                       */
/* counts: 4 per matrix.                                                     */
/* ------------------------------------------------------------------------ */
void orc_measure_mask(const uint8_t *S, const int32_t sd[3], const uint8_t *T, const int32_t td[3],
                      const float *mats, const float a[3], int32_t m, uint64_t *counts)
{
    for (int32_t p = 0; p < m; ++p) {
        const float *M = mats + 12 * (int64_t)p;
        uint64_t n = 0, A = 0, B = 0, C = 0;
        for (int z = 0; z < td[2]; ++z)
            for (int y = 0; y < td[1]; ++y)
                for (int x = 0; x < td[0]; ++x) {
                    float q[3];
                    int64_t si;
                    coord(M, a, x, y, z, q);
                    if (!nn_inside(q, sd, &si)) continue;
                    uint64_t s = S[si] != 0;
                    uint64_t t = T[x + (int64_t)td[0] * (y + (int64_t)td[1] * z)] != 0;
                    n += 1;
                    A += s;
                    B += t;
                    C += s & t;
                }
        counts[4 * p + 0] = n;
        counts[4 * p + 1] = A;
        counts[4 * p + 2] = B;
        counts[4 * p + 3] = C;
    }
}

/* ------------------------------------------------------------------------ */
/* Measurement, image mode: moments of the trilinear sample s and target t   */
/* over the overlap set (voxels whose sample is inside the source grid).     */
/* Reading: s is rounded to 15 fractional bits, s_q = rint(32768 s), so     */
/* every moment is an exact integer sum (order-free, identical on any        */
/* hardware): n, S1 = sum s_q, S2 = sum s_q^2 (128-bit), ST = sum s_q t,      */
/* T1 = sum t, T2 = sum t^2.  s_q < 2^23.                                    */
/* mom: 7 per matrix = n, S1, S2 low word, S2 high word, ST, T1, T2.         */
/* ------------------------------------------------------------------------ */
void orc_measure_image(const uint8_t *S, const int32_t sd[3], const uint8_t *T, const int32_t td[3],
                       const float *mats, const float a[3], int32_t m, uint64_t *mom)
{
    for (int32_t p = 0; p < m; ++p) {
        const float *M = mats + 12 * (int64_t)p;
        uint64_t n = 0, S1 = 0, ST = 0, T1 = 0, T2 = 0;
        u128 S2 = 0;
        for (int z = 0; z < td[2]; ++z)
            for (int y = 0; y < td[1]; ++y)
                for (int x = 0; x < td[0]; ++x) {
                    float q[3], s;
                    coord(M, a, x, y, z, q);
                    if (!tri_sample(S, sd, q, &s)) continue;
                    uint64_t sq = (uint64_t)lrintf(s * 32768.0f);
                    uint64_t t = T[x + (int64_t)td[0] * (y + (int64_t)td[1] * z)];
                    n += 1;
                    S1 += sq;
                    S2 += (u128)(sq * sq);
                    ST += sq * t;
                    T1 += t;
                    T2 += t * t;
                }
        uint64_t *o = mom + 7 * (int64_t)p;
        o[0] = n; o[1] = S1; o[2] = (uint64_t)S2; o[3] = (uint64_t)(S2 >> 64);
        o[4] = ST; o[5] = T1; o[6] = T2;
    }
}

/* Independent fp64 check of the image score: the printed form of Eq. 2      */
/* (centred sums, two passes), with the trilinear sample taken in fp64 from  */
/* the same fp32 coordinates and no rounding of s.  Returns NCC^2 per matrix */
/* (0 when the overlap is empty or a variance vanishes).                     */
void orc_ncc2_f64(const uint8_t *S, const int32_t sd[3], const uint8_t *T, const int32_t td[3],
                  const float *mats, const float a[3], int32_t m, double *out)
{
    int64_t nt = (int64_t)td[0] * td[1] * td[2];
    double *sv = (double *)malloc(sizeof(double) * (size_t)nt);
    double *tv = (double *)malloc(sizeof(double) * (size_t)nt);
    for (int32_t p = 0; p < m; ++p) {
        const float *M = mats + 12 * (int64_t)p;
        int64_t n = 0;
        for (int z = 0; z < td[2]; ++z)
            for (int y = 0; y < td[1]; ++y)
                for (int x = 0; x < td[0]; ++x) {
                    float q[3];
                    coord(M, a, x, y, z, q);
                    int ok = 1;
                    for (int d = 0; d < 3; ++d)
                        if (!(q[d] >= 0.0f && q[d] <= (float)(sd[d] - 1))) ok = 0;
                    if (!ok) continue;
                    int i[3];
                    double f[3];
                    for (int d = 0; d < 3; ++d) {
                        int fl = (int)floorf(q[d]);
                        if (fl > sd[d] - 2) fl = sd[d] - 2;
                        i[d] = fl;
                        f[d] = (double)q[d] - (double)fl;
                    }
                    double acc = 0.0;
                    for (int c = 0; c < 8; ++c) {
                        int ox = c & 1, oy = (c >> 1) & 1, oz = (c >> 2) & 1;
                        double w = (ox ? f[0] : 1.0 - f[0]) * (oy ? f[1] : 1.0 - f[1]) *
                                   (oz ? f[2] : 1.0 - f[2]);
                        int64_t idx = (i[0] + ox) + (int64_t)sd[0] * ((i[1] + oy) + (int64_t)sd[1] * (i[2] + oz));
                        acc += w * (double)S[idx];
                    }
                    sv[n] = acc;
                    tv[n] = (double)T[x + (int64_t)td[0] * (y + (int64_t)td[1] * z)];
                    ++n;
                }
        if (n == 0) { out[p] = 0.0; continue; }
        double ms = 0.0, mt = 0.0;
        for (int64_t i = 0; i < n; ++i) { ms += sv[i]; mt += tv[i]; }
        ms /= (double)n;
        mt /= (double)n;
        double cst = 0.0, css = 0.0, ctt = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double ds = sv[i] - ms, dt = tv[i] - mt;
            cst += dt * ds;
            css += ds * ds;
            ctt += dt * dt;
        }
        out[p] = (css > 0.0 && ctt > 0.0) ? (cst * cst) / (ctt * css) : 0.0;
    }
    free(sv);
    free(tv);
}

/* ------------------------------------------------------------------------ */
/* Scores from integer moments.  NCC^2 of Eq. 2 multiplied through by n^2:   */
/*   NCC^2 = (n ST - S1 T1)^2 / ((n S2 - S1^2)(n T2 - T1^2)),                */
/* each bracket exact in 128-bit integers, then converted to fp64 by the     */
/* split hi*2^64 + lo (two round-to-nearest conversions and one add), and    */
/* combined as (c*c) / (vs*vt).  Dice of Eq. 4: 2C / (A + |T|).              */
/* A score is 0 when the overlap n is below n_min or a variance is 0.        */
/* ------------------------------------------------------------------------ */
static double u128_to_f64(u128 v)
{
    uint64_t hi = (uint64_t)(v >> 64), lo = (uint64_t)v;
    return (double)hi * 18446744073709551616.0 + (double)lo;
}

double orc_ncc2_from_moments(uint64_t n, uint64_t S1, uint64_t S2lo, uint64_t S2hi, uint64_t ST,
                             uint64_t T1, uint64_t T2, uint64_t n_min)
{
    if (n == 0 || n < n_min) return 0.0;
    u128 S2 = ((u128)S2hi << 64) | S2lo;
    u128 nS2 = (u128)n * S2, S1S1 = (u128)S1 * S1;
    u128 nT2 = (u128)n * T2, T1T1 = (u128)T1 * T1;
    if (nS2 <= S1S1 || nT2 <= T1T1) return 0.0;
    u128 vs = nS2 - S1S1, vt = nT2 - T1T1;
    u128 nST = (u128)n * ST, S1T1 = (u128)S1 * T1;
    u128 cv = nST >= S1T1 ? nST - S1T1 : S1T1 - nST;
    double c = u128_to_f64(cv);
    return (c * c) / (u128_to_f64(vs) * u128_to_f64(vt));
}

double orc_dice_from_counts(uint64_t n, uint64_t A, uint64_t C, uint64_t b_full, uint64_t n_min)
{
    if (n < n_min) return 0.0;
    if (A + b_full == 0) return 0.0;
    return (double)(2 * C) / (double)(A + b_full);
}

/* Score modes (reading): 0 mask Dice, 1 mask NCC^2 (binary moments), 2 image */
/* NCC^2, 3 combined 0.5*(image NCC^2 + mask Dice).                          */
/* mom12 = [n S1 S2lo S2hi ST T1 T2 0 | n_nn A B C].                         */
double orc_score(int32_t mode, const uint64_t mom12[12], uint64_t b_full, uint64_t n_min)
{
    const uint64_t *im = mom12, *mk = mom12 + 8;
    switch (mode) {
    case 0:
        return orc_dice_from_counts(mk[0], mk[1], mk[3], b_full, n_min);
    case 1:
        return orc_ncc2_from_moments(mk[0], mk[1], mk[1], 0, mk[3], mk[2], mk[2], n_min);
    case 2:
        return orc_ncc2_from_moments(im[0], im[1], im[2], im[3], im[4], im[5], im[6], n_min);
    case 3:
        return 0.5 * (orc_ncc2_from_moments(im[0], im[1], im[2], im[3], im[4], im[5], im[6], n_min) +
                      orc_dice_from_counts(mk[0], mk[1], mk[3], b_full, n_min));
    default:
        return 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* Update (Fig. 1): likelihood w_i = (s_i / s_max)^gamma, gamma = 2^g by g     */
/* squarings (reading), quantised to W_i = floor(w_i * 2^24).  All W = 0 when */
/* no particle scores above 0.                                               */
/* ------------------------------------------------------------------------ */
void orc_weights(const double *s, int32_t N, int32_t g, uint64_t *W)
{
    double smax = 0.0;
    for (int32_t i = 0; i < N; ++i)
        if (s[i] > smax) smax = s[i];
    for (int32_t i = 0; i < N; ++i) {
        if (!(smax > 0.0)) { W[i] = 0; continue; }
        double r = s[i] / smax;
        for (int32_t j = 0; j < g; ++j) r = r * r;
        W[i] = (uint64_t)(r * 16777216.0);
    }
}

/* ------------------------------------------------------------------------ */
/* Resampling (Fig. 1), reading: systematic resampling on the integer CDF.   */
/* C_i = W_0 + ... + W_i, S = C_{N-1}; with one offset u (32-bit draw) the    */
/* j-th pointer is T_j = floor((j 2^32 + u) S / (N 2^32)) and particle j     */
/* copies a_j = min{ i : C_i > T_j }.  S = 0 keeps every particle.           */
/* ------------------------------------------------------------------------ */
void orc_resample(const uint64_t *W, int32_t N, uint32_t u, int32_t *idx)
{
    uint64_t *C = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(N > 0 ? N : 1));
    uint64_t run = 0;
    for (int32_t i = 0; i < N; ++i) { run += W[i]; C[i] = run; }
    uint64_t S = N > 0 ? C[N - 1] : 0;
    int32_t i = 0;
    for (int32_t j = 0; j < N; ++j) {
        if (S == 0) { idx[j] = j; continue; }
        u128 num = (u128)((((uint64_t)j) << 32) + (uint64_t)u) * (u128)S;
        uint64_t T = (uint64_t)(num >> 32) / (uint64_t)N;
        while (!(C[i] > T)) ++i;   /* T_j is non-decreasing in j */
        idx[j] = i;
    }
    free(C);
}

/* Estimation (Fig. 1), reading: the weighted mean of the 6-vectors with the */
/* integer weights, before resampling; plain mean when S = 0.                 */
void orc_estimate(const float *poses, int32_t N, const uint64_t *W, double est[6])
{
    uint64_t S = 0;
    for (int32_t i = 0; i < N; ++i) S += W[i];
    for (int d = 0; d < 6; ++d) {
        const float *x = poses + (int64_t)d * N;
        double acc = 0.0;
        if (S > 0) {
            for (int32_t i = 0; i < N; ++i) acc = acc + (double)W[i] * (double)x[i];
            est[d] = acc / (double)S;
        } else {
            for (int32_t i = 0; i < N; ++i) acc = acc + (double)x[i];
            est[d] = acc / (double)N;
        }
    }
}

/* Initial particles inside the limits (Abstract: the method starts from      */
/* rotation and translation limits): x_id = L_d (2u - 1), u from Philox     */
/* counter (i, 0, INIT, d/4) word d%4.  poses: SoA [6][N].                   */
void orc_init(float *poses, int32_t N, uint64_t seed, const float lim[6])
{
    for (int32_t i = 0; i < N; ++i) {
        uint32_t r0[4], r1[4];
        philox_seeded(seed, (uint32_t)i, 0u, ORC_STREAM_INIT, 0u, r0);
        philox_seeded(seed, (uint32_t)i, 0u, ORC_STREAM_INIT, 1u, r1);
        uint32_t u[6] = {r0[0], r0[1], r0[2], r0[3], r1[0], r1[1]};
        for (int d = 0; d < 6; ++d)
            poses[(int64_t)d * N + i] = lim[d] * (2.0f * unit24(u[d]) - 1.0f);
    }
}

/* Initial particles drawn around a proposal (the learned approach of Sec. 6,  */
/* which seeds and shrinks the cloud): x_id = clamp(m_d + s_d eps, -L_d, L_d)  */
/* with the Irwin-Hall draw eps = (u1+u2+u3+u4 - 2) sqrt(3) of Philox counter  */
/* (i, 0, SEED, d).  poses: SoA [6][N].                                       */
void orc_init_gaussian(float *poses, int32_t N, uint64_t seed, const float mean[6], const float std[6],
                       const float lim[6])
{
    const float sqrt3 = 1.7320508075688772f;
    for (int32_t i = 0; i < N; ++i)
        for (int d = 0; d < 6; ++d) {
            uint32_t r[4];
            philox_seeded(seed, (uint32_t)i, 0u, ORC_STREAM_SEED, (uint32_t)d, r);
            float e = ((((unit24(r[0]) + unit24(r[1])) + unit24(r[2])) + unit24(r[3])) - 2.0f) * sqrt3;
            float v = mean[d] + std[d] * e;
            if (v > lim[d]) v = lim[d];
            if (v < -lim[d]) v = -lim[d];
            poses[(int64_t)d * N + i] = v;
        }
}

/* Noise scale of iteration k (reading): sigma_kd = sigma0_frac * L_d *       */
/* decay^k, decay^k by k fp64 products, rounded once to fp32.                */
void orc_sigma(float sigma0_frac, float decay, int32_t k, const float lim[6], float sigma[6])
{
    double p = 1.0;
    for (int32_t j = 0; j < k; ++j) p = p * (double)decay;
    for (int d = 0; d < 6; ++d) sigma[d] = (float)(((double)sigma0_frac * (double)lim[d]) * p);
}

/* Prediction (Fig. 1), reading: x <- clamp(x + sigma * eps, -L, L) with the  */
/* bounded unit-variance Irwin-Hall draw eps = (u1+u2+u3+u4 - 2) sqrt(3),    */
/* u_m from Philox counter (i, k, PERTURB, d).                               */
void orc_perturb(float *poses, int32_t N, uint64_t seed, int32_t k, const float sigma[6],
                 const float lim[6])
{
    const float sqrt3 = 1.7320508075688772f;
    for (int32_t i = 0; i < N; ++i)
        for (int d = 0; d < 6; ++d) {
            uint32_t r[4];
            philox_seeded(seed, (uint32_t)i, (uint32_t)k, ORC_STREAM_PERTURB, (uint32_t)d, r);
            float e = ((((unit24(r[0]) + unit24(r[1])) + unit24(r[2])) + unit24(r[3])) - 2.0f) * sqrt3;
            float *x = poses + (int64_t)d * N + i;
            float v = *x + sigma[d] * e;
            if (v > lim[d]) v = lim[d];
            if (v < -lim[d]) v = -lim[d];
            *x = v;
        }
}

uint32_t orc_resample_offset(uint64_t seed, int32_t k)
{
    uint32_t r[4];
    philox_seeded(seed, 0u, (uint32_t)k, ORC_STREAM_RESAMPLE, 0u, r);
    return r[0];
}

/* ------------------------------------------------------------------------ */
/* The whole filter, iteration k = 0..K-1 (Fig. 1 cycle, reading of order):   */
/*   k > 0: prediction (perturb);  every k: pose -> matrix, measurement,     */
/*   score, update (weights), estimation, resampling.                        */
/* Output: the estimate of the last iteration.  Optional traces (NULL skips): */
/*   tr_poses [K][6][N] (measured poses), tr_mom [K][N][12], tr_score [K][N], */
/*   tr_W [K][N], tr_idx [K][N], tr_est [K][6].                              */
/* Volumes unused by the mode may be NULL; so are the spacings ss, ts (1).  */
/* sig_base (6 floats or NULL): the per-DOF noise base that replaces         */
/* sigma0_frac * L_d (a proposal's spread), sigma_kd = sig_base_d * decay^k.  */
/* ------------------------------------------------------------------------ */
int32_t orc_register(int32_t mode, const uint8_t *src, const uint8_t *tgt, const uint8_t *src_mask,
                     const uint8_t *tgt_mask, const int32_t sd[3], const float so[3], const float ss[3],
                     const int32_t td[3], const float to[3], const float ts[3], int32_t N, int32_t K,
                     const float rot_lim[3], const float trans_lim[3], float sigma0_frac,
                     float decay, int32_t gamma_log2, uint64_t seed, float min_overlap_frac,
                     float *poses_inout, int32_t have_poses, int32_t k0, double est_out[6],
                     float *tr_poses, uint64_t *tr_mom, double *tr_score, uint64_t *tr_W,
                     int32_t *tr_idx, double *tr_est, const float *sig_base)
{
    const float lim[6] = {rot_lim[0], rot_lim[1], rot_lim[2], trans_lim[0], trans_lim[1], trans_lim[2]};
    int64_t nt = (int64_t)td[0] * td[1] * td[2];
    uint64_t n_min = (uint64_t)((double)min_overlap_frac * (double)nt);
    uint64_t b_full = 0;
    if (tgt_mask)
        for (int64_t v = 0; v < nt; ++v) b_full += tgt_mask[v] != 0;

    float *x = poses_inout;
    float *xn = (float *)malloc(sizeof(float) * 6 * (size_t)N);
    float *mats = (float *)malloc(sizeof(float) * 12 * (size_t)N);
    uint64_t *mom = (uint64_t *)calloc(12 * (size_t)N, sizeof(uint64_t));
    double *s = (double *)malloc(sizeof(double) * (size_t)N);
    uint64_t *W = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    float a[3];
    if (!have_poses) orc_init(x, N, seed, lim);

    for (int32_t kk = 0; kk < K; ++kk) {
        int32_t k = k0 + kk;
        if (k > 0) {
            float sig[6];
            orc_sigma(sigma0_frac, decay, k, lim, sig);
            if (sig_base) {
                double p = 1.0;
                for (int32_t j = 0; j < k; ++j) p = p * (double)decay;
                for (int d = 0; d < 6; ++d) sig[d] = (float)((double)sig_base[d] * p);
            }
            orc_perturb(x, N, seed, k, sig, lim);
        }
        for (int32_t i = 0; i < N; ++i) {
            float pose[6];
            for (int d = 0; d < 6; ++d) pose[d] = x[(int64_t)d * N + i];
            orc_pose_matrix_sp(pose, sd, so, ss, to, ts, mats + 12 * (int64_t)i, a);
        }
        memset(mom, 0, sizeof(uint64_t) * 12 * (size_t)N);
        for (int32_t i = 0; i < N; ++i) {
            if (mode == 2 || mode == 3)
                orc_measure_image(src, sd, tgt, td, mats + 12 * (int64_t)i, a, 1, mom + 12 * (int64_t)i);
            if (mode == 0 || mode == 1 || mode == 3)
                orc_measure_mask(src_mask, sd, tgt_mask, td, mats + 12 * (int64_t)i, a, 1,
                                 mom + 12 * (int64_t)i + 8);
        }
        for (int32_t i = 0; i < N; ++i) s[i] = orc_score(mode, mom + 12 * (int64_t)i, b_full, n_min);
        orc_weights(s, N, gamma_log2, W);
        double est[6];
        orc_estimate(x, N, W, est);
        orc_resample(W, N, orc_resample_offset(seed, k), idx);

        if (tr_poses) memcpy(tr_poses + (int64_t)kk * 6 * N, x, sizeof(float) * 6 * (size_t)N);
        if (tr_mom) memcpy(tr_mom + (int64_t)kk * 12 * N, mom, sizeof(uint64_t) * 12 * (size_t)N);
        if (tr_score) memcpy(tr_score + (int64_t)kk * N, s, sizeof(double) * (size_t)N);
        if (tr_W) memcpy(tr_W + (int64_t)kk * N, W, sizeof(uint64_t) * (size_t)N);
        if (tr_idx) memcpy(tr_idx + (int64_t)kk * N, idx, sizeof(int32_t) * (size_t)N);
        if (tr_est) memcpy(tr_est + (int64_t)kk * 6, est, sizeof(double) * 6);
        for (int d = 0; d < 6; ++d) {
            est_out[d] = est[d];
            for (int32_t j = 0; j < N; ++j) xn[(int64_t)d * N + j] = x[(int64_t)d * N + idx[j]];
        }
        memcpy(x, xn, sizeof(float) * 6 * (size_t)N);
    }
    free(xn); free(mats); free(mom); free(s); free(W); free(idx);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sequence warp (Abstract, Sec. 3.3: the ED-frame transform is applied to    */
/* every frame).  out(p) = rint(trilinear(frame, q(p))) (round half to even, */
/* saturated to 0..255), 0 where q is outside; interp 0 = nearest neighbour. */
/* ------------------------------------------------------------------------ */
void orc_warp(const uint8_t *src, const int32_t sd[3], uint8_t *out, const int32_t td[3],
              const float M[12], const float a[3], int32_t interp)
{
    for (int z = 0; z < td[2]; ++z)
        for (int y = 0; y < td[1]; ++y)
            for (int x = 0; x < td[0]; ++x) {
                float q[3];
                coord(M, a, x, y, z, q);
                uint8_t v = 0;
                if (interp == 0) {
                    int64_t si;
                    if (nn_inside(q, sd, &si)) v = src[si];
                } else {
                    float s;
                    if (tri_sample(src, sd, q, &s)) {
                        long r = lrintf(s);
                        v = (uint8_t)(r < 0 ? 0 : (r > 255 ? 255 : r));
                    }
                }
                out[x + (int64_t)td[0] * (y + (int64_t)td[1] * z)] = v;
            }
}
