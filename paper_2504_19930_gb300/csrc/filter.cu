// filter.cu -- the particle-filter cycle around the measurement (Fig. 1
// caption): initial cloud within the limits, prediction (perturbation),
// pose -> matrix, and the update / estimation / resampling step.
#include <atomic>
#include <climits>

#include "kernels.h"
#include "score.cuh"

namespace pfreg {

namespace {

std::atomic_uint64_t g_launches{0};

// Initial particles (Abstract: the search starts from rotation and translation
// limits): x_id = L_d (2u - 1), u = word d%4 of Philox counter (i, 0, INIT, d/4).
__global__ void k_init(const FilterParams P, float *poses) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const u32x4 r0 = philox_seeded(P.seed, (uint32_t)i, 0u, kStreamInit, 0u);
    const u32x4 r1 = philox_seeded(P.seed, (uint32_t)i, 0u, kStreamInit, 1u);
    const uint32_t u[6] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y};
#pragma unroll
    for (int d = 0; d < 6; ++d)
        poses[(size_t)d * P.N + i] = __fmul_rn(P.lim[d], __fsub_rn(__fmul_rn(2.0f, unit24(u[d])), 1.0f));
}

// Initial particles around a proposal (the learned approach of Sec. 6 seeds
// and shrinks the cloud): x_id = clamp(m_d + s_d eps, -L_d, L_d), eps the
// Irwin-Hall draw of Philox counter (i, 0, SEED, d).
struct Seed6 {
    float m[6], s[6];
};
__global__ void k_seed_gaussian(const FilterParams P, float *poses, const Seed6 sd) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const float sqrt3 = 1.7320508075688772f;
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        const u32x4 r = philox_seeded(P.seed, (uint32_t)i, 0u, kStreamSeed, (uint32_t)d);
        const float e = __fmul_rn(
            __fsub_rn(__fadd_rn(__fadd_rn(__fadd_rn(unit24(r.x), unit24(r.y)), unit24(r.z)), unit24(r.w)), 2.0f),
            sqrt3);
        float v = __fadd_rn(sd.m[d], __fmul_rn(sd.s[d], e));
        if (v > P.lim[d]) v = P.lim[d];
        if (v < -P.lim[d]) v = -P.lim[d];
        poses[(size_t)d * P.N + i] = v;
    }
}

// Prediction for k > 0 (reading: bounded Irwin-Hall noise of unit variance,
// eps = (u1+u2+u3+u4 - 2) sqrt(3) from Philox counter (i, k, PERTURB, d),
// scale sigma_kd = sigma0_frac * L_d * decay^k, clamped to the limits), then
// the pose -> matrix map of Eq. 3 and zeroed moment accumulators.
//
// One particle per group of 8 lanes: lane d < 6 perturbs DOF d; lanes 0-2
// take sin of the three angles and lanes 3-5 their cos (fp64 runs at 2
// operations per clock per SM on this part, so spreading the six series over
// lanes and over many small blocks is what bounds this kernel's latency);
// lane 0 assembles the matrix.  Every lane of the group must call this.
constexpr int kGroup = 8;

__device__ __forceinline__ void predict_particle(const FilterParams &P, const FilterBuffers &B, int i, int j,
                                                 unsigned gmask, int gbase) {
    const int k = *B.k;
    float x = j < 6 ? B.poses[(size_t)j * P.N + i] : 0.0f;
    if (k > 0 && j < 6) {
        double pk = 1.0;
        for (int q = 0; q < k; ++q) pk = __dmul_rn(pk, (double)P.sigma_decay);
        const float sqrt3 = 1.7320508075688772f;
        const float sig = __double2float_rn(__dmul_rn(P.sig0[j], pk));
        const u32x4 r = philox_seeded(P.seed, (uint32_t)i, (uint32_t)k, kStreamPerturb, (uint32_t)j);
        const float e = __fmul_rn(
            __fsub_rn(__fadd_rn(__fadd_rn(__fadd_rn(unit24(r.x), unit24(r.y)), unit24(r.z)), unit24(r.w)), 2.0f),
            sqrt3);
        float v = __fadd_rn(x, __fmul_rn(sig, e));
        if (v > P.lim[j]) v = P.lim[j];
        if (v < -P.lim[j]) v = -P.lim[j];
        x = v;
        B.poses[(size_t)j * P.N + i] = v;
    }
    // lanes 0-2: sin(angle j); lanes 3-5: cos(angle j-3)
    const float ang = __shfl_sync(gmask, x, gbase + (j < 3 ? j : (j < 6 ? j - 3 : 0)));
    double tv = 0.0;
    if (j < 6) tv = taylor_sincos(ang, j >= 3);   // one chain for the sine and cosine lanes
    double sc[6];
    float pose[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        sc[q] = __shfl_sync(gmask, tv, gbase + q);
        pose[q] = __shfl_sync(gmask, x, gbase + q);
    }
    if (j == 0) {
        float M[12];
        matrix_from_sincos(pose, sc[0], sc[3], sc[1], sc[4], sc[2], sc[5], P.g, M);
#pragma unroll
        for (int q = 0; q < 12; ++q) B.mats[(size_t)i * 12 + q] = M[q];
    }
    if (P.estimator == 1) {   // quaternion of the pose for the estimate: half angles on lanes 0-2
        const double cf = __shfl_sync(gmask, tv, gbase + (j < 3 ? j + 3 : 0));
        double hc = 0.0, hs = 0.0;
        if (j < 3) {
            hc = __dsqrt_rn(__dmul_rn(__dadd_rn(1.0, cf), 0.5));
            hs = __ddiv_rn(tv, __dmul_rn(2.0, hc));
        }
        double h[6];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            h[2 * q] = __shfl_sync(gmask, hc, gbase + q);
            h[2 * q + 1] = __shfl_sync(gmask, hs, gbase + q);
        }
        if (j == 0) {
            double qv[4];
            quat_from_half(h[0], h[1], h[2], h[3], h[4], h[5], qv);
#pragma unroll
            for (int q = 0; q < 4; ++q) B.quat[(size_t)q * P.N + i] = qv[q];
        }
    }
    for (int q = j; q < kMomStride; q += kGroup) B.mom[(size_t)i * kMomStride + q] = 0ull;
    if (i == 0 && j == kGroup - 1) {   // accumulators of the score kernel
        B.stats[0] = 0ull;
        B.stats[1] = 0ull;
    }
}

__global__ void __launch_bounds__(32) k_predict(const FilterParams P, const FilterBuffers B) {
    const int g = (blockIdx.x * blockDim.x + threadIdx.x) / kGroup;   // whole groups exit together
    if (g >= P.N) return;
    const int lane = threadIdx.x & 31, gbase = lane & ~(kGroup - 1);
    predict_particle(P, B, g, lane - gbase, 0xFFu << gbase, gbase);
}

// Weighted quaternion average: the unit eigenvector of the largest
// eigenvalue of the symmetric 4x4 A (upper triangle, row by row: a00 a01 a02
// a03 a11 a12 a13 a22 a23 a33) by cyclic Jacobi rotations, then the angles of
// its rotation matrix: R21 = sin rx, R20 = -cos rx sin ry, R22 = cos rx cos ry,
// R01 = -sin rz cos rx, R11 = cos rz cos rx.
__device__ __noinline__ void quat_average_angles(const double A10[10], double rot[3]) {
    double a[4][4], v[4][4];
    int t = 0;
    for (int i = 0; i < 4; ++i)
        for (int j = i; j < 4; ++j) {
            a[i][j] = a[j][i] = A10[t++];
        }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) v[i][j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 16; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int i = 0; i < 4; ++i) {
            diag += a[i][i] * a[i][i];
            for (int j = i + 1; j < 4; ++j) off += a[i][j] * a[i][j];
        }
        if (off <= 1e-32 * diag) break;
        for (int p = 0; p < 3; ++p)
            for (int q = p + 1; q < 4; ++q) {
                if (a[p][q] == 0.0) continue;
                const double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
                const double tt = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(tt * tt + 1.0), s = tt * c;
                for (int k = 0; k < 4; ++k) {   // columns p, q of A P
                    const double akp = a[k][p], akq = a[k][q];
                    a[k][p] = c * akp - s * akq;
                    a[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 4; ++k) {   // rows p, q of P^T (A P)
                    const double apk = a[p][k], aqk = a[q][k];
                    a[p][k] = c * apk - s * aqk;
                    a[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 4; ++k) {   // eigenvectors V P
                    const double vkp = v[k][p], vkq = v[k][q];
                    v[k][p] = c * vkp - s * vkq;
                    v[k][q] = s * vkp + c * vkq;
                }
            }
    }
    int m = 0;
    for (int i = 1; i < 4; ++i)
        if (a[i][i] > a[m][m]) m = i;
    double w = v[0][m], x = v[1][m], y = v[2][m], z = v[3][m];
    const double n = sqrt(w * w + x * x + y * y + z * z);
    w /= n; x /= n; y /= n; z /= n;
    const double r21 = 2.0 * (y * z + w * x), r20 = 2.0 * (x * z - w * y), r22 = 1.0 - 2.0 * (x * x + y * y);
    const double r01 = 2.0 * (x * y - w * z), r11 = 1.0 - 2.0 * (x * x + z * z);
    rot[0] = asin(fmax(-1.0, fmin(1.0, r21)));
    rot[1] = atan2(-r20, r22);
    rot[2] = atan2(-r01, r11);
}

constexpr int kFinThreads = 1024;
constexpr int kFinWarps = kFinThreads / 32;

constexpr int kCdfSmem = 12288;            // CDF entries staged in shared memory (96 KiB)
constexpr int kRed = 17;                   // reduced values: 6 pose sums, sum W^2, 10 of sum W q q^T

// Update, part 1 (one thread per particle, many CTAs): score s_i from the
// integer moments (Eq. 2 / Eq. 4); the maximum score, kept as the bits of a
// non-negative double (which order like the values) by a 64-bit atomic max,
// and the number of evaluations (sum of the overlap counts).  stats[0..1] are
// zeroed by the prediction kernel.
// The warp's maximum score bits and evaluation count are returned on every lane.
__device__ __forceinline__ void score_particle_warp(const FilterParams &P, const FilterBuffers &B, int i,
                                                    bool valid, unsigned long long &bits,
                                                    unsigned long long &ev) {
    double s = 0.0;
    ev = 0;
    if (valid) {
        const unsigned long long *m = B.mom + (size_t)i * kMomStride;
        s = score_from_moments(P.mode, m, P.b_full, P.n_min);
        B.scores[i] = s;
        ev = m[(P.mode == 2 || P.mode == 3) ? 0 : 8];
    }
    bits = (unsigned long long)__double_as_longlong(s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, bits, o);
        bits = ob > bits ? ob : bits;
        ev += __shfl_xor_sync(0xffffffffu, ev, o);
    }
}

__device__ __forceinline__ void score_particle(const FilterParams &P, const FilterBuffers &B, int i, bool valid) {
    unsigned long long bits, ev;
    score_particle_warp(P, B, i, valid, bits, ev);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(B.stats + 0, bits);
        if (ev) atomicAdd(B.stats + 1, ev);
    }
}

// Update, part 2: W_i = floor((s_i / max s)^(2^g) * 2^24).
__device__ __forceinline__ void weight_particle(const FilterParams &P, const FilterBuffers &B, int i) {
    const double smax = __longlong_as_double((long long)B.stats[0]);
    B.W[i] = quantised_weight(B.scores[i], smax > 0.0 ? smax : 0.0, P.gamma_log2);
}

__global__ void __launch_bounds__(128) k_score(const FilterParams P, const FilterBuffers B) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    score_particle(P, B, i, i < P.N);
}

__global__ void __launch_bounds__(128) k_weights(const FilterParams P, const FilterBuffers B) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P.N) weight_particle(P, B, i);
}

// Update, part 3, estimation and resampling of one iteration, in one CTA:
//   1. arg-max: the first particle whose score equals the maximum;
//   2. inclusive integer scan C of W (warp shuffles + warp totals), staged
//      in shared memory when it fits;
//   3. estimate = sum W_i x_i / sum W_i per DOF (fp64, before resampling)
//      and sum W_i^2 (effective sample size), one 7-value block reduction;
//   4. systematic resampling: T_j = floor((j 2^32 + u) S / (N 2^32)),
//      a_j = min{i : C_i > T_j} (binary search), gather the poses;
//   5. log the iteration and advance k.
__device__ __forceinline__ void finalise_block(const FilterParams &P, const FilterBuffers &B) {
    extern __shared__ unsigned long long sh_cdf[];
    __shared__ double sh_d[kFinWarps][kRed];
    __shared__ unsigned long long sh_u[kFinWarps];
    __shared__ int sh_i[kFinWarps];
    __shared__ double sh_est[kRed];
    __shared__ int sh_best_idx;
    const int N = P.N, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k = *B.k;
    const bool cdf_in_smem = N <= kCdfSmem;
    const unsigned long long smax_bits = B.stats[0];

    // 1. first index attaining the maximum
    int bidx = INT_MAX;
    for (int i = tid; i < N; i += kFinThreads)
        if ((unsigned long long)__double_as_longlong(B.scores[i]) == smax_bits) {
            bidx = i;
            break;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bidx = min(bidx, __shfl_xor_sync(0xffffffffu, bidx, o));
    if (lane == 0) sh_i[warp] = bidx;

    // 2. inclusive scan C of W, 1024 at a time with a running carry
    unsigned long long carry = 0;
    for (int base = 0; base < N; base += kFinThreads) {
        const int i = base + tid;
        unsigned long long v = i < N ? B.W[i] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        if (lane == 31) sh_u[warp] = v;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = sh_u[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long t = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += t;
            }
            sh_u[lane] = w;   // inclusive warp-total prefix
        }
        __syncthreads();
        const unsigned long long off = (warp > 0 ? sh_u[warp - 1] : 0ull) + carry;
        if (i < N) {
            B.C[i] = v + off;
            if (cdf_in_smem) sh_cdf[i] = v + off;
        }
        carry += sh_u[kFinWarps - 1];
        __syncthreads();
    }
    const unsigned long long S = carry;

    // 3. estimate and sum of squared weights, one block reduction of 7 values.
    // Only the warps that hold particles reduce: the others' sums are +0.0,
    // which warp 0 substitutes, and the fp64 pipe (2 lanes per clock per SM)
    // would spend ~16 clocks per warp instruction on their zeros.
    const int nw = N < kFinThreads ? (N + 31) / 32 : kFinWarps;
    double acc[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int i = tid; i < N; i += kFinThreads) {
        const double w = (double)B.W[i];
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            const double x = (double)B.poses[(size_t)d * N + i];
            acc[d] = __dadd_rn(acc[d], S > 0 ? __dmul_rn(w, x) : x);
        }
        acc[6] = __dadd_rn(acc[6], __dmul_rn(w, w));
    }
    if (warp < nw) {
#pragma unroll
        for (int d = 0; d < 7; ++d) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[d] = __dadd_rn(acc[d], __shfl_xor_sync(0xffffffffu, acc[d], o));
            if (lane == 0) sh_d[warp][d] = acc[d];
        }
    }
    if (P.estimator == 1) {   // the 10 entries of sum W q q^T (upper triangle, row by row)
        double aq[10];
#pragma unroll
        for (int t = 0; t < 10; ++t) aq[t] = 0.0;
        for (int i = tid; i < N; i += kFinThreads) {
            const double w = (double)B.W[i];
            double q[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) q[a] = B.quat[(size_t)a * N + i];
            int t = 0;
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = a; b < 4; ++b, ++t) {
                    const double qq = __dmul_rn(q[a], q[b]);
                    aq[t] = __dadd_rn(aq[t], S > 0 ? __dmul_rn(w, qq) : qq);
                }
        }
        if (warp < nw) {
#pragma unroll
            for (int t = 0; t < 10; ++t) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) aq[t] = __dadd_rn(aq[t], __shfl_xor_sync(0xffffffffu, aq[t], o));
                if (lane == 0) sh_d[warp][7 + t] = aq[t];
            }
        }
    }
    __syncthreads();
    if (warp == 0) {
        int bi = sh_i[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) bi = min(bi, __shfl_xor_sync(0xffffffffu, bi, o));
        if (lane == 0) sh_best_idx = bi;
        // the warps' partial sums, lane = warp, as trees (the estimate has no
        // fixed summation order; fp64 adds are ~60 clocks of dependent latency)
        const int nred = P.estimator == 1 ? kRed : 7;
#pragma unroll
        for (int d = 0; d < kRed; ++d) {
            if (d < nred) {
                double t = lane < nw ? sh_d[lane][d] : 0.0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) t = __dadd_rn(t, __shfl_xor_sync(0xffffffffu, t, o));
                if (lane == 0) sh_est[d] = t;
            }
        }
    }
    // 4. resampling: keep the measured cloud, gather the copies
    for (size_t e = tid; e < (size_t)6 * N; e += kFinThreads) B.poses_meas[e] = B.poses[e];
    __syncthreads();
    const unsigned long long *cdf = cdf_in_smem ? sh_cdf : B.C;
    const uint32_t u = philox_seeded(P.seed, 0u, (uint32_t)k, kStreamResample, 0u).x;
    for (int j = tid; j < N; j += kFinThreads) {
        int a = j;
        if (S > 0) {
            const unsigned __int128 num =
                (unsigned __int128)((((unsigned long long)j) << 32) + (unsigned long long)u) * S;
            const unsigned long long T = (unsigned long long)(num >> 32) / (unsigned long long)N;
            int lo = 0, hi = N - 1;          // first i with C_i > T (exists: C_{N-1} = S > T)
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (cdf[mid] > T) hi = mid; else lo = mid + 1;
            }
            a = lo;
        }
        B.idx[j] = a;
#pragma unroll
        for (int d = 0; d < 6; ++d) B.poses[(size_t)d * N + j] = B.poses_meas[(size_t)d * N + a];
    }

    // 5. log and advance the iteration counter (the six quotients on six lanes)
    IterLog &L = B.log[k % P.log_capacity];
    if (tid < 6) L.est[tid] = S > 0 ? __ddiv_rn(sh_est[tid], (double)S) : __ddiv_rn(sh_est[tid], (double)N);
    if (tid == 6) {
        const double Sd = (double)S, w2 = sh_est[6];
        L.ess = w2 > 0.0 ? Sd * Sd / w2 : 0.0;
    }
    __syncwarp();
    if (tid == 0) {
        if (P.estimator == 1) {
            double A10[10], rot[3];
            const double norm = S > 0 ? (double)S : (double)N;
            for (int t = 0; t < 10; ++t) A10[t] = __ddiv_rn(sh_est[7 + t], norm);
            quat_average_angles(A10, rot);
            for (int d = 0; d < 3; ++d) L.est[d] = rot[d];
        }
        L.best = __longlong_as_double((long long)smax_bits);
        L.best_idx = sh_best_idx;
        L.evals = B.stats[1];
        L.est_dice = -1.0;
        L.k = k;
        *B.k = k + 1;
    }
}

__global__ void __launch_bounds__(kFinThreads) k_finalise(const FilterParams P, const FilterBuffers B) {
    finalise_block(P, B);
}

// The whole update of a cloud that fits one CTA (N <= kFinThreads) in one
// launch: thread i scores particle i, the block reduces the maximum score and
// the evaluation count (the integers the atomics of the multi-CTA form
// produce), then the weights, then the estimate and resampling.  It saves
// the two small launches and their gaps, which on a 64^3 mask registration
// are a few percent of each iteration.
__global__ void __launch_bounds__(kFinThreads) k_update_small(const FilterParams P, const FilterBuffers B) {
    __shared__ unsigned long long sh_bits[kFinWarps], sh_ev[kFinWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long bits, ev;
    score_particle_warp(P, B, tid, tid < P.N, bits, ev);
    if (lane == 0) {
        sh_bits[warp] = bits;
        sh_ev[warp] = ev;
    }
    __syncthreads();
    if (warp == 0) {
        bits = sh_bits[lane];
        ev = sh_ev[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ob = __shfl_xor_sync(0xffffffffu, bits, o);
            bits = ob > bits ? ob : bits;
            ev += __shfl_xor_sync(0xffffffffu, ev, o);
        }
        if (lane == 0) {
            B.stats[0] = bits;
            B.stats[1] = ev;
        }
    }
    __syncthreads();
    if (tid < P.N) weight_particle(P, B, tid);
    __syncthreads();
    finalise_block(P, B);
}

// Batched prediction: group of 8 lanes -> (registration, particle) by binary
// search on the particle prefix; registrations that have finished are skipped
// (every lane of a group takes the same branch).
__global__ void __launch_bounds__(32) k_predict_batch(const BatchReg *__restrict__ regs,
                                                      const long long *__restrict__ poffs, int nregs) {
    const long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / kGroup;
    if (g >= poffs[nregs]) return;
    int lo = 0, hi = nregs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (poffs[mid] <= g) lo = mid; else hi = mid - 1;
    }
    const BatchReg &R = regs[lo];
    if (*R.B.k >= R.n_iters) return;
    const int lane = threadIdx.x & 31, gbase = lane & ~(kGroup - 1);
    predict_particle(R.P, R.B, (int)(g - poffs[lo]), lane - gbase, 0xFFu << gbase, gbase);
}

// Batched update: scores and weights over all particles, each registration's
// particles padded to whole warps (poffs32) so that every warp belongs to one
// registration; then one CTA per registration.
__device__ __forceinline__ int find_reg(const long long *offs, int n, long long g) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (offs[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(128) k_score_batch(const BatchReg *__restrict__ regs,
                                                     const long long *__restrict__ poffs32, int nregs) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long gw = g & ~31ll;                   // warp-uniform
    if (gw >= poffs32[nregs]) return;
    const int r = find_reg(poffs32, nregs, gw);
    const BatchReg &R = regs[r];
    if (*R.B.k >= R.n_iters) return;
    const int i = (int)(g - poffs32[r]);
    score_particle(R.P, R.B, i, i < R.P.N);
}

__global__ void __launch_bounds__(128) k_weights_batch(const BatchReg *__restrict__ regs,
                                                       const long long *__restrict__ poffs32, int nregs) {
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= poffs32[nregs]) return;
    const int r = find_reg(poffs32, nregs, g);
    const BatchReg &R = regs[r];
    if (*R.B.k >= R.n_iters) return;
    const int i = (int)(g - poffs32[r]);
    if (i < R.P.N) weight_particle(R.P, R.B, i);
}

__global__ void __launch_bounds__(kFinThreads) k_finalise_batch(const BatchReg *__restrict__ regs) {
    const BatchReg &R = regs[blockIdx.x];
    if (*R.B.k >= R.n_iters) return;   // block-uniform: before any barrier
    finalise_block(R.P, R.B);
}

// Matrix of one pose by a group of 8 lanes (lanes 0-2: sin of the angles,
// 3-5: their cos; lane 0 assembles); every lane of the group calls this and
// lane 0 holds M on return.
__device__ __forceinline__ void group_pose_matrix(const float pose[6], int j, unsigned gmask, int gbase,
                                                  const Geometry &g, float M[12]) {
    double tv = 0.0;
    if (j < 6) tv = taylor_sincos(pose[j < 3 ? j : j - 3], j >= 3);
    double sc[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) sc[q] = __shfl_sync(gmask, tv, gbase + q);
    if (j == 0) matrix_from_sincos(pose, sc[0], sc[3], sc[1], sc[4], sc[2], sc[5], g, M);
}

// Estimate of iteration k-1 (the counter has advanced) rounded to fp32, as
// the pose whose matrix the masks are warped with; zeroes the counts.
__global__ void k_trace_prepare(const FilterParams P, const FilterBuffers B) {
    if (blockIdx.x != 0 || threadIdx.x >= kGroup) return;
    const int j = threadIdx.x;
    const int k = *B.k - 1;
    const IterLog &L = B.log[k % P.log_capacity];
    float pose[6];
    for (int d = 0; d < 6; ++d) pose[d] = __double2float_rn(L.est[d]);
    float M[12];
    group_pose_matrix(pose, j, 0xFFu, 0, P.g, M);
    if (j == 0)
        for (int q = 0; q < 12; ++q) B.trace_mat[q] = M[q];
    for (int q = j; q < kMomStride; q += kGroup) B.trace_mom[q] = 0ull;
}

// Dice (Eq. 4, whole target grid, no overlap threshold) of the estimate.
__global__ void k_trace_finish(const FilterParams P, const FilterBuffers B) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int k = *B.k - 1;
    const unsigned long long *m = B.trace_mom + 8;
    B.log[k % P.log_capacity].est_dice = dice_from_counts(m[0], m[1], m[3], P.b_full, 0ull);
}

__global__ void k_pack_bits(const uint8_t *mask, int64_t nvox, uint32_t *bits) {
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w * 32 >= nvox) return;
    uint32_t v = 0;
    for (int b = 0; b < 32; ++b) {
        const int64_t i = w * 32 + b;
        if (i < nvox && mask[i] != 0) v |= 1u << b;
    }
    bits[w] = v;
}

__global__ void k_count_nonzero(const uint8_t *v, int64_t n, unsigned long long *out) {
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += v[i] != 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

__global__ void k_binarise(const uint8_t *in, uint8_t *out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i] != 0;
}

__global__ void k_pose_matrix(const float *pose, Geometry g, float *out) {
    if (blockIdx.x != 0 || threadIdx.x >= kGroup) return;
    const int j = threadIdx.x;
    float x[6], M[12];
    for (int d = 0; d < 6; ++d) x[d] = pose[d];
    group_pose_matrix(x, j, 0xFFu, 0, g, M);
    if (j == 0)
        for (int q = 0; q < 12; ++q) out[q] = M[q];
}

__global__ void k_score_one(int mode, const unsigned long long *mom, unsigned long long b_full,
                            unsigned long long n_min, double *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *out = score_from_moments(mode, mom, b_full, n_min);
}

__global__ void k_philox(const uint32_t *ck, uint32_t *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const u32x4 r = philox10(u32x4{ck[0], ck[1], ck[2], ck[3]}, ck[4], ck[5]);
        out[0] = r.x; out[1] = r.y; out[2] = r.z; out[3] = r.w;
    }
}

unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

void count_launches(uint64_t n) {
    if (!capturing()) g_launches.fetch_add(n, std::memory_order_relaxed);
}
uint64_t launches() { return g_launches.load(std::memory_order_relaxed); }

// Every device allocation the library makes goes through these two calls,
// which count the successful ones process-wide (pf_debug_device_allocs).
static std::atomic<uint64_t> g_device_allocs{0};
cudaError_t dev_malloc_bytes(void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) g_device_allocs.fetch_add(1, std::memory_order_relaxed);
    return e;
}
cudaError_t dev_malloc_async_bytes(void **p, size_t bytes, cudaStream_t s) {
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e == cudaSuccess) g_device_allocs.fetch_add(1, std::memory_order_relaxed);
    return e;
}
uint64_t device_allocs() { return g_device_allocs.load(std::memory_order_relaxed); }

cudaError_t launch_init_particles(const FilterParams &p, const FilterBuffers &b, cudaStream_t s) {
    k_init<<<blocks_for(p.N, 256), 256, 0, s>>>(p, b.poses);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_seed_gaussian(const FilterParams &p, const FilterBuffers &b, const float mean[6],
                                 const float std[6], cudaStream_t s) {
    Seed6 sd;
    for (int d = 0; d < 6; ++d) {
        sd.m[d] = mean[d];
        sd.s[d] = std[d];
    }
    k_seed_gaussian<<<blocks_for(p.N, 256), 256, 0, s>>>(p, b.poses, sd);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_predict(const FilterParams &p, const FilterBuffers &b, cudaStream_t s) {
    k_predict<<<blocks_for((int64_t)p.N * kGroup, 32), 32, 0, s>>>(p, b);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_predict_batch(const BatchReg *regs, const long long *poffs, int nregs, long long total,
                                 cudaStream_t s) {
    if (nregs <= 0 || total <= 0) return cudaSuccess;
    k_predict_batch<<<blocks_for(total * kGroup, 32), 32, 0, s>>>(regs, poffs, nregs);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_finalise_batch(const BatchReg *regs, const long long *poffs32, int nregs, long long total32,
                                  cudaStream_t s) {
    if (nregs <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_finalise_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kCdfSmem * sizeof(unsigned long long)));
    if (e != cudaSuccess) return e;
    k_score_batch<<<blocks_for(total32, 128), 128, 0, s>>>(regs, poffs32, nregs);
    k_weights_batch<<<blocks_for(total32, 128), 128, 0, s>>>(regs, poffs32, nregs);
    k_finalise_batch<<<nregs, kFinThreads, kCdfSmem * sizeof(unsigned long long), s>>>(regs);
    count_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_finalise(const FilterParams &p, const FilterBuffers &b, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_finalise, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kCdfSmem * sizeof(unsigned long long)));
    if (e != cudaSuccess) return e;
    if (p.N <= kFinThreads) {
        e = cudaFuncSetAttribute(k_update_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kCdfSmem * sizeof(unsigned long long)));
        if (e != cudaSuccess) return e;
        k_update_small<<<1, kFinThreads, kCdfSmem * sizeof(unsigned long long), s>>>(p, b);
        count_launches(1);
        return cudaGetLastError();
    }
    k_score<<<blocks_for(p.N, 128), 128, 0, s>>>(p, b);
    k_weights<<<blocks_for(p.N, 128), 128, 0, s>>>(p, b);
    k_finalise<<<1, kFinThreads, kCdfSmem * sizeof(unsigned long long), s>>>(p, b);
    count_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_trace_prepare(const FilterParams &p, const FilterBuffers &b, cudaStream_t s) {
    k_trace_prepare<<<1, 32, 0, s>>>(p, b);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_trace_finish(const FilterParams &p, const FilterBuffers &b, cudaStream_t s) {
    k_trace_finish<<<1, 32, 0, s>>>(p, b);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_pack_bits(const uint8_t *mask, int64_t nvox, uint32_t *bits, cudaStream_t s) {
    const int64_t words = (nvox + 31) / 32;
    k_pack_bits<<<blocks_for(words, 256), 256, 0, s>>>(mask, nvox, bits);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_count_nonzero(const uint8_t *v, int64_t n, unsigned long long *out, cudaStream_t s) {
    unsigned g = blocks_for(n, 256);
    if (g > 4096) g = 4096;
    k_count_nonzero<<<g, 256, 0, s>>>(v, n, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_binarise(const uint8_t *in, uint8_t *out, int64_t n, cudaStream_t s) {
    unsigned g = blocks_for(n, 256);
    if (g > 4096) g = 4096;
    k_binarise<<<g, 256, 0, s>>>(in, out, n);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_pose_matrix(const float *pose, Geometry g, float *mat_out, cudaStream_t s) {
    k_pose_matrix<<<1, 32, 0, s>>>(pose, g, mat_out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_score_one(int mode, const unsigned long long *mom, unsigned long long b_full,
                             unsigned long long n_min, double *out, cudaStream_t s) {
    k_score_one<<<1, 32, 0, s>>>(mode, mom, b_full, n_min, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t *ctr_key, uint32_t *out, cudaStream_t s) {
    k_philox<<<1, 32, 0, s>>>(ctr_key, out);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pfreg
