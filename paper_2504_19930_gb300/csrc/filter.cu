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

// Prediction for k > 0 (reading: bounded Irwin-Hall noise of unit variance,
// eps = (u1+u2+u3+u4 - 2) sqrt(3) from Philox counter (i, k, PERTURB, d),
// scale sigma_kd = sigma0_frac * L_d * decay^k, clamped to the limits), then
// the pose -> matrix map of Eq. 3 and zeroed moment accumulators.
__global__ void k_predict(const FilterParams P, const FilterBuffers B) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.N) return;
    const int k = *B.k;
    float x[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) x[d] = B.poses[(size_t)d * P.N + i];
    if (k > 0) {
        double pk = 1.0;
        for (int j = 0; j < k; ++j) pk = __dmul_rn(pk, (double)P.sigma_decay);
        const float sqrt3 = 1.7320508075688772f;
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            const float sig = __double2float_rn(__dmul_rn(__dmul_rn((double)P.sigma0_frac, (double)P.lim[d]), pk));
            const u32x4 r = philox_seeded(P.seed, (uint32_t)i, (uint32_t)k, kStreamPerturb, (uint32_t)d);
            const float e = __fmul_rn(
                __fsub_rn(__fadd_rn(__fadd_rn(__fadd_rn(unit24(r.x), unit24(r.y)), unit24(r.z)), unit24(r.w)), 2.0f),
                sqrt3);
            float v = __fadd_rn(x[d], __fmul_rn(sig, e));
            if (v > P.lim[d]) v = P.lim[d];
            if (v < -P.lim[d]) v = -P.lim[d];
            x[d] = v;
            B.poses[(size_t)d * P.N + i] = v;
        }
    }
    float M[12];
    pose_to_matrix(x, P.g, M);
#pragma unroll
    for (int j = 0; j < 12; ++j) B.mats[(size_t)i * 12 + j] = M[j];
#pragma unroll
    for (int j = 0; j < kMomStride; ++j) B.mom[(size_t)i * kMomStride + j] = 0ull;
}

constexpr int kFinThreads = 1024;
constexpr int kFinWarps = kFinThreads / 32;

__device__ __forceinline__ double block_sum_f64(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = sh[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t = __dadd_rn(t, __shfl_xor_sync(0xffffffffu, t, o));
        if (threadIdx.x == 0) sh[0] = t;
    }
    __syncthreads();
    return sh[0];
}

// Update, estimation and resampling of one iteration, in one CTA:
//   1. score s_i from the integer moments (Eq. 2 / Eq. 4), max s (first index);
//   2. W_i = floor((s_i / max s)^(2^g) * 2^24);
//   3. inclusive integer scan C of W (warp shuffles + warp totals);
//   4. estimate = sum W_i x_i / sum W_i per DOF (fp64), effective sample size;
//   5. systematic resampling: T_j = floor((j 2^32 + u) S / (N 2^32)),
//      a_j = min{i : C_i > T_j} (binary search), gather the poses;
//   6. log the iteration and advance k.
__global__ void __launch_bounds__(kFinThreads) k_finalise(const FilterParams P, const FilterBuffers B) {
    __shared__ double sh_d[kFinWarps];
    __shared__ unsigned long long sh_u[kFinWarps];
    __shared__ int sh_i[kFinWarps];
    __shared__ double sh_best;
    __shared__ int sh_best_idx;
    __shared__ unsigned long long sh_evals;
    const int N = P.N, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k = *B.k;

    // 1. scores and the arg-max (smallest index among equal maxima)
    double bmax = -1.0;
    int bidx = INT_MAX;
    unsigned long long evals = 0;
    const int n_col = (P.mode == 2 || P.mode == 3) ? 0 : 8;
    for (int i = tid; i < N; i += kFinThreads) {
        const unsigned long long *m = B.mom + (size_t)i * kMomStride;
        const double s = score_from_moments(P.mode, m, P.b_full, P.n_min);
        B.scores[i] = s;
        evals += m[n_col];
        if (s > bmax) { bmax = s; bidx = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) evals += __shfl_xor_sync(0xffffffffu, evals, o);
    if (lane == 0) sh_u[warp] = evals;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bmax, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
        if (ov > bmax || (ov == bmax && oi < bidx)) { bmax = ov; bidx = oi; }
    }
    if (lane == 0) { sh_d[warp] = bmax; sh_i[warp] = bidx; }
    __syncthreads();
    if (tid == 0) {
        unsigned long long ev = 0;
        for (int w = 0; w < kFinWarps; ++w) ev += sh_u[w];
        sh_evals = ev;
        double m = sh_d[0];
        int mi = sh_i[0];
        for (int w = 1; w < kFinWarps; ++w)
            if (sh_d[w] > m || (sh_d[w] == m && sh_i[w] < mi)) { m = sh_d[w]; mi = sh_i[w]; }
        sh_best = m;
        sh_best_idx = mi;
    }
    __syncthreads();
    const double smax = sh_best > 0.0 ? sh_best : 0.0;

    // 2. quantised likelihood weights
    for (int i = tid; i < N; i += kFinThreads) B.W[i] = quantised_weight(B.scores[i], smax, P.gamma_log2);
    __syncthreads();

    // 3. inclusive scan C of W, 1024 at a time with a running carry
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
        if (i < N) B.C[i] = v + off;
        carry += sh_u[kFinWarps - 1];
        __syncthreads();
    }
    const unsigned long long S = carry;

    // 4. estimate (before resampling) and effective sample size
    double est[6];
    for (int d = 0; d < 6; ++d) {
        double acc = 0.0;
        for (int i = tid; i < N; i += kFinThreads) {
            const double x = (double)B.poses[(size_t)d * N + i];
            acc = __dadd_rn(acc, S > 0 ? __dmul_rn((double)B.W[i], x) : x);
        }
        const double tot = block_sum_f64(acc, sh_d);
        est[d] = S > 0 ? __ddiv_rn(tot, (double)S) : __ddiv_rn(tot, (double)N);
    }
    double w2 = 0.0;
    for (int i = tid; i < N; i += kFinThreads) {
        const double w = (double)B.W[i];
        w2 = __dadd_rn(w2, __dmul_rn(w, w));
    }
    w2 = block_sum_f64(w2, sh_d);

    // 5. resampling: keep the measured cloud, gather the copies
    for (size_t e = tid; e < (size_t)6 * N; e += kFinThreads) B.poses_meas[e] = B.poses[e];
    __syncthreads();
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
                if (B.C[mid] > T) hi = mid; else lo = mid + 1;
            }
            a = lo;
        }
        B.idx[j] = a;
#pragma unroll
        for (int d = 0; d < 6; ++d) B.poses[(size_t)d * N + j] = B.poses_meas[(size_t)d * N + a];
    }

    // 6. log and advance the iteration counter
    if (tid == 0) {
        IterLog &L = B.log[k % P.log_capacity];
        for (int d = 0; d < 6; ++d) L.est[d] = est[d];
        L.best = sh_best;
        L.best_idx = sh_best_idx;
        L.evals = sh_evals;
        L.est_dice = -1.0;
        const double Sd = (double)S;
        L.ess = w2 > 0.0 ? Sd * Sd / w2 : 0.0;
        L.k = k;
        *B.k = k + 1;
    }
}

// Estimate of iteration k-1 (the counter has advanced) rounded to fp32, as
// the pose whose matrix the masks are warped with; zeroes the counts.
__global__ void k_trace_prepare(const FilterParams P, const FilterBuffers B) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int k = *B.k - 1;
    const IterLog &L = B.log[k % P.log_capacity];
    float pose[6];
    for (int d = 0; d < 6; ++d) pose[d] = __double2float_rn(L.est[d]);
    float M[12];
    pose_to_matrix(pose, P.g, M);
    for (int j = 0; j < 12; ++j) B.trace_mat[j] = M[j];
    for (int j = 0; j < kMomStride; ++j) B.trace_mom[j] = 0ull;
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
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        float x[6], M[12];
        for (int d = 0; d < 6; ++d) x[d] = pose[d];
        pose_to_matrix(x, g, M);
        for (int j = 0; j < 12; ++j) out[j] = M[j];
    }
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

cudaError_t launch_init_particles(const FilterParams &p, const FilterBuffers &b, cudaStream_t s) {
    k_init<<<blocks_for(p.N, 256), 256, 0, s>>>(p, b.poses);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_predict(const FilterParams &p, const FilterBuffers &b, cudaStream_t s) {
    k_predict<<<blocks_for(p.N, 128), 128, 0, s>>>(p, b);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_finalise(const FilterParams &p, const FilterBuffers &b, cudaStream_t s) {
    k_finalise<<<1, kFinThreads, 0, s>>>(p, b);
    count_launches(1);
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
