// Whole filter iterations as the iteration graph runs them -- k_predict,
// k_measure, then k_update_small or k_score / k_weights / k_finalise --
// copied verbatim by the test out of filter.cu and measure.cu (into
// batch_filter.inc and batch_measure.inc, their dynamic shared arrays
// declared here) and run block by block on the host under the emulation of
// tests/host_shim/warp_emulation.h, iteration after iteration from the
// initial cloud.  Exported with a C ABI for tests/test_device_identities.py.
// Test infrastructure only.
#include "host_shim/warp_emulation.h"

#include <climits>

#include "../paper_2504_19930_gb300/csrc/kernels.h"
#include "../paper_2504_19930_gb300/csrc/score.cuh"
#include "host_layouts.h"

dim3 threadIdx, blockIdx, blockDim, gridDim;
#define threadIdx (dim3{(unsigned)host_warp::tid, 1u, 1u})

#define PF_DEBUG 0
#define PF_USE_F32X2 0
namespace pfreg {
float4 smem_dyn[1 << 16];           // the measurement kernel's dynamic shared memory
unsigned long long sh_cdf[12288];   // the update's (the CDF)
#include "batch_measure.inc"
#include "batch_filter.inc"
}

namespace {
using namespace pfreg;
template <class K>
void launch(unsigned blocks, unsigned threads, K &&kernel) {
    gridDim.x = blocks;
    blockDim.x = threads;
    for (unsigned b = 0; b < blocks; ++b) {
        blockIdx.x = b;
        host_warp::run((int)threads, [&](int) { kernel(); });
    }
}
}  // namespace

// K iterations from the initial cloud poses [6][N].
// Per iteration kk the traces receive the measured cloud tr_poses [K][6][N],
// moments tr_mom [K][N][12], scores tr_s [K][N], weights tr_W [K][N],
// indices tr_idx [K][N] and the estimate tr_est [K][6].  Volumes the mode
// does not use are NULL, and so are unit voxel spacings ss / ts.  ipw: work
// items per warp of the measurement.
extern "C" void dm_trajectory(int mode, int N, int K, uint64_t seed, const float lim[6], float sigma0_frac,
                              float decay, int gamma_log2, float min_overlap_frac, const uint8_t *src,
                              const uint8_t *src_mask, const int32_t sd[3], const float so[3], const uint8_t *tgt,
                              const uint8_t *tgt_mask, const int32_t td[3], const float to[3], const float a_off[3],
                              const float *ss, const float *ts, int ipw, float *poses, float *tr_poses, uint64_t *tr_mom, double *tr_s,
                              uint64_t *tr_W, int32_t *tr_idx, double *tr_est) {
    const bool img = mode == 2 || mode == 3, mask = mode != 2;
    std::vector<uint32_t> quad, bits;
    host_layouts(src, src_mask, sd, quad, bits);
    const size_t nt = (size_t)td[0] * td[1] * td[2];
    uint64_t b_full = 0;
    if (tgt_mask)
        for (size_t v = 0; v < nt; ++v) b_full += tgt_mask[v] != 0;
    FilterParams P{};
    P.mode = mode;
    P.N = N;
    P.seed = seed;
    P.gamma_log2 = gamma_log2;
    P.b_full = b_full;
    P.n_min = (uint64_t)((double)min_overlap_frac * (double)nt);
    P.log_capacity = 64;
    P.sigma0_frac = sigma0_frac;
    P.sigma_decay = decay;
    for (int d = 0; d < 6; ++d) {
        P.lim[d] = lim[d];
        P.sig0[d] = (double)sigma0_frac * (double)lim[d];
    }
    for (int d = 0; d < 3; ++d) {
        P.g.sd[d] = sd[d];
        P.g.td[d] = td[d];
        P.g.so[d] = so[d];
        P.g.to[d] = to[d];
        P.g.ss[d] = ss ? ss[d] : 1.0f;
        P.g.ts[d] = ts ? ts[d] : 1.0f;
        P.g.a[d] = a_off[d];
    }
    std::vector<float> pm(6 * (size_t)N), mats(12 * (size_t)N);
    std::vector<unsigned long long> mom(12 * (size_t)N), W(N), C(N), stats(2);
    std::vector<double> scores(N);
    std::vector<int32_t> idx(N);
    std::vector<IterLog> log(64);
    int32_t k = 0;
    FilterBuffers B{};
    B.poses = poses;
    B.poses_meas = pm.data();
    B.mats = mats.data();
    B.mom = mom.data();
    B.scores = scores.data();
    B.W = W.data();
    B.C = C.data();
    B.idx = idx.data();
    B.k = &k;
    B.log = log.data();
    B.stats = stats.data();
    MeasureArgs A{};
    A.src_quad = quad.data();
    A.tgt_img = tgt;
    A.src_bits = bits.data();
    A.tgt_mask = tgt_mask;
    A.mats = mats.data();
    A.mom = mom.data();
    A.g = P.g;
    A.P = N;
    A.items_per_warp = ipw;
    A.fdims[0] = (float)sd[0];
    A.fdims[1] = (float)((int64_t)sd[0] * sd[1]);
    A.fdims[2] = (float)(sd[1] - 2);
    A.fdims[3] = (float)(sd[2] - 2);
    const int rows = td[1] * td[2];
    const long long items = (long long)N * ((rows + kRowsPerWarp - 1) / kRowsPerWarp);
    const unsigned mgrid = (unsigned)((items + kWarps * ipw_of(ipw) - 1) / (kWarps * ipw_of(ipw)));
    const bool fidx = (size_t)sd[0] * sd[1] * sd[2] <= ((size_t)1 << 23);
    for (int kk = 0; kk < K; ++kk) {
        launch((unsigned)((N * kGroup + 31) / 32), 32, [&] { k_predict(P, B); });
        launch(mgrid, kThreads, [&] {   // per-warp tables, mask bits from the global array
            if (img && mask)
                fidx ? k_measure<true, true, false, true, true, false>(A) : k_measure<true, true, false, false, true, false>(A);
            else if (img)
                fidx ? k_measure<true, false, false, true, true, false>(A) : k_measure<true, false, false, false, true, false>(A);
            else
                k_measure<false, true, false, false, true, false>(A);
        });
        if (N <= kFinThreads) {
            launch(1, kFinThreads, [&] { k_update_small(P, B); });
        } else {
            const unsigned ub = (unsigned)((N + 127) / 128);
            launch(ub, 128, [&] { k_score(P, B); });
            launch(ub, 128, [&] { k_weights(P, B); });
            launch(1, kFinThreads, [&] { k_finalise(P, B); });
        }
        const size_t n = (size_t)N;
        for (size_t e = 0; e < 6 * n; ++e) tr_poses[kk * 6 * n + e] = pm[e];
        for (size_t e = 0; e < 12 * n; ++e) tr_mom[kk * 12 * n + e] = mom[e];
        for (size_t i = 0; i < n; ++i) {
            tr_s[kk * n + i] = scores[i];
            tr_W[kk * n + i] = W[i];
            tr_idx[kk * n + i] = idx[i];
        }
        for (int d = 0; d < 6; ++d) tr_est[kk * 6 + d] = log[kk % 64].est[d];
    }
}
