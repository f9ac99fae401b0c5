// The update step of one filter iteration -- k_update_small (scores,
// weights, estimate and resampling in one block of 1024 threads) and the
// three-kernel form k_score / k_weights / k_finalise -- copied verbatim by
// the test out of filter.cu into update.inc (its one dynamic shared array
// declared here) and run on the host under the block emulation of
// tests/host_shim/warp_emulation.h.  Exported with a C ABI for
// tests/test_device_identities.py.  Test infrastructure only.
#include "host_shim/warp_emulation.h"

#include <climits>

#include "../paper_2504_19930_gb300/csrc/kernels.h"
#include "../paper_2504_19930_gb300/csrc/score.cuh"

dim3 threadIdx, blockIdx, blockDim, gridDim;
#define threadIdx (dim3{(unsigned)host_warp::tid, 1u, 1u})

namespace pfreg {
unsigned long long sh_cdf[12288];   // the kernels' dynamic shared memory (the CDF)
#include "update.inc"
}

namespace {
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

extern "C" {

// One update of a cloud of N particles from their moments (mom [N][12]):
// three_kernels = 1 takes k_score / k_weights / k_finalise whatever N.
// Outputs: scores, W, C, idx [N]; poses [6][N] resampled in place (the
// measured cloud copied to poses_meas); log6 = the iteration's estimate;
// scal = {best, ess}; ints = {best_idx, k after}; evals.
void dm_update(int mode, int N, int gamma_log2, uint64_t b_full, uint64_t n_min, uint64_t seed, int k,
               int three_kernels, const uint64_t *mom, float *poses, float *poses_meas, double *scores,
               uint64_t *W, uint64_t *C, int32_t *idx, double log6[6], double scal[2], int32_t ints[2],
               uint64_t *evals, int estimator, const double *quat) {
    pfreg::FilterParams P{};
    P.mode = mode;
    P.N = N;
    P.gamma_log2 = gamma_log2;
    P.b_full = b_full;
    P.n_min = n_min;
    P.seed = seed;
    P.log_capacity = 16;
    P.estimator = estimator;   // 1: the rotation from the quaternions quat [4][N]
    std::vector<unsigned long long> momv(mom, mom + 12 * (size_t)N), stats(2, 0ull);
    std::vector<pfreg::IterLog> log(16);
    int32_t kk = k;
    pfreg::FilterBuffers B{};
    B.poses = poses;
    B.poses_meas = poses_meas;
    B.mom = momv.data();
    B.scores = scores;
    B.W = reinterpret_cast<unsigned long long *>(W);
    B.C = reinterpret_cast<unsigned long long *>(C);
    B.idx = idx;
    B.k = &kk;
    B.log = log.data();
    B.stats = stats.data();
    B.quat = const_cast<double *>(quat);
    if (N <= pfreg::kFinThreads && !three_kernels) {
        launch(1, pfreg::kFinThreads, [&] { pfreg::k_update_small(P, B); });
    } else {
        const unsigned blocks = (unsigned)((N + 127) / 128);
        launch(blocks, 128, [&] { pfreg::k_score(P, B); });
        launch(blocks, 128, [&] { pfreg::k_weights(P, B); });
        launch(1, pfreg::kFinThreads, [&] { pfreg::k_finalise(P, B); });
    }
    const pfreg::IterLog &L = log[k % 16];
    for (int d = 0; d < 6; ++d) log6[d] = L.est[d];
    scal[0] = L.best;
    scal[1] = L.ess;
    ints[0] = L.best_idx;
    ints[1] = kk;
    *evals = L.evals;
}
}
