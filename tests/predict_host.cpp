// The prediction kernel k_predict (perturbation, the shared sin/cos chain,
// pose -> matrix; 8 lanes per particle exchanging values by shuffles),
// copied verbatim by the test out of filter.cu into predict.inc, run on the
// host warp by warp under the lockstep emulation of
// tests/host_shim/warp_emulation.h.  Exported with a C ABI for
// tests/test_device_identities.py.  Test infrastructure only.
#include "host_shim/warp_emulation.h"

#include "../paper_2504_19930_gb300/csrc/kernels.h"

dim3 threadIdx, blockIdx, blockDim, gridDim;
// under the emulation every lane sees its own thread index
#define threadIdx (dim3{(unsigned)host_warp::tid, 1u, 1u})

namespace pfreg {
#include "predict.inc"
}

// N a multiple of 4 (whole warps of 4 particles x 8 lanes); poses [6][N] in
// and out (perturbed for k > 0), mats [N][12] out; with estimator = 1 also
// each pose's quaternion, quat [4][N].
extern "C" void dm_predict(int N, int k, uint64_t seed, const float lim[6], float sigma0_frac, float decay,
                           const int32_t sd[3], const float so[3], const float ss[3], const int32_t td[3],
                           const float to[3], const float ts[3], const float a_off[3], float *poses, float *mats,
                           int estimator, double *quat) {
    pfreg::FilterParams P{};
    P.N = N;
    P.seed = seed;
    P.sigma0_frac = sigma0_frac;
    P.sigma_decay = decay;
    P.estimator = estimator;
    for (int d = 0; d < 6; ++d) {
        P.lim[d] = lim[d];
        P.sig0[d] = (double)sigma0_frac * (double)lim[d];
    }
    for (int d = 0; d < 3; ++d) {
        P.g.sd[d] = sd[d];
        P.g.so[d] = so[d];
        P.g.ss[d] = ss[d];
        P.g.td[d] = td[d];
        P.g.to[d] = to[d];
        P.g.ts[d] = ts[d];
        P.g.a[d] = a_off[d];
    }
    std::vector<unsigned long long> mom((size_t)N * pfreg::kMomStride, 1ull), stats(2, 1ull);
    int32_t kk = k;
    pfreg::FilterBuffers B{};
    B.poses = poses;
    B.mats = mats;
    B.mom = mom.data();
    B.stats = stats.data();
    B.k = &kk;
    B.quat = quat;
    blockDim.x = 32;
    gridDim.x = (unsigned)(N * 8 / 32);
    for (unsigned b = 0; b < gridDim.x; ++b) {
        blockIdx.x = b;
        host_warp::run([&](int) { pfreg::k_predict(P, B); });
    }
    for (unsigned long long v : mom)   // the kernel zeroes the moment accumulators
        if (v) std::abort();
}
