// One batch iteration -- k_predict_batch, k_measure_batch (image, mask and
// combined lists over the members' concatenated work items), k_score_batch,
// k_weights_batch and k_finalise_batch -- copied verbatim by the test out of
// filter.cu and measure.cu into batch_filter.inc and batch_measure.inc (their
// dynamic shared arrays declared here) and run block by block on the host
// under the emulation of tests/host_shim/warp_emulation.h, with the members'
// lists and offsets laid out the way the batch builds them.  Exported with a
// C ABI for tests/test_device_identities.py.  Test infrastructure only.
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
float4 smem_dyn[1 << 16];           // the measurement kernels' dynamic shared memory
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

// One member of the batch, as the test hands it over.  Volumes are host
// arrays (NULL where the mode has none); poses [6][N] enter at iteration k
// (>= 1) and leave resampled; the other arrays are outputs.
struct DmMember {
    int32_t mode, N, k, gamma_log2;
    uint64_t seed, b_full, n_min;
    float lim[6], sigma0_frac, sigma_decay;
    int32_t sd[3], td[3];
    float so[3], ss[3], to[3], ts[3], a[3];
    const uint8_t *src, *src_mask, *tgt, *tgt_mask;
    float *poses, *poses_meas, *mats;
    uint64_t *mom, *W, *C;
    double *scores, *est;
    int32_t *idx;
};

extern "C" void dm_batch_step(DmMember *m, int n, int ipw, int use_tab) {
    std::vector<std::vector<uint32_t>> quads(n), bits(n);
    std::vector<int32_t> kcur(n);
    std::vector<std::vector<IterLog>> logs(n, std::vector<IterLog>(16));
    std::vector<std::vector<unsigned long long>> stats(n, std::vector<unsigned long long>(2, 7ull));
    std::vector<BatchReg> regs(n);
    std::vector<long long> poffs(1, 0), poffs32(1, 0);
    std::vector<int32_t> list[3];
    std::vector<long long> offs[3] = {{0}, {0}, {0}};
    int max_tx[3] = {0, 0, 0};
    for (int r = 0; r < n; ++r) {
        DmMember &M = m[r];
        host_layouts(M.src, M.src_mask, M.sd, quads[r], bits[r]);
        BatchReg &R = regs[r];
        R = BatchReg{};
        FilterParams &P = R.P;
        P.mode = M.mode;
        P.N = M.N;
        P.seed = M.seed;
        P.gamma_log2 = M.gamma_log2;
        P.b_full = M.b_full;
        P.n_min = M.n_min;
        P.log_capacity = 16;
        P.sigma0_frac = M.sigma0_frac;
        P.sigma_decay = M.sigma_decay;
        for (int d = 0; d < 6; ++d) {
            P.lim[d] = M.lim[d];
            P.sig0[d] = (double)M.sigma0_frac * (double)M.lim[d];
        }
        for (int d = 0; d < 3; ++d) {
            P.g.sd[d] = M.sd[d];
            P.g.td[d] = M.td[d];
            P.g.so[d] = M.so[d];
            P.g.ss[d] = M.ss[d];
            P.g.to[d] = M.to[d];
            P.g.ts[d] = M.ts[d];
            P.g.a[d] = M.a[d];
        }
        kcur[r] = M.k;
        FilterBuffers &B = R.B;
        B.poses = M.poses;
        B.poses_meas = M.poses_meas;
        B.mats = M.mats;
        B.mom = reinterpret_cast<unsigned long long *>(M.mom);
        B.scores = M.scores;
        B.W = reinterpret_cast<unsigned long long *>(M.W);
        B.C = reinterpret_cast<unsigned long long *>(M.C);
        B.idx = M.idx;
        B.k = &kcur[r];
        B.log = logs[r].data();
        B.stats = stats[r].data();
        MeasureArgs &A = R.ma;
        A.src_quad = quads[r].data();
        A.tgt_img = M.tgt;
        A.src_bits = bits[r].data();
        A.tgt_mask = M.tgt_mask;
        A.mats = M.mats;
        A.mom = B.mom;
        A.g = P.g;
        A.P = M.N;
        A.items_per_warp = ipw;
        A.fdims[0] = (float)M.sd[0];
        A.fdims[1] = (float)((int64_t)M.sd[0] * M.sd[1]);
        A.fdims[2] = (float)(M.sd[1] - 2);
        A.fdims[3] = (float)(M.sd[2] - 2);
        R.n_iters = M.k + 1;
        R.img = M.mode == 2 || M.mode == 3;
        R.mask = M.mode != 2;
        const int kind = R.img && R.mask ? 2 : (R.img ? 0 : 1);
        list[kind].push_back(r);
        const long long rb = (M.td[1] * M.td[2] + kRowsPerWarp - 1) / kRowsPerWarp;   // row blocks per particle
        offs[kind].push_back(offs[kind].back() + (long long)M.N * rb);
        max_tx[kind] = std::max(max_tx[kind], M.td[0]);
        poffs.push_back(poffs.back() + M.N);
        poffs32.push_back(poffs32.back() + (M.N + 31) / 32 * 32);
    }
    // prediction: 8 lanes per particle, 32 lanes per block
    launch((unsigned)((poffs[n] * kGroup + 31) / 32), 32,
           [&] { k_predict_batch(regs.data(), poffs.data(), n); });
    // measurement: one launch per list
    for (int kind = 0; kind < 3; ++kind) {
        const int nl = (int)list[kind].size();
        if (!nl) continue;
        const long long total = offs[kind][nl];
        const long long per_cta = (long long)kWarps * ipw_of(ipw);
        const int tab_x = use_tab && max_tx[kind] <= kTabMaxX ? max_tx[kind] : 0;
        const unsigned grid = (unsigned)((total + per_cta - 1) / per_cta);
        launch(grid, kThreads, [&] {
            if (kind == 0)
                k_measure_batch<true, false>(regs.data(), list[kind].data(), offs[kind].data(), nl, ipw, tab_x);
            else if (kind == 1)
                k_measure_batch<false, true>(regs.data(), list[kind].data(), offs[kind].data(), nl, ipw, tab_x);
            else
                k_measure_batch<true, true>(regs.data(), list[kind].data(), offs[kind].data(), nl, ipw, tab_x);
        });
    }
    // update: scores and weights over all particles (members padded to whole
    // warps), then one block per member
    const unsigned ub = (unsigned)((poffs32[n] + 127) / 128);
    launch(ub, 128, [&] { k_score_batch(regs.data(), poffs32.data(), n); });
    launch(ub, 128, [&] { k_weights_batch(regs.data(), poffs32.data(), n); });
    launch((unsigned)n, kFinThreads, [&] { k_finalise_batch(regs.data()); });
    for (int r = 0; r < n; ++r) {
        const IterLog &L = logs[r][m[r].k % 16];
        for (int d = 0; d < 6; ++d) m[r].est[d] = L.est[d];
        if (kcur[r] != m[r].k + 1) std::abort();
    }
}
