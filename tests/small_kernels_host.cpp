// The registration's remaining kernels -- the set-up kernels (k_pack_bits,
// k_binarise, k_count_nonzero), the pose -> matrix export (k_pose_matrix),
// the single-score export (k_score_one) and the estimate's traced Dice
// (k_trace_prepare, k_trace_finish) -- copied verbatim by the test out of
// filter.cu into small_kernels.inc and run on the host under the emulation
// of tests/host_shim/warp_emulation.h.  Exported with a C ABI for
// tests/test_device_identities.py.  Test infrastructure only.
#include "host_shim/warp_emulation.h"

#include "../paper_2504_19930_gb300/csrc/kernels.h"
#include "../paper_2504_19930_gb300/csrc/score.cuh"

dim3 threadIdx, blockIdx, blockDim, gridDim;
#define threadIdx (dim3{(unsigned)host_warp::tid, 1u, 1u})

namespace pfreg {
constexpr int kGroup = 8;   // the lanes of one pose, as in filter.cu
#include "small_kernels.inc"
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

void dm_pack_bits(const uint8_t *mask, int64_t n, uint32_t *bits) {
    launch((unsigned)((n + 31) / 32 + 127) / 128, 128, [&] { pfreg::k_pack_bits(mask, n, bits); });
}
void dm_binarise(const uint8_t *in, uint8_t *out, int64_t n) {
    launch(2, 64, [&] { pfreg::k_binarise(in, out, n); });
}
unsigned long long dm_count_nonzero(const uint8_t *v, int64_t n) {
    unsigned long long c = 0;
    launch(3, 64, [&] { pfreg::k_count_nonzero(v, n, &c); });
    return c;
}
void dm_pose_matrix_kernel(const float pose[6], const int32_t sd[3], const float so[3], const float to[3],
                           const float a_off[3], float M[12]) {
    pfreg::Geometry g{};
    for (int d = 0; d < 3; ++d) {
        g.sd[d] = sd[d];
        g.so[d] = so[d];
        g.to[d] = to[d];
        g.ss[d] = g.ts[d] = 1.0f;
        g.a[d] = a_off[d];
    }
    launch(1, 32, [&] { pfreg::k_pose_matrix(pose, g, M); });
}
double dm_score_one(int mode, const uint64_t mom[12], uint64_t b_full, uint64_t n_min) {
    double out = -1.0;
    launch(1, 32, [&] {
        pfreg::k_score_one(mode, reinterpret_cast<const unsigned long long *>(mom), b_full, n_min, &out);
    });
    return out;
}
// The traced Dice of an estimate est (the log entry of iteration k - 1):
// k_trace_prepare writes the estimate's matrix and zeroes the counts, the
// caller's counts of that matrix (counts [4] = n A B C) stand in for the
// one-particle measurement, k_trace_finish writes the Dice.
void dm_trace(const double est[6], const int32_t sd[3], const float so[3], const float to[3], const float a_off[3],
              uint64_t b_full, float mat_out[12], const uint64_t counts[4], double *dice_out) {
    pfreg::FilterParams P{};
    for (int d = 0; d < 3; ++d) {
        P.g.sd[d] = sd[d];
        P.g.so[d] = so[d];
        P.g.to[d] = to[d];
        P.g.ss[d] = P.g.ts[d] = 1.0f;
        P.g.a[d] = a_off[d];
    }
    P.log_capacity = 4;
    P.b_full = b_full;
    pfreg::IterLog log[4] = {};
    for (int d = 0; d < 6; ++d) log[2].est[d] = est[d];
    int32_t k = 3;
    float mat[12];
    unsigned long long mom[12];
    for (auto &v : mom) v = 99;
    pfreg::FilterBuffers B{};
    B.k = &k;
    B.log = log;
    B.trace_mat = mat;
    B.trace_mom = mom;
    launch(1, 32, [&] { pfreg::k_trace_prepare(P, B); });
    for (int q = 0; q < 12; ++q) {
        mat_out[q] = mat[q];
        if (mom[q] != 0) std::abort();   // the kernel zeroes the counts
    }
    for (int q = 0; q < 4; ++q) mom[8 + q] = counts[q];
    launch(1, 32, [&] { pfreg::k_trace_finish(P, B); });
    *dice_out = log[2].est_dice;
}
}
