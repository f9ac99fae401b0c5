// Kernels without shared memory, barriers or shuffles -- the initial clouds
// (k_init, k_seed_gaussian, copied verbatim by the test out of filter.cu
// into filter_init.inc) and the quad packing of image sources (k_pack_quads,
// out of measure.cu into pack_quads.inc) -- run on the host through
// tests/host_shim as a loop over their threads.  Exported with a C ABI for
// tests/test_device_identities.py.  Test infrastructure only.
#include "../paper_2504_19930_gb300/csrc/kernels.h"

dim3 threadIdx, blockIdx, blockDim, gridDim;

namespace pfreg {
#include "filter_init.inc"
#include "pack_quads.inc"
}

namespace {
// every thread of a launch of `blocks` x `threads`, one after the other
template <class F>
void run_threads(unsigned blocks, unsigned threads, F &&body) {
    gridDim.x = blocks;
    blockDim.x = threads;
    for (unsigned b = 0; b < blocks; ++b)
        for (unsigned t = 0; t < threads; ++t) {
            blockIdx.x = b;
            threadIdx.x = t;
            body();
        }
}
pfreg::FilterParams params(int N, uint64_t seed, const float lim[6]) {
    pfreg::FilterParams P{};
    P.N = N;
    P.seed = seed;
    for (int d = 0; d < 6; ++d) P.lim[d] = lim[d];
    return P;
}
}  // namespace

extern "C" {

void dm_init(int N, uint64_t seed, const float lim[6], float *poses) {
    const pfreg::FilterParams P = params(N, seed, lim);
    run_threads((N + 255) / 256, 256, [&] { pfreg::k_init(P, poses); });
}

void dm_seed(int N, uint64_t seed, const float lim[6], const float mean[6], const float sdev[6], float *poses) {
    const pfreg::FilterParams P = params(N, seed, lim);
    pfreg::Seed6 s;
    for (int d = 0; d < 6; ++d) {
        s.m[d] = mean[d];
        s.s[d] = sdev[d];
    }
    run_threads((N + 255) / 256, 256, [&] { pfreg::k_seed_gaussian(P, poses, s); });
}

void dm_pack_quads(const uint8_t *S, const int32_t dims[3], uint32_t *Q) {
    run_threads(3, 64, [&] { pfreg::k_pack_quads(S, dims[0], dims[1], dims[2], Q); });
}
}
