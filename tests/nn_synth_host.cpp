// The proposal network's training-pair parameters -- k_synth_params, which
// draws each pair's pose, heart shape, gain fields and field-of-view shift --
// copied verbatim by the test out of nn.cu into nn_synth.inc and run on the
// host as a loop over its threads (it has no shared memory, barrier or
// shuffle).  Exported with a C ABI for tests/test_device_identities.py.  Test
// infrastructure only.
#include <cmath>
#include <vector>

#include "../paper_2504_19930_gb300/csrc/kernels.h"

dim3 threadIdx, blockIdx, blockDim, gridDim;

namespace pfreg {
namespace nn {
#include "nn_synth.inc"
}
}  // namespace pfreg

using namespace pfreg::nn;

extern "C" {
// B pairs of a batch at optimiser step `step`; per pair the rotation R [9],
// translation t [3], rotation centre c [3], target shift (voxels along x) and
// the label y [6] (pose / limits)
void dm_synth_params(int X, int Y, int Z, float rot_lim, float trans_lim, uint64_t seed, int step, int B, float *R,
                     float *t, float *c, int32_t *shift, float *y) {
    std::vector<SynthSample> s((size_t)B);
    SynthArgs a{};
    a.X = X;
    a.Y = Y;
    a.Z = Z;
    a.G = 64;
    a.rot_lim = rot_lim;
    a.trans_lim = trans_lim;
    a.seed = seed;
    a.step = step;
    a.step_ptr = nullptr;
    a.samples = s.data();
    a.y = y;
    gridDim.x = 1;
    blockDim.x = (unsigned)B;
    blockIdx.x = 0;
    for (int b = 0; b < B; ++b) {
        threadIdx.x = (unsigned)b;
        k_synth_params(a, B);
    }
    for (int b = 0; b < B; ++b) {
        for (int q = 0; q < 9; ++q) R[9 * b + q] = s[b].R[q];
        for (int d = 0; d < 3; ++d) {
            t[3 * b + d] = s[b].t[d];
            c[3 * b + d] = s[b].c[d];
        }
        shift[b] = s[b].shift;
    }
}
}
