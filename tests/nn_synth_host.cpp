// The proposal network's synthetic training pairs -- k_synth_params (each
// pair's pose, heart shape, gain fields and field-of-view shift) and
// k_synth_views (both views box-averaged into the network input), with the
// CUDA-core helpers they use -- copied verbatim by the test out of nn.cu into
// nn_small.inc and nn_synth.inc and run on the host under the emulation of
// tests/host_shim/warp_emulation.h.  dm_synth_full evaluates the kernels'
// own per-voxel function synth_voxel over the full-resolution grids, so the
// test can box-average them with the oracle.  Exported with a C ABI for
// tests/test_device_identities.py.  Test infrastructure only.
#include "host_shim/warp_emulation.h"

#include <vector>

#include "../paper_2504_19930_gb300/csrc/kernels.h"
#include "host_shim/nn_device.h"

dim3 threadIdx, blockIdx, blockDim, gridDim;
#define threadIdx (dim3{(unsigned)host_warp::tid, 1u, 1u})

namespace pfreg {
namespace nn {
#include "nn_small.inc"
#include "nn_synth.inc"
}
}  // namespace pfreg

using namespace pfreg::nn;

namespace {
std::vector<SynthSample> g_samples;

SynthArgs args(int X, int Y, int Z, int G, float rot_lim, float trans_lim, uint64_t seed, int step, int B,
               float *y, uint16_t *x) {
    g_samples.assign((size_t)B, SynthSample{});
    SynthArgs a{};
    a.X = X;
    a.Y = Y;
    a.Z = Z;
    a.G = G;
    a.rot_lim = rot_lim;
    a.trans_lim = trans_lim;
    a.seed = seed;
    a.step = step;
    a.step_ptr = nullptr;
    a.samples = g_samples.data();
    a.x = x;
    a.y = y;
    gridDim = dim3{(unsigned)((B + 31) / 32), 1u, 1u};
    blockDim = dim3{32u, 1u, 1u};
    for (unsigned b = 0; b < gridDim.x; ++b) {
        blockIdx = dim3{b, 0u, 0u};
        host_warp::run(32, [&](int) { k_synth_params(a, B); });
    }
    return a;
}
}  // namespace

extern "C" {
// B pairs of a batch at optimiser step `step`; per pair the rotation R [9],
// translation t [3], rotation centre c [3], target shift (voxels along x) and
// the label y [6] (pose / limits)
void dm_synth_params(int X, int Y, int Z, float rot_lim, float trans_lim, uint64_t seed, int step, int B, float *R,
                     float *t, float *c, int32_t *shift, float *y) {
    args(X, Y, Z, 64, rot_lim, trans_lim, seed, step, B, y, nullptr);
    for (int b = 0; b < B; ++b) {
        const SynthSample &s = g_samples[b];
        for (int q = 0; q < 9; ++q) R[9 * b + q] = s.R[q];
        for (int d = 0; d < 3; ++d) {
            t[3 * b + d] = s.t[d];
            c[3 * b + d] = s.c[d];
        }
        shift[b] = s.shift;
    }
}
// The network input x [B][G^3][2] (bf16 bits) of the same batch.
void dm_synth_views(int X, int Y, int Z, int G, float rot_lim, float trans_lim, uint64_t seed, int step, int B,
                    float *y, uint16_t *x) {
    const SynthArgs a = args(X, Y, Z, G, rot_lim, trans_lim, seed, step, B, y, x);
    const long long cells = (long long)G * G * G;
    gridDim = dim3{(unsigned)((cells + 255) / 256), (unsigned)B, 1u};
    blockDim = dim3{256u, 1u, 1u};
    for (unsigned b = 0; b < gridDim.y; ++b)
        for (unsigned bx = 0; bx < gridDim.x; ++bx) {
            blockIdx = dim3{bx, b, 0u};
            host_warp::run(256, [&](int) { k_synth_views(a); });
        }
}
// Pair b of the batch at full resolution: the source view S [Z][Y][X] at
// world (x, y, z) and the target view T [Z][Y][X], whose voxel p sits at
// source-grid x = p + shift and shows the tissue at R (x - c) + c + t, each
// voxel from synth_voxel with the grid fractions k_synth_views passes.
void dm_synth_full(int X, int Y, int Z, float rot_lim, float trans_lim, uint64_t seed, int step, int B, int b,
                   float *S, float *T) {
    std::vector<float> y(6 * (size_t)B);
    args(X, Y, Z, 64, rot_lim, trans_lim, seed, step, B, y.data(), nullptr);
    const SynthSample &s = g_samples[b];
    const float inv[3] = {1.0f / X, 1.0f / Y, 1.0f / Z};
    for (int z = 0; z < Z; ++z)
        for (int yy = 0; yy < Y; ++yy)
            for (int x = 0; x < X; ++x) {
                const size_t v = ((size_t)z * Y + yy) * X + x;
                const float ws[3] = {(float)x, (float)yy, (float)z};
                const float us[3] = {x * inv[0], yy * inv[1], z * inv[2]};
                S[v] = synth_voxel(s, 0, ws, us);
                const float q[3] = {(float)(x + s.shift) - s.c[0], (float)yy - s.c[1], (float)z - s.c[2]};
                float wt[3];
                for (int r = 0; r < 3; ++r)
                    wt[r] = s.R[3 * r] * q[0] + s.R[3 * r + 1] * q[1] + s.R[3 * r + 2] * q[2] + s.c[r] + s.t[r];
                const float ut[3] = {x * inv[0], yy * inv[1], z * inv[2]};
                T[v] = synth_voxel(s, 1, wt, ut);
            }
}
}
