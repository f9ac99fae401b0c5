// The sequence-warp kernel k_warp (each block builds the pose's matrix in
// shared memory from six lanes' sin/cos, then walks target rows, sampling
// up to 64 frames per voxel, four at a time), copied verbatim by the test
// out of warp.cu into k_warp.inc and run block by block on the host under
// the emulation of tests/host_shim/warp_emulation.h.  Exported with a C ABI
// for tests/test_device_identities.py.  Test infrastructure only.
#include "host_shim/warp_emulation.h"

#include <type_traits>

#include "../paper_2504_19930_gb300/csrc/kernels.h"

dim3 threadIdx, blockIdx, blockDim, gridDim;
#define threadIdx (dim3{(unsigned)host_warp::tid, 1u, 1u})

#ifndef PF_DEBUG
#define PF_DEBUG 0   // -DPF_DEBUG=1: the debug build's gather bounds checks
#endif
namespace pfreg {
#include "k_warp.inc"
}

// frames: n_frames source volumes of sd (consecutive), out: n_frames target
// volumes of td; wide = 1 takes the 64-bit-offset form of the kernel.
extern "C" void dm_k_warp(const uint8_t *frames, int n_frames, const int32_t sd[3], const float so[3],
                          const float ss[3], uint8_t *out, const int32_t td[3], const float to[3], const float ts[3],
                          const float a_off[3], const float pose[6], int interp, int wide, int blocks) {
    using namespace pfreg;
    WarpArgs a{};
    const size_t ns = (size_t)sd[0] * sd[1] * sd[2], nt = (size_t)td[0] * td[1] * td[2];
    for (int f = 0; f < n_frames; ++f) {
        a.f.in[f] = frames + f * ns;
        a.f.out[f] = out + f * nt;
    }
    for (int j = 0; j < 6; ++j) a.pose[j] = pose[j];
    for (int d = 0; d < 3; ++d) {
        a.g.sd[d] = sd[d];
        a.g.td[d] = td[d];
        a.g.so[d] = so[d];
        a.g.to[d] = to[d];
        a.g.ss[d] = ss[d];
        a.g.ts[d] = ts[d];
        a.g.a[d] = a_off[d];
    }
    a.interp = interp;
    a.n_frames = n_frames;
    gridDim.x = (unsigned)blocks;
    blockDim.x = kWarpThreads;
    for (int b = 0; b < blocks; ++b) {
        blockIdx.x = (unsigned)b;
        host_warp::run(kWarpThreads, [&](int) {
            if (wide)
                k_warp<true>(a);
            else
                k_warp<false>(a);
        });
    }
}

// Out-of-bounds gather indices the debug build's checks recorded.
extern "C" unsigned long long dm_debug_hits() {
#if PF_DEBUG
    return pfreg::g_wdbg_hits;
#else
    return 0;
#endif
}
