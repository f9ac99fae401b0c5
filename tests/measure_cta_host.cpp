// The measurement kernel k_measure itself -- its blocks of 8 warps, the
// per-warp or per-block (CTAB) x-product tables, the mask bits staged in
// shared memory, the work items of each warp -- copied verbatim by the test
// out of measure.cu into k_measure.inc (its dynamic shared array declared
// here) and run block by block on the host under the emulation of
// tests/host_shim/warp_emulation.h.  Exported with a C ABI for
// tests/test_device_identities.py.  Test infrastructure only.
#include "host_shim/warp_emulation.h"

#include "../paper_2504_19930_gb300/csrc/kernels.h"
#include "host_layouts.h"

dim3 threadIdx, blockIdx, blockDim, gridDim;
#define threadIdx (dim3{(unsigned)host_warp::tid, 1u, 1u})

#define PF_DEBUG 0
#define PF_USE_F32X2 0
namespace pfreg {
float4 smem_dyn[1 << 16];   // the kernel's dynamic shared memory (1 MiB here)
#include "k_measure.inc"
}

namespace {
using namespace pfreg;

template <bool IMG, bool MASK, bool SMEM, bool FIDX, bool XTAB, bool CTAB>
void launch(const MeasureArgs &a) {
    const int rows = a.g.td[1] * a.g.td[2];
    const long long items = (long long)a.P * ((rows + kRowsPerWarp - 1) / kRowsPerWarp);
    const long long per_cta = (long long)kWarps * ipw_of(a.items_per_warp);
    const unsigned grid = (unsigned)((items + per_cta - 1) / per_cta);
    gridDim.x = grid;
    blockDim.x = kThreads;
    for (unsigned b = 0; b < grid; ++b) {
        blockIdx.x = b;
        host_warp::run(kThreads, [&](int) { k_measure<IMG, MASK, SMEM, FIDX, XTAB, CTAB>(a); });
    }
}
template <bool IMG, bool MASK, bool SMEM, bool FIDX>
void by_tab(const MeasureArgs &a, int xtab, int ctab) {
    if (xtab && ctab && MASK)
        launch<IMG, MASK, SMEM, FIDX, true, true>(a);
    else if (xtab)
        launch<IMG, MASK, SMEM, FIDX, true, false>(a);
    else
        launch<IMG, MASK, SMEM, FIDX, false, false>(a);
}
}  // namespace

// Returns 0 after a run, -1 for a shape the kernel is not launched with
// (CTAB needs kWarps * items_per_warp <= row blocks per particle).
extern "C" int dm_k_measure(int img, int mask, int smem_bits, int int_index, int xtab, int ctab, int ipw,
                            const uint8_t *S, const uint8_t *Smask, const int32_t sd[3], const uint8_t *T,
                            const uint8_t *Tmask, const int32_t td[3], const float *mats, int P,
                            const float a_off[3], uint64_t *mom) {
    const int SX = sd[0], SY = sd[1], SZ = sd[2];
    const size_t ns = (size_t)SX * SY * SZ;
    std::vector<uint32_t> quad, bits;
    host_layouts(S, Smask, sd, quad, bits);
    pfreg::MeasureArgs a{};
    a.src_quad = quad.data();
    a.tgt_img = T;
    a.src_bits = bits.data();
    a.tgt_mask = Tmask;
    a.mats = mats;
    a.mom = reinterpret_cast<unsigned long long *>(mom);
    for (int d = 0; d < 3; ++d) {
        a.g.sd[d] = sd[d];
        a.g.td[d] = td[d];
        a.g.a[d] = a_off[d];
    }
    a.P = P;
    a.items_per_warp = ipw;
    a.fdims[0] = (float)SX;
    a.fdims[1] = (float)((int64_t)SX * SY);
    a.fdims[2] = (float)(SY - 2);
    a.fdims[3] = (float)(SZ - 2);
    const int rows = td[1] * td[2];
    const int nblocks = (rows + pfreg::kRowsPerWarp - 1) / pfreg::kRowsPerWarp;
    if (ctab && !(mask && xtab && (long long)pfreg::kWarps * pfreg::ipw_of(ipw) <= nblocks)) return -1;
    const size_t slots = (size_t)pfreg::tab_slots(td[0], img && !mask);
    if (xtab && td[0] > pfreg::kTabMaxX) return -1;
    if ((ctab ? 2 : pfreg::kWarps) * slots + (bits.size() + 3) / 4 + 1 > (size_t)(1 << 16)) return -1;
    for (size_t k = 0; k < 12 * (size_t)P; ++k) mom[k] = 0;
    const bool fidx = !int_index && ns <= ((size_t)1 << 23);
    if (img && mask) {
        if (smem_bits)
            fidx ? by_tab<true, true, true, true>(a, xtab, ctab) : by_tab<true, true, true, false>(a, xtab, ctab);
        else
            fidx ? by_tab<true, true, false, true>(a, xtab, ctab) : by_tab<true, true, false, false>(a, xtab, ctab);
    } else if (img) {
        fidx ? by_tab<true, false, false, true>(a, xtab, 0) : by_tab<true, false, false, false>(a, xtab, 0);
    } else {
        smem_bits ? by_tab<false, true, true, false>(a, xtab, ctab) : by_tab<false, true, false, false>(a, xtab, ctab);
    }
    return 0;
}
