// The measurement kernel's warp routine measure_item -- row set-up, the
// sweep of the 32 rows' intervals in passes of 64 voxels (row-crossing
// passes included), the per-voxel code and the warp reduction with its
// atomics -- together with the warp's x-product table (build_xtab), copied
// verbatim by the test out of measure.cu into measure_item.inc and
// measure_xtab.inc, run on the host by a lockstep emulation of one warp
// (tests/host_shim/warp_emulation.h), the packed fp32 pairs in their scalar
// form.  The emulated warp takes the work items one after the other, as a
// warp of k_measure with the per-warp table does.  Exported with a C ABI for
// tests/test_device_identities.py.  Test infrastructure only.
#include "host_shim/warp_emulation.h"

#include "../paper_2504_19930_gb300/csrc/kernels.h"
#include "host_layouts.h"

#ifndef PF_DEBUG
#define PF_DEBUG 0   // -DPF_DEBUG=1: the debug build's gather bounds checks
#endif
#define PF_USE_F32X2 0
namespace pfreg {
#include "measure_item.inc"
#include "measure_xtab.inc"
}

namespace {
using namespace pfreg;

template <bool IMG, bool MASK, bool FIDX, bool XTAB>
void run_warp(const MeasureArgs &a) {
    constexpr bool PAIRED = paired_tab<IMG, MASK>();
    const int TX = a.g.td[0];
    std::vector<float4> tabmem((size_t)tab_slots(TX, PAIRED) + 1);
    float4 *tab = XTAB ? tabmem.data() : nullptr;
    float2 *tabz = XTAB ? reinterpret_cast<float2 *>(tab + TX) : nullptr;
    const int rows = a.g.td[1] * a.g.td[2];
    const int nblocks = (rows + kRowsPerWarp - 1) / kRowsPerWarp;
    const long long items = (long long)a.P * nblocks;
    host_warp::run([&](int l) {
        int tab_p = -1;
        for (long long item = 0; item < items; ++item) {
            if (XTAB) {
                const int p = (int)(item / nblocks);
                if (p != tab_p) {
                    build_xtab<PAIRED>(tab, tabz, TX, a.g.a[0], a.mats + 12 * (size_t)p, l);
                    tab_p = p;
                }
            }
            measure_item<IMG, MASK, FIDX, XTAB>(a, a.src_bits, tab, tabz, item, l);
        }
    });
}

template <bool IMG, bool MASK, bool FIDX>
void run_tab(const MeasureArgs &a, bool xtab) {
    if (xtab)
        run_warp<IMG, MASK, FIDX, true>(a);
    else
        run_warp<IMG, MASK, FIDX, false>(a);
}
}  // namespace

// mom [P][12] is zeroed here and accumulated by the emulated warp's atomics.
// int_index = 1 takes the integer quad index whatever the source size;
// xtab = 1 reads the coordinates' x products from the warp's table.
extern "C" void dm_measure_warp(int img, int mask, int int_index, int xtab, const uint8_t *S, const uint8_t *Smask,
                                const int32_t sd[3], const uint8_t *T, const uint8_t *Tmask, const int32_t td[3],
                                const float *mats, int P, const float a_off[3], uint64_t *mom) {
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
    a.fdims[0] = (float)SX;
    a.fdims[1] = (float)((int64_t)SX * SY);
    a.fdims[2] = (float)(SY - 2);
    a.fdims[3] = (float)(SZ - 2);
    for (size_t k = 0; k < 12 * (size_t)P; ++k) mom[k] = 0;
    const bool fidx = !int_index && ns <= ((size_t)1 << 23);
    const bool xt = xtab != 0;
    if (img && mask)
        fidx ? run_tab<true, true, true>(a, xt) : run_tab<true, true, false>(a, xt);
    else if (img)
        fidx ? run_tab<true, false, true>(a, xt) : run_tab<true, false, false>(a, xt);
    else
        run_tab<false, true, false>(a, xt);
}

// Out-of-bounds gather indices the debug build's checks recorded (0 in the
// release build, which has no checks).
extern "C" unsigned long long dm_debug_hits() {
#if PF_DEBUG
    return pfreg::g_dbg_hits;
#else
    return 0;
#endif
}

// fp32 lane operations executed so far (with -DPF_HOST_COUNT_FP32), reset by
// dm_fp32_ops_reset.
extern "C" unsigned long long dm_fp32_ops() {
#ifdef PF_HOST_COUNT_FP32
    return g_host_fp32_ops;
#else
    return 0;
#endif
}
extern "C" void dm_fp32_ops_reset() {
#ifdef PF_HOST_COUNT_FP32
    g_host_fp32_ops = 0;
#endif
}
