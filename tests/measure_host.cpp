// The measurement kernel's per-voxel code compiled for the host through
// tests/host_shim, with the scalar forms of the packed fp32 pairs
// (PF_USE_F32X2 = 0: the packed instructions are, lane by lane, the same IEEE
// operations).  eval_pair, the row set-up and the helpers they use are copied
// verbatim by the test out of measure.cu into measure_voxel.inc and driven
// one target row at a time, two voxels per call, over each row's exact
// inside interval; the per-row sums are folded into whole moments.  Exported
// with a C ABI for tests/test_device_identities.py.  Test infrastructure only.
#include "../paper_2504_19930_gb300/csrc/kernels.h"
#include "host_layouts.h"

#define PF_DEBUG 0
#define PF_USE_F32X2 0
namespace pfreg {
#include "measure_voxel.inc"
}

namespace {
using namespace pfreg;

template <bool IMG, bool MASK, bool FIDX>
void measure_one(const MeasureArgs &a, const float *M, uint64_t mom[12]) {
    constexpr bool BOTH = IMG && MASK;
    const int SX = a.g.sd[0], SY = a.g.sd[1], SZ = a.g.sd[2];
    const int TX = a.g.td[0], TY = a.g.td[1], TZ = a.g.td[2];
    float lo[3], hi[3];
    lo[0] = lo[1] = lo[2] = MASK ? -0.5f : 0.0f;
    hi[0] = MASK ? (float)SX - 0.5f : (float)(SX - 1);
    hi[1] = MASK ? (float)SY - 0.5f : (float)(SY - 1);
    hi[2] = MASK ? (float)SZ - 0.5f : (float)(SZ - 1);
    const float D[3] = {(float)SX, (float)SY, (float)SZ};
    const float r0[3] = {M[0], M[4], M[8]};
    uint64_t n = 0, S1 = 0, ST = 0, T1 = 0, T2 = 0, nn = 0, A = 0, B = 0, C = 0;
    unsigned __int128 S2 = 0;
    for (int z = 0; z < TZ; ++z)
        for (int y = 0; y < TY; ++y) {
            const float dy = __fsub_rn((float)y, a.g.a[1]), dz = __fsub_rn((float)z, a.g.a[2]);
            const float K[3] = {row_K(M[1], M[2], M[3], dy, dz), row_K(M[5], M[6], M[7], dy, dz),
                                row_K(M[9], M[10], M[11], dy, dz)};
            int xb, xe, vb = 0, ve = 0, ib = 0, ie = 0;
            row_interval(r0, K, a.g.a[0], lo, hi, TX, xb, xe);
            if (xb < xe) {
                int xl, xr;
                exact_interval<!MASK>(r0, K, a.g.a[0], D, xb, xe, xl, xr);
                vb = xl;
                ve = xr + 1 > xl ? xr + 1 : xl;
                ib = vb;
                ie = ve;
                if (BOTH && vb < ve) {
                    exact_interval<true>(r0, K, a.g.a[0], D, vb, ve, xl, xr);
                    ib = xl;
                    ie = xr + 1 > xl ? xr + 1 : xl;
                }
            }
            ImgAcc ia;
            MaskAcc ma;
            const uint32_t row0 = (uint32_t)(y + TY * z) * (uint32_t)TX;
            for (int x = vb; x < ve; x += 2) {
                const bool v1 = x + 1 < ve;
                const int x1 = v1 ? x + 1 : x;   // a voxel not taken keeps in-bounds indices
                const PairIn pin{pair((float)x, (float)x1), x, x1, splat(K[0]), splat(K[1]), splat(K[2]),
                                 row0 + (uint32_t)x, row0 + (uint32_t)x1, nullptr, nullptr};
                const bool iv0 = x >= ib && x < ie, iv1 = v1 && x1 >= ib && x1 < ie;
                eval_pair<IMG, MASK, false, false, false, FIDX, false>(a, a.src_bits, nullptr, nullptr, r0[0], r0[1],
                                                                      r0[2], pin, true, v1, iv0, iv1, ia, ma);
            }
            if (IMG) {
                n += (uint64_t)(ie - ib);
                S1 += ia.S1row;
                S2 += ia.S2;
                ST += ia.ST;
                T1 += ia.T1;
                T2 += ia.T2;
            }
            if (MASK) {
                nn += (uint64_t)(ve - vb);
                A += ma.A;
                B += ma.B;
                C += ma.C;
            }
        }
    const uint64_t out[12] = {n, S1, (uint64_t)S2, (uint64_t)(S2 >> 64), ST, T1, T2, 0, nn, A, B, C};
    for (int k = 0; k < 12; ++k) mom[k] = out[k];
}
}  // namespace

// int_index = 1 takes the integer quad index the kernel uses for sources
// above 2^23 voxels, whatever the size; 0 takes the kernel's own choice.
extern "C" void dm_measure(int img, int mask, int int_index, const uint8_t *S, const uint8_t *Smask,
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
    for (int d = 0; d < 3; ++d) {
        a.g.sd[d] = sd[d];
        a.g.td[d] = td[d];
        a.g.a[d] = a_off[d];
    }
    a.P = 1;
    a.fdims[0] = (float)SX;
    a.fdims[1] = (float)((int64_t)SX * SY);
    a.fdims[2] = (float)(SY - 2);
    a.fdims[3] = (float)(SZ - 2);
    const bool fidx = !int_index && ns <= ((size_t)1 << 23);
    for (int p = 0; p < P; ++p) {
        const float *M = mats + 12 * (size_t)p;
        uint64_t *m = mom + 12 * (size_t)p;
        if (img && mask)
            fidx ? measure_one<true, true, true>(a, M, m) : measure_one<true, true, false>(a, M, m);
        else if (img)
            fidx ? measure_one<true, false, true>(a, M, m) : measure_one<true, false, false>(a, M, m);
        else
            measure_one<false, true, false>(a, M, m);
    }
}
