// The measurement kernel's row set-up compiled for the host through
// tests/host_shim: the conservative x-range of a target row (row_interval,
// device.cuh) and its exact inside interval (coord1 / axis_conds /
// exact_interval, which the test copies verbatim out of measure.cu into
// measure_row_interval.inc).  Exported with a C ABI for
// tests/test_device_identities.py.  Test infrastructure only.
#include "../paper_2504_19930_gb300/csrc/device.cuh"

namespace pfreg {
#include "measure_row_interval.inc"
}

extern "C" {

// For every row (y, z) of the target grid, the visited interval [xl, xr]
// (xr < xl: empty) as the kernel sets it up: nearest-neighbour bounds
// (0 <= q + 0.5 < D) with tri = 0, trilinear bounds (0 <= q <= D - 1) with
// tri = 1.  Rows are z-major: row = y + TY z.
void dm_row_intervals(const float M[12], const float a[3], const int32_t sd[3], const int32_t td[3], int tri,
                      int32_t *xl_out, int32_t *xr_out) {
    using namespace pfreg;
    float lo[3], hi[3];
    const float D[3] = {(float)sd[0], (float)sd[1], (float)sd[2]};
    for (int d = 0; d < 3; ++d) {
        lo[d] = tri ? 0.0f : -0.5f;
        hi[d] = tri ? (float)(sd[d] - 1) : (float)sd[d] - 0.5f;
    }
    const float r0[3] = {M[0], M[4], M[8]};
    for (int z = 0; z < td[2]; ++z)
        for (int y = 0; y < td[1]; ++y) {
            const float dy = __fsub_rn((float)y, a[1]);
            const float dz = __fsub_rn((float)z, a[2]);
            const float K[3] = {row_K(M[1], M[2], M[3], dy, dz), row_K(M[5], M[6], M[7], dy, dz),
                                row_K(M[9], M[10], M[11], dy, dz)};
            int xb, xe, xl = 0, xr = -1;
            row_interval(r0, K, a[0], lo, hi, td[0], xb, xe);
            if (xb < xe) {
                if (tri)
                    exact_interval<true>(r0, K, a[0], D, xb, xe, xl, xr);
                else
                    exact_interval<false>(r0, K, a[0], D, xb, xe, xl, xr);
            }
            xl_out[y + td[1] * z] = xl;
            xr_out[y + td[1] * z] = xr;
        }
}
}
