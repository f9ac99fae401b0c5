// The sequence warp's per-voxel code (warp.cu: WarpArgs, uint_of, Sample,
// sample_at, sample_frame, which the test copies verbatim into
// warp_sample.inc) compiled for the host through tests/host_shim and driven
// the way k_warp drives it: the pose's matrix from the device functions,
// each row's hoisted offsets and conservative range, then every voxel of the
// row.  Exported with a C ABI for tests/test_device_identities.py.  Test
// infrastructure only.
#include <type_traits>

#include "../paper_2504_19930_gb300/csrc/kernels.h"

#define PF_DEBUG 0
namespace pfreg {
#include "warp_sample.inc"
}

extern "C" void dm_warp(const uint8_t *src, const int32_t sd[3], const float so[3], const float ss[3], uint8_t *out,
                        const int32_t td[3], const float to[3], const float ts[3], const float a_off[3],
                        const float pose[6], int interp) {
    using namespace pfreg;
    WarpArgs a{};
    for (int d = 0; d < 3; ++d) {
        a.g.sd[d] = sd[d];
        a.g.td[d] = td[d];
        a.g.so[d] = so[d];
        a.g.to[d] = to[d];
        a.g.ss[d] = ss[d];
        a.g.ts[d] = ts[d];
        a.g.a[d] = a_off[d];
    }
    for (int j = 0; j < 6; ++j) a.pose[j] = pose[j];
    a.interp = interp;
    a.n_frames = 1;
    float M[12];
    pose_to_matrix(a.pose, a.g, M);
    const float r0[3] = {M[0], M[4], M[8]};
    const float SXf = (float)sd[0], SYf = (float)sd[1], SZf = (float)sd[2];
    float lo[3], hi[3];
    lo[0] = lo[1] = lo[2] = interp ? 0.0f : -0.5f;
    hi[0] = interp ? SXf - 1.0f : SXf - 0.5f;
    hi[1] = interp ? SYf - 1.0f : SYf - 0.5f;
    hi[2] = interp ? SZf - 1.0f : SZf - 0.5f;
    const size_t sx = (size_t)sd[0], sxy = (size_t)sd[0] * (size_t)sd[1];
    for (long long r = 0; r < (long long)td[1] * td[2]; ++r) {
        const int y = (int)(r % td[1]), z = (int)(r / td[1]);
        const float dy = __fsub_rn((float)y, a.g.a[1]), dz = __fsub_rn((float)z, a.g.a[2]);
        const float K[3] = {row_K(M[1], M[2], M[3], dy, dz), row_K(M[5], M[6], M[7], dy, dz),
                            row_K(M[9], M[10], M[11], dy, dz)};
        int xb, xe;
        row_interval(r0, K, a.g.a[0], lo, hi, td[0], xb, xe);
        for (int x = 0; x < td[0]; ++x) {
            Sample<false> s;
            s.valid = false;
            if (x >= xb && x < xe) s = sample_at<false>(a, M, x, K[0], K[1], K[2]);
            out[(size_t)r * td[0] + x] = s.valid ? sample_frame<false>(src, s, interp, sx, sxy) : 0;
        }
    }
}
