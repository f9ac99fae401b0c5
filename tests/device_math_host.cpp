// The device headers' scalar arithmetic (fp64 sin/cos chain, pose -> matrix,
// Philox; scores and quantised weights from the integer moments) compiled for
// the host through tests/host_shim, exported with a C ABI for
// tests/test_device_identities.py.  Test infrastructure only.
#include "../paper_2504_19930_gb300/csrc/device.cuh"
#include "../paper_2504_19930_gb300/csrc/score.cuh"

extern "C" {

double dm_sincos(float x, int cosine) { return pfreg::taylor_sincos(x, cosine != 0); }

void dm_pose_matrix(const float pose[6], const int32_t sd[3], const float so[3], const float ss[3],
                    const float to[3], const float ts[3], float M[12]) {
    pfreg::Geometry g{};
    for (int d = 0; d < 3; ++d) {
        g.sd[d] = sd[d];
        g.so[d] = so[d];
        g.ss[d] = ss[d];
        g.to[d] = to[d];
        g.ts[d] = ts[d];
    }
    pfreg::pose_to_matrix(pose, g, M);
}

void dm_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const pfreg::u32x4 r = pfreg::philox10(pfreg::u32x4{ctr[0], ctr[1], ctr[2], ctr[3]}, key[0], key[1]);
    out[0] = r.x;
    out[1] = r.y;
    out[2] = r.z;
    out[3] = r.w;
}

double dm_score(int mode, const uint64_t mom[12], uint64_t b_full, uint64_t n_min) {
    return pfreg::score_from_moments(mode, reinterpret_cast<const unsigned long long *>(mom), b_full, n_min);
}

uint64_t dm_weight(double s, double smax, int g) { return pfreg::quantised_weight(s, smax, g); }
}
