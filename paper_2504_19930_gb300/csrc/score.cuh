// score.cuh -- similarity scores and likelihood weights from the integer
// moments (device, fixed IEEE operation sequence).
#pragma once
#include "device.cuh"

namespace pfreg {

typedef unsigned __int128 u128;

// 128-bit -> fp64 by the split hi * 2^64 + lo (two round-to-nearest
// conversions, one exact product, one rounded add).
PF_HD double u128_to_f64(u128 v) {
    return d_add(d_mul(u64_to_f64((unsigned long long)(v >> 64)), 18446744073709551616.0),
                 u64_to_f64((unsigned long long)v));
}

// Eq. 2 multiplied through by n^2:
//   NCC^2 = (n ST - S1 T1)^2 / ((n S2 - S1^2)(n T2 - T1^2)),
// the brackets exact in 128-bit integers (S2 is itself a 128-bit sum).
// 0 when n < n_min or a variance is 0.
PF_HD double ncc2_from_moments(unsigned long long n, unsigned long long S1, u128 S2, unsigned long long ST,
                               unsigned long long T1, unsigned long long T2, unsigned long long n_min) {
    if (n == 0 || n < n_min) return 0.0;
    const u128 nS2 = (u128)n * S2, S1S1 = (u128)S1 * S1;
    const u128 nT2 = (u128)n * T2, T1T1 = (u128)T1 * T1;
    if (nS2 <= S1S1 || nT2 <= T1T1) return 0.0;
    const u128 vs = nS2 - S1S1, vt = nT2 - T1T1;
    const u128 nST = (u128)n * ST, S1T1 = (u128)S1 * T1;
    const u128 cv = nST >= S1T1 ? nST - S1T1 : S1T1 - nST;
    const double c = u128_to_f64(cv);
    return d_div(d_mul(c, c), d_mul(u128_to_f64(vs), u128_to_f64(vt)));
}

// Eq. 4 over the whole target grid: 2C / (A + |T|).
PF_HD double dice_from_counts(unsigned long long n, unsigned long long A, unsigned long long C,
                              unsigned long long b_full, unsigned long long n_min) {
    if (n < n_min) return 0.0;
    if (A + b_full == 0) return 0.0;
    return d_div(u64_to_f64(2 * C), u64_to_f64(A + b_full));
}

// mom = [n S1 S2lo S2hi ST T1 T2 0 | n_nn A B C]; modes as pf_mode.
PF_HD double score_from_moments(int mode, const unsigned long long *m, unsigned long long b_full,
                                unsigned long long n_min) {
    const unsigned long long *k = m + 8;
    const u128 S2 = ((u128)m[3] << 64) | (u128)m[2];
    switch (mode) {
    case 0: return dice_from_counts(k[0], k[1], k[3], b_full, n_min);
    case 1: return ncc2_from_moments(k[0], k[1], (u128)k[1], k[3], k[2], k[2], n_min);
    case 2: return ncc2_from_moments(m[0], m[1], S2, m[4], m[5], m[6], n_min);
    case 3:
        return d_mul(0.5, d_add(ncc2_from_moments(m[0], m[1], S2, m[4], m[5], m[6], n_min),
                                dice_from_counts(k[0], k[1], k[3], b_full, n_min)));
    default: return 0.0;
    }
}

// Likelihood (reading): w = (s / s_max)^(2^g) by g squarings, W = floor(w 2^24).
PF_HD unsigned long long quantised_weight(double s, double smax, int g) {
    if (!(smax > 0.0)) return 0ull;
    double r = d_div(s, smax);
    for (int j = 0; j < g; ++j) r = d_mul(r, r);
    return __double2ull_rz(d_mul(r, 16777216.0));
}

}  // namespace pfreg
