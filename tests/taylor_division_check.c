/* Exhaustive check of the division shortcut in the device Taylor chains.
 *
 * The device sin/cos chain divides each term by a constant c_k and takes the
 * quotient as fma(fma(-q, c_k, a), y, q) with q = RN(a * y), y = RN(1 / c_k)
 * (Markstein's correction step) whenever the fp32 angle x has
 * 2^-32 <= |x| <= 64.  This program walks every fp32 x >= 0 in that range
 * whose bit pattern is part (mod nparts), runs both chains (the sine's terms
 * from x, the cosine's from 1, both times -x^2 each step) with the IEEE
 * division, and counts the divisions where the shortcut differs from it.
 * Negative angles need no walk: the terms are odd or even in x and
 * round-to-nearest is symmetric.
 *
 * Usage: taylor_division_check PART NPARTS  -> prints "checked N mismatches M".
 * Build with -ffp-contract=off so that no product is fused.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

int main(int argc, char **argv) {
    if (argc < 3) {
        fprintf(stderr, "usage: %s PART NPARTS\n", argv[0]);
        return 2;
    }
    const uint32_t part = (uint32_t)strtoul(argv[1], 0, 10), nparts = (uint32_t)strtoul(argv[2], 0, 10);
    if (nparts == 0 || part >= nparts) return 2;
    double c[2][14], y[2][14];
    for (int k = 1; k < 14; ++k) {
        c[0][k] = (double)((2 * k) * (2 * k + 1));   /* sine */
        c[1][k] = (double)((2 * k - 1) * (2 * k));   /* cosine */
        y[0][k] = 1.0 / c[0][k];
        y[1][k] = 1.0 / c[1][k];
    }
    const float lo = 0x1p-32f, hi = 64.0f;
    uint32_t blo, bhi;
    memcpy(&blo, &lo, 4);
    memcpy(&bhi, &hi, 4);
    unsigned long long checked = 0, bad = 0;
    for (uint32_t b = blo + part; b <= bhi; b += nparts) {
        float xf;
        memcpy(&xf, &b, 4);
        const double x = (double)xf, mx2 = -(x * x);
        for (int f = 0; f < 2; ++f) {
            double t = f == 0 ? x : 1.0;
            for (int k = 1; k < 14; ++k) {
                const double a = t * mx2;
                const double ref = a / c[f][k];
                const double q = a * y[f][k];
                const double r = __builtin_fma(-q, c[f][k], a);
                const double fast = __builtin_fma(r, y[f][k], q);
                ++checked;
                if (memcmp(&ref, &fast, sizeof ref) != 0) ++bad;
                t = ref;
            }
        }
    }
    printf("checked %llu mismatches %llu\n", checked, bad);
    return 0;
}
