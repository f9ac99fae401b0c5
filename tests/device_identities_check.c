/* Exhaustive checks of the fp32 shortcuts the measurement kernel takes in
 * place of a conversion instruction, against the plain operations the
 * oracle spells out.  Walks every fp32 value of the stated range whose bit
 * pattern is part (mod nparts).
 *
 *   floor:  for 0 <= q < 2^23, the bits of RD(2^23 + q) minus the bits of
 *           2^23 equal floorf(q) (the kernel's floors and nearest-neighbour
 *           indices; RD = rounding toward -infinity);
 *   fixed:  for 0 <= s <= 255, the bits of RN(s + 256) minus the bits of 256
 *           equal lrintf(s * 32768) (the 15-bit fixed-point sample);
 *   byte:   for 0 <= b <= 255, the float with bits 0x4B000000 | b minus 2^23
 *           is (float)b, and the difference of two such biased values is
 *           the difference of the bytes (exact).
 *
 * Usage: device_identities_check PART NPARTS -> "checked N mismatches M".
 * Build with -ffp-contract=off -frounding-math.
 */
#include <fenv.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

static float f_of(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static uint32_t b_of(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

/* volatile keeps each add at run time, in the rounding mode then in force */
static float add_now(float a, float b) {
    volatile float x = a, y = b;
    volatile float r = x + y;
    return r;
}

int main(int argc, char **argv) {
    if (argc < 3) {
        fprintf(stderr, "usage: %s PART NPARTS\n", argv[0]);
        return 2;
    }
    const uint32_t part = (uint32_t)strtoul(argv[1], 0, 10), nparts = (uint32_t)strtoul(argv[2], 0, 10);
    if (nparts == 0 || part >= nparts) return 2;
    const float two23 = 8388608.0f;
    unsigned long long checked = 0, bad = 0;
    /* floor: q in [0, 2^23) */
    fesetround(FE_DOWNWARD);
    for (uint32_t b = part; b < b_of(two23); b += nparts) {
        const float q = f_of(b);
        const uint32_t got = b_of(add_now(two23, q)) - b_of(two23);
        ++checked;
        if (got != (uint32_t)floorf(q)) ++bad;
    }
    fesetround(FE_TONEAREST);
    /* fixed: s in [0, 255] */
    for (uint32_t b = part; b <= b_of(255.0f); b += nparts) {
        const float s = f_of(b);
        const uint32_t got = b_of(add_now(s, 256.0f)) - b_of(256.0f);
        ++checked;
        if ((long)got != lrintf(s * 32768.0f)) ++bad;
    }
    /* byte: every pair of bytes (part 0 only) */
    if (part == 0)
        for (uint32_t x = 0; x < 256; ++x)
            for (uint32_t y = 0; y < 256; ++y) {
                const float A = f_of(0x4B000000u | x), B = f_of(0x4B000000u | y);
                ++checked;
                if (A - two23 != (float)x || B - A != (float)y - (float)x) ++bad;
            }
    printf("checked %llu mismatches %llu\n", checked, bad);
    return 0;
}
