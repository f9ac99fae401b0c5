// The source layouts the measurement kernel reads, built on the host for the
// host-compiled tests: quads Q[x,y,z] = S[x,y,z] | S[x+1,y,z] << 8 |
// S[x,y+1,z] << 16 | S[x+1,y+1,z] << 24 (0 past the grid; the layout
// k_pack_quads writes) and mask bits (bit i & 31 of word i >> 5; the layout
// k_pack_bits writes).  S or Smask may be NULL (that layout stays zero).
// Test infrastructure only.
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>

inline void host_layouts(const uint8_t *S, const uint8_t *Smask, const int32_t sd[3], std::vector<uint32_t> &quad,
                         std::vector<uint32_t> &bits) {
    const int SX = sd[0], SY = sd[1], SZ = sd[2];
    const size_t ns = (size_t)SX * SY * SZ;
    quad.assign(ns, 0u);
    bits.assign((ns + 31) / 32, 0u);
    for (size_t i = 0; i < ns; ++i) {
        const int x = (int)(i % SX), y = (int)((i / SX) % SY);
        const bool xn = x + 1 < SX, yn = y + 1 < SY;
        const uint32_t b0 = S ? S[i] : 0u, b1 = S && xn ? S[i + 1] : 0u;
        const uint32_t b2 = S && yn ? S[i + SX] : 0u, b3 = S && xn && yn ? S[i + SX + 1] : 0u;
        quad[i] = b0 | (b1 << 8) | (b2 << 16) | (b3 << 24);
        if (Smask && Smask[i]) bits[i >> 5] |= 1u << (i & 31);
    }
}
