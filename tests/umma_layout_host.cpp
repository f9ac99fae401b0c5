// The tensor-core path's operand-layout arithmetic (umma.cuh: the byte
// offset of an element in a K-major no-swizzle tile, the shared-memory and
// instruction descriptors) compiled for the host through tests/host_shim, so
// the test can check them against the layout the descriptors describe.
// Exported with a C ABI for tests/test_device_identities.py.  Test
// infrastructure only.
#include "cuda_runtime.h"

// never called here: the shared-window conversion the descriptors start from
inline uint64_t __cvta_generic_to_shared(const void *) { return 0; }

#include "../paper_2504_19930_gb300/csrc/umma.cuh"

extern "C" {
uint32_t dm_tile_offset(int r, int k, int kcols) { return pfreg::umma::tile_offset(r, k, kcols); }
uint64_t dm_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) { return pfreg::umma::smem_desc(addr, lbo, sbo); }
uint32_t dm_idesc(int M, int N) { return pfreg::umma::idesc_bf16_f32(M, N); }
}
