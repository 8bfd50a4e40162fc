// tcgen05 helpers shared by the tensor-core kernels (fused blocks, tensor-core tile
// passes): K-major operands in shared memory with the 128-byte swizzle, shared-memory
// matrix and instruction descriptors for kind::tf32, the MMA issue and TMEM loads.
#pragma once

#include <stdint.h>

namespace qcgb {

constexpr int kTcAtom = 1024;                  // swizzle atom: 8 rows x 128 bytes
constexpr long long kTcSpinLimit = 1ll << 24;  // bounded mbarrier waits

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }

// byte offset of element (row, col) (32-bit elements) in a K-major SWIZZLE_128B operand
// with `rows` rows: K slices of 32 columns, each slice rows x 128 bytes
__device__ __host__ __forceinline__ uint32_t sw128_offset(int row, int col, int rows) {
  const int slice = col >> 5;
  const int b = (col & 31) * 4;  // byte within the 128-byte row of the slice
  const int chunk = b >> 4;
  return uint32_t(slice * rows * 128 + (row >> 3) * kTcAtom + (row & 7) * 128 + ((chunk ^ (row & 7)) << 4) +
                  (b & 15));
}

// sm_100 shared-memory matrix descriptor: start address, leading byte offset, stride
// byte offset (between 8-row groups), version 1, layout SWIZZLE_128B (2)
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr, uint32_t sbo) {
  uint64_t d = 0;
  d |= uint64_t((saddr & 0x3FFFF) >> 4);
  d |= uint64_t(16 >> 4) << 16;
  d |= uint64_t(sbo >> 4) << 32;
  d |= uint64_t(1) << 46;
  d |= uint64_t(2) << 61;
  return d;
}

// instruction descriptor: D = F32, A = B = TF32, both K-major, N, M
__host__ __device__ constexpr uint32_t tf32_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtm),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

}  // namespace qcgb
