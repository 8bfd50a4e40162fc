// Kernel parameter blocks and reduction helpers shared by the .cu files.
#pragma once

#include "common.cuh"

namespace qcgb {

// Index groups of a sweep: `items` groups; a group's base index is the item counter
// with zero bits inserted at pos[0..cnt) (ascending; already shifted down by one when
// neighbouring amplitude pairs are moved together), OR set_mask.  t0/t1 are the masks
// of the gate's target bits.
struct SweepSpec {
  uint64_t items;
  uint64_t set_mask;
  uint64_t t0, t1;
  int cnt;
  int8_t pos[12];
};

template <typename R>
struct Mat2 {
  R m[8];
};
template <typename R>
struct Mat4 {
  R m[32];
};

// Sum over the block (any blockDim multiple of 32, <= 1024); result valid in
// thread 0.  Fixed reduction order.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[32];
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
  if (w == 0) v = warp_sum(v);
  return v;
}

// host entry points shared between translation units (bit positions, not qubits)
qc_status apply_1q_bits(qc_state* s, int tbit, const int* cbits, const int* cvals, int nctrl, const double* U);
qc_status apply_2q_bits(qc_state* s, int pa, int pb, const double* U);
qc_status apply_kq_bits(qc_state* s, const int* bits, int k, const double* U, qc_prec prec);

// Complex128 states of at least 2^kDfMinQubits amplitudes run their arithmetic gate
// sweeps in double-float arithmetic (sweeps_df.cu: FP32 pairs, 48-bit significands,
// no FP64 instruction); smaller ones, where the sweep is launch-bound, keep FP64.
constexpr int kDfMinQubits = 14;
// Entries as (re, im) binary64; low: -1 when bit 0 is not a target, else 1 when the
// first target (qa) is bit 0 and 0 when the second is.
qc_status df_1q_dense(double* a, const SweepSpec& sp, bool vec, bool low, const double* U, unsigned g,
                      cudaStream_t st);
qc_status df_1q_diag(double* a, const SweepSpec& sp, bool vec, bool only1, const double* d0, const double* d1,
                     unsigned g, cudaStream_t st);
qc_status df_1q_anti(double* a, const SweepSpec& sp, bool vec, const double* b, const double* c, unsigned g,
                     cudaStream_t st);
qc_status df_2q_dense(double* a, const SweepSpec& sp, bool vec, int low, const double* U, unsigned g,
                      cudaStream_t st);

}  // namespace qcgb
