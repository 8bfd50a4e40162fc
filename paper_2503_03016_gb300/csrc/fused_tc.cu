// Fused k-qubit blocks on the tensor cores (QC_PREC_TF32X3, complex64).
//
// A block U (2^k x 2^k, Sec. 3.2's U' for k qubits) maps each group of 2^k amplitudes
// that differ only in the block's bits: out_d = sum_c U[d][c] in_c.  With the groups as
// rows this is one real GEMM D = A B over interleaved (re, im) columns:
//   A[r][2c + ri] = (re, im)_ri of amplitude (row r, column c),
//   B[2c][2d] = Ur[d][c], B[2c+1][2d] = -Ui[d][c], B[2c][2d+1] = Ui[d][c], B[2c+1][2d+1] = Ur[d][c].
// TF32 keeps 10 mantissa bits, so each product is split as
//   a*b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi,  a_hi = a with the low 13 mantissa bits
// cleared, a_lo = a - a_hi (exact), the same for b; the three products accumulate in
// FP32 in tensor memory (TMEM).
//
// Kernel shape (k = 5: K = N = 64 real columns): one CTA of 128 threads handles tiles of
// 128 rows.  Threads gather their row's 32 amplitudes (8-byte loads, coalesced across
// the warp when index bit 0 is a row bit), split them and store A_hi / A_lo in the
// canonical K-major layout with the 128-byte swizzle (8-row x 128-byte atoms, 16-byte
// chunk c of row r at c ^ (r mod 8)).  One elected thread issues 3 x 8 tcgen05.mma
// (M=128, N=64, K=8, kind::tf32) and commits them to an mbarrier; every thread waits
// (bounded), reads its row of D from TMEM (tcgen05.ld 32x32b) and scatters it back.  B_hi /
// B_lo stay in shared memory for the whole launch.  Smaller blocks (k < 5) are padded
// with identity qubits.
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "circuit.cuh"
#include "common.cuh"
#include "kernels.cuh"
#include "tc_common.cuh"

namespace qcgb {

constexpr int kTcK = 5;                     // block qubits
constexpr int kTcCols = 2 << kTcK;          // 64 real columns (K = N)
constexpr int kTcRows = 128;                // rows per tile (MMA M)
constexpr int kTcAregion = kTcRows * 128;   // one 32-float K slice of A: 16 KiB
constexpr int kTcBregion = kTcCols * 128;   // one 32-float K slice of B: 8 KiB
constexpr int kTcKslices = kTcCols / 32;    // 2
// shared memory: A_hi, A_lo (2 x 32 KiB), B_hi, B_lo (2 x 16 KiB), offsets, barrier
constexpr int kTcSmem = 2 * kTcKslices * kTcAregion + 2 * kTcKslices * kTcBregion + 1024 + 1024;

// bsplit: [B_hi (64x64)][B_lo (64x64)] fp32, then 32 uint64 column offsets, then 5 int32
// ascending block bit positions (row -> index: zero bits inserted there)
__global__ void __launch_bounds__(kTcRows, 1) k_block_tc(float* __restrict__ amps, uint64_t ntiles,
                                                         const float* __restrict__ bsplit, int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned regions (the swizzle pattern is taken from address bits 4..9)
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* a_hi = base;
  unsigned char* a_lo = a_hi + kTcKslices * kTcAregion;
  unsigned char* b_hi = a_lo + kTcKslices * kTcAregion;
  unsigned char* b_lo = b_hi + kTcKslices * kTcBregion;
  uint64_t* offs = reinterpret_cast<uint64_t*>(b_lo + kTcKslices * kTcBregion);  // 32 column offsets
  uint64_t* bar = offs + 32;  // 8-byte aligned
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
  int8_t* spos = reinterpret_cast<int8_t*>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // B_hi / B_lo (host-split, [n][k] row-major fp32) into the swizzled K-major layout
  for (int i = tid; i < kTcCols * kTcCols; i += blockDim.x) {
    const int n = i / kTcCols, k = i % kTcCols;
    *reinterpret_cast<float*>(b_hi + sw128_offset(n, k, kTcCols)) = bsplit[i];
    *reinterpret_cast<float*>(b_lo + sw128_offset(n, k, kTcCols)) = bsplit[kTcCols * kTcCols + i];
  }
  const uint64_t* goffs = reinterpret_cast<const uint64_t*>(bsplit + 2 * kTcCols * kTcCols);
  const int* gpos = reinterpret_cast<const int*>(goffs + 32);
  if (tid < 32) offs[tid] = goffs[tid];
  if (tid < kTcK) spos[tid] = int8_t(gpos[tid]);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(64)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  constexpr uint32_t idesc = tf32_idesc(kTcRows, kTcCols);
  uint32_t phase = 0;
  bool failed = false;

  // software pipeline, two tiles deep: a thread's rows of tile t live in one of two
  // register buffers; right after they are split into shared memory that buffer is
  // refilled with tile t + 2 grid, so the gathers of the next two tiles are in flight
  // while the tensor cores and the epilogue work on tile t
  const uint64_t G = gridDim.x;
  auto gather = [&](float2 (&x)[32], uint64_t& rb, uint64_t t) {
    rb = insert_zero_bits(t * kTcRows + tid, spos, kTcK);
#pragma unroll
    for (int c = 0; c < 32; ++c) x[c] = reinterpret_cast<const float2*>(amps)[rb | offs[c]];
  };
  auto step = [&](float2 (&x)[32], uint64_t& rb, uint64_t t) {
    // split this thread's row (in registers) into hi / lo; amplitudes 2c and 2c+1 fill
    // one 16-byte chunk of the swizzled layout, written with one 16-byte store (a warp's
    // stores then take the minimum number of shared-memory wavefronts)
    auto hi = [](float v) { return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u); };
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const float2 u = x[2 * c], v = x[2 * c + 1];
      const float4 h = make_float4(hi(u.x), hi(u.y), hi(v.x), hi(v.y));
      const uint32_t o = sw128_offset(tid, 4 * c, kTcRows);  // start of the chunk
      *reinterpret_cast<float4*>(a_hi + o) = h;
      *reinterpret_cast<float4*>(a_lo + o) = make_float4(u.x - h.x, u.y - h.y, v.x - h.z, v.y - h.w);
    }
    // make the generic-proxy shared-memory writes visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (tid == 0) {
      const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi), bl = smem_u32(b_lo);
      int first = 1;
      for (int prod = 0; prod < 3; ++prod) {
        const uint32_t A = prod == 2 ? al : ah;
        const uint32_t B = prod == 1 ? bl : bh;
        for (int ks = 0; ks < kTcCols / 8; ++ks) {
          const uint32_t koff = uint32_t((ks & 3) * 32);  // 8 tf32 = 32 bytes per K step
          const uint64_t ad = sw128_desc(A + (ks >> 2) * kTcAregion + koff, kTcAtom);
          const uint64_t bd = sw128_desc(B + (ks >> 2) * kTcBregion + koff, kTcAtom);
          tc_mma(tmem, ad, bd, idesc, first ? 0u : 1u);
          first = 0;
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_u32(bar))
                   : "memory");
    }
    // the buffer is free: gather tile t + 2 grid into it (disjoint rows, own tiles)
    const uint64_t rb_cur = rb;
    if (t + 2 * G < ntiles) gather(x, rb, t + 2 * G);
    // bounded wait for the products
    {
      uint32_t done = 0;
      for (long long it = 0; it < kTcSpinLimit; ++it) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(phase)
            : "memory");
        if (done) break;
      }
      // block-uniform outcome
      failed = __syncthreads_or(done ? 0 : 1) != 0;
      if (failed && tid == 0) atomicExch(status, 1);
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (!failed) {
      // row tid of D: TMEM lane tid, 64 columns, stored 16 columns (8 amplitudes) at a time
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t r[16];
        tmem_ld16(tmem + (uint32_t(warp * 32) << 16) + uint32_t(q * 16), r);
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
        for (int i = 0; i < 8; ++i)
          reinterpret_cast<float2*>(amps)[rb_cur | offs[q * 8 + i]] =
              make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
      }
    }
    // one barrier: the epilogue's TMEM reads are done before the next tile's products
    // overwrite the accumulator, and a timed-out block stops; the others stop at their
    // next tile (block-uniform test)
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    failed = __syncthreads_or(*((volatile int*)status) != 0) != 0;
  };
  float2 xa[32], xb[32];
  uint64_t rba = 0, rbb = 0;
  const uint64_t t0 = blockIdx.x;
  if (t0 < ntiles) gather(xa, rba, t0);
  if (t0 + G < ntiles) gather(xb, rbb, t0 + G);
  for (uint64_t t = t0; t < ntiles && !failed; t += 2 * G) {
    step(xa, rba, t);
    if (t + G < ntiles && !failed) step(xb, rbb, t + G);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(64) : "memory");
  (void)lane;
}

// Six-qubit blocks (k = 6): rows of 64 amplitudes, K = N = 128 real columns.  B (128 x
// 128, hi and lo: 128 KiB) stays in shared memory for the launch; A would need another
// 128 KiB, so it passes through one 64 KiB buffer in two K halves: the threads holding
// block-index bit 5 = 0 store their half of every row (K slices 0, 1), one thread issues
// that half's 3 x 8 products (M = N = 128, K = 8) into the accumulator, and after they
// complete the other threads store K slices 2, 3 for the second half.  256 threads, two
// per row (thread t: row t mod 128, block-index bit 5 = t / 128).
constexpr int k6K = 6;
constexpr int k6Cols = 2 << k6K;                    // 128
constexpr int k6Aregion = kTcRows * 128;            // one K slice of A: 16 KiB
constexpr int k6Bregion = k6Cols * 128;             // one K slice of B: 16 KiB
constexpr int k6Smem = 2 * 2 * k6Aregion /* A_hi, A_lo: two slices each */ +
                       2 * 4 * k6Bregion /* B_hi, B_lo: four slices each */ + 1024 + 1024;

__global__ void __launch_bounds__(2 * kTcRows, 1) k_block_tc6(float* __restrict__ amps, uint64_t ntiles,
                                                              const float* __restrict__ bsplit,
                                                              int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* a_hi = base;
  unsigned char* a_lo = a_hi + 2 * k6Aregion;
  unsigned char* b_hi = a_lo + 2 * k6Aregion;
  unsigned char* b_lo = b_hi + 4 * k6Bregion;
  uint64_t* offs = reinterpret_cast<uint64_t*>(b_lo + 4 * k6Bregion);  // 64 column offsets
  uint64_t* bar = offs + 64;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
  int8_t* spos = reinterpret_cast<int8_t*>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & (kTcRows - 1), half = tid >> 7;

  for (int i = tid; i < k6Cols * k6Cols; i += blockDim.x) {
    const int n = i / k6Cols, k = i % k6Cols;
    *reinterpret_cast<float*>(b_hi + sw128_offset(n, k, k6Cols)) = bsplit[i];
    *reinterpret_cast<float*>(b_lo + sw128_offset(n, k, k6Cols)) = bsplit[k6Cols * k6Cols + i];
  }
  const uint64_t* goffs = reinterpret_cast<const uint64_t*>(bsplit + 2 * k6Cols * k6Cols);
  const int* gpos = reinterpret_cast<const int*>(goffs + 64);
  if (tid < 64) offs[tid] = goffs[tid];
  if (tid < k6K) spos[tid] = int8_t(gpos[tid]);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(k6Cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  constexpr uint32_t idesc = tf32_idesc(kTcRows, k6Cols);
  uint32_t phase = 0;
  bool failed = false;
  auto hi = [](float v) { return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u); };

  // software pipeline, two tiles deep (as for five-qubit blocks): once a thread's half
  // row of tile t is in the A buffer, its register buffer is refilled with tile t + 2 grid
  const uint64_t G = gridDim.x;
  auto gather = [&](float2 (&x)[32], uint64_t& rb, uint64_t t) {
    rb = insert_zero_bits(t * kTcRows + row, spos, k6K);
#pragma unroll
    for (int j = 0; j < 32; ++j) x[j] = reinterpret_cast<const float2*>(amps)[rb | offs[32 * half + j]];
  };
  auto step = [&](float2 (&x)[32], uint64_t& rb, uint64_t t) {
    const uint64_t rb_cur = rb;
    for (int h = 0; h < 2 && !failed; ++h) {
      if (half == h) {
        // K columns 64 h .. 64 h + 63 of this row: slices 0 and 1 of the A buffer
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const float2 u = x[2 * c], v = x[2 * c + 1];
          const float4 hv = make_float4(hi(u.x), hi(u.y), hi(v.x), hi(v.y));
          const uint32_t o = sw128_offset(row, 4 * c, kTcRows);
          *reinterpret_cast<float4*>(a_hi + o) = hv;
          *reinterpret_cast<float4*>(a_lo + o) = make_float4(u.x - hv.x, u.y - hv.y, v.x - hv.z, v.y - hv.w);
        }
        if (t + 2 * G < ntiles) gather(x, rb, t + 2 * G);  // the buffer is free
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      if (tid == 0) {
        const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi), bl = smem_u32(b_lo);
        for (int prod = 0; prod < 3; ++prod) {
          const uint32_t A = prod == 2 ? al : ah;
          const uint32_t B = prod == 1 ? bl : bh;
          for (int ks = 0; ks < 8; ++ks) {
            const uint32_t koff = uint32_t((ks & 3) * 32);
            const uint64_t ad = sw128_desc(A + (ks >> 2) * k6Aregion + koff, kTcAtom);
            const uint64_t bd = sw128_desc(B + (2 * h + (ks >> 2)) * k6Bregion + koff, kTcAtom);
            tc_mma(tmem, ad, bd, idesc, (h == 0 && prod == 0 && ks == 0) ? 0u : 1u);
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         smem_u32(bar))
                     : "memory");
      }
      // bounded wait for this half's products (they read the A buffer the next half
      // overwrites, and the accumulator the epilogue reads)
      uint32_t done = 0;
      for (long long it = 0; it < kTcSpinLimit; ++it) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(phase)
            : "memory");
        if (done) break;
      }
      phase ^= 1u;
      failed = __syncthreads_or(done ? 0 : 1) != 0;
      if (failed && tid == 0) atomicExch(status, 1);
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    }
    if (failed) return;
    // row `row` of D, the 64 columns of this thread's outputs (block index 32 half + j)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t r[16];
      tmem_ld16(tmem + (uint32_t(32 * (warp & 3)) << 16) + uint32_t(64 * half + 16 * q), r);
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
      for (int i = 0; i < 8; ++i)
        reinterpret_cast<float2*>(amps)[rb_cur | offs[32 * half + 8 * q + i]] =
            make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
    }
    // the epilogue's TMEM reads end before the next tile's products overwrite D
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    failed = __syncthreads_or(*((volatile int*)status) != 0) != 0;
  };
  float2 xa[32], xb[32];
  uint64_t rba = 0, rbb = 0;
  const uint64_t t0 = blockIdx.x;
  if (t0 < ntiles) gather(xa, rba, t0);
  if (t0 + G < ntiles) gather(xb, rbb, t0 + G);
  for (uint64_t t = t0; t < ntiles && !failed; t += 2 * G) {
    step(xa, rba, t);
    if (t + G < ntiles && !failed) step(xb, rbb, t + G);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(k6Cols) : "memory");
}

// host: real form of U on kq qubits (row-major Bt[n][k], 2^(kq+1) columns), split hi / lo
static void tc_bmatrix(const std::vector<double>& U5, std::vector<float>& out, int kq = kTcK) {
  const int D = 1 << kq, C = 2 << kq;
  out.assign(2 * C * C, 0.0f);
  auto hi_of = [](float v) {
    uint32_t u;
    memcpy(&u, &v, 4);
    u &= 0xFFFFE000u;
    float h;
    memcpy(&h, &u, 4);
    return h;
  };
  for (int d = 0; d < D; ++d)
    for (int c = 0; c < D; ++c) {
      const double ur = U5[2 * (d * D + c)], ui = U5[2 * (d * D + c) + 1];
      // Bt[n][k] with n = output column, k = input column
      const float vals[4] = {float(ur), float(-ui), float(ui), float(ur)};
      const int ns[4] = {2 * d, 2 * d, 2 * d + 1, 2 * d + 1};
      const int ks[4] = {2 * c, 2 * c + 1, 2 * c, 2 * c + 1};
      for (int e = 0; e < 4; ++e) {
        const float v = vals[e], h = hi_of(v);
        out[ns[e] * C + ks[e]] = h;
        out[C * C + ns[e] * C + ks[e]] = v - h;
      }
    }
}

// k = 6: the whole 64 x 64 block (no padding) through k_block_tc6
static qc_status apply_k6_tf32x3(qc_state* s, const int* bits, const double* U) {
  if (s->dtype != QC_C64 || s->n < k6K + 7) {
    set_error("TF32x3 six-qubit blocks need complex64 and n >= %d", k6K + 7);
    return QC_ERR_UNSUPPORTED;
  }
  constexpr int D = 1 << k6K;
  std::vector<double> U6(U, U + 2 * D * D);
  std::vector<float> bs;
  tc_bmatrix(U6, bs, k6K);
  // column c of a row (block index c, bits[0] its MSB) sits at offset off[c]; rows
  // enumerate the other bits (zeros inserted at the block's bits, ascending)
  std::vector<int> sorted(bits, bits + k6K);
  std::sort(sorted.begin(), sorted.end());
  {
    const size_t nb = bs.size();
    bs.resize(nb + 64 * 2 + k6K);
    uint64_t o64[64];
    for (int r = 0; r < D; ++r) {
      uint64_t off = 0;
      for (int j = 0; j < k6K; ++j)
        if ((r >> (k6K - 1 - j)) & 1) off |= uint64_t(1) << bits[j];
      o64[r] = off;
    }
    memcpy(bs.data() + nb, o64, sizeof(o64));
    int p32[k6K];
    for (int j = 0; j < k6K; ++j) p32[j] = sorted[j];
    memcpy(bs.data() + nb + 128, p32, sizeof(p32));
  }
  void* scr = nullptr;
  const size_t bbytes = sizeof(float) * bs.size();
  if (qc_status st = state_scratch(s, 256 + bbytes, &scr)) return st;
  int* status = reinterpret_cast<int*>(scr);
  float* dB = reinterpret_cast<float*>(static_cast<char*>(scr) + 256);
  if (qc_status st = check_cuda(cudaMemsetAsync(status, 0, sizeof(int), s->stream), "status reset")) return st;
  if (qc_status st = check_cuda(cudaMemcpyAsync(dB, bs.data(), bbytes, cudaMemcpyHostToDevice, s->stream), "B upload"))
    return st;
  if (qc_status st = check_cuda(cudaFuncSetAttribute(k_block_tc6, cudaFuncAttributeMaxDynamicSharedMemorySize, k6Smem),
                                "tc6 smem"))
    return st;
  const uint64_t ntiles = (state_len(s) >> k6K) / kTcRows;
  const unsigned grid = unsigned(std::min<uint64_t>(ntiles, uint64_t(device_sm_count())));
  QC_COUNT(), k_block_tc6<<<grid, 2 * kTcRows, k6Smem, s->stream>>>(reinterpret_cast<float*>(s->amps), ntiles, dB,
                                                                    status);
  if (qc_status st = check_launch("tensor-core six-qubit block")) return st;
  int h = 0;
  if (qc_status st = check_cuda(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s->stream), "status"))
    return st;
  if (qc_status st = check_cuda(cudaStreamSynchronize(s->stream), "tensor-core six-qubit block")) return st;
  return device_status(h, "tensor-core block");
}

qc_status apply_kq_tf32x3(qc_state* s, const int* bits, int k, const double* U) {
  if (k == k6K) return apply_k6_tf32x3(s, bits, U);
  if (s->dtype != QC_C64 || k < 1 || k > kTcK || s->n < kTcK + 7) {
    set_error("TF32x3 blocks need complex64, k <= %d and n >= %d", kTcK, kTcK + 7);
    return QC_ERR_UNSUPPORTED;
  }
  bool handled = false;
  if (qc_status st = apply_block_tile_tc(s, bits, k, U, &handled)) return st;
  if (handled) return QC_OK;
  // pad with the lowest bits not in the block: U5 = U (x) I on (bits..., extra...)
  int b5[kTcK];
  for (int j = 0; j < k; ++j) b5[j] = bits[j];
  int kk = k;
  for (int b = 0; kk < kTcK && b < s->n; ++b) {
    bool used = false;
    for (int j = 0; j < kk; ++j) used |= (b5[j] == b);
    if (!used) b5[kk++] = b;
  }
  const int D = 1 << kTcK, Dk = 1 << k, Dp = 1 << (kTcK - k);
  std::vector<double> U5(2 * D * D, 0.0);
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) {
      if ((r % Dp) != (c % Dp)) continue;
      const int rr = r / Dp, cc = c / Dp;
      U5[2 * (r * D + c)] = U[2 * (rr * Dk + cc)];
      U5[2 * (r * D + c) + 1] = U[2 * (rr * Dk + cc) + 1];
    }
  std::vector<float> bs;
  tc_bmatrix(U5, bs);
  KqSpec sp{};
  std::vector<int> sorted(b5, b5 + kTcK);
  std::sort(sorted.begin(), sorted.end());
  sp.cnt = kTcK;
  for (int j = 0; j < kTcK; ++j) sp.pos[j] = int8_t(sorted[j]);
  for (int r = 0; r < D; ++r) {
    uint64_t off = 0;
    for (int j = 0; j < kTcK; ++j)
      if ((r >> (kTcK - 1 - j)) & 1) off |= uint64_t(1) << b5[j];
    sp.off[r] = off;
  }
  // device buffers: status word + split B + offsets + positions, in the state's scratch
  {
    const size_t nb = bs.size();
    bs.resize(nb + 32 * 2 + kTcK);
    uint64_t o64[32];
    for (int r = 0; r < 32; ++r) o64[r] = sp.off[r];
    memcpy(bs.data() + nb, o64, sizeof(o64));
    int p32[kTcK];
    for (int j = 0; j < kTcK; ++j) p32[j] = sp.pos[j];
    memcpy(bs.data() + nb + 64, p32, sizeof(p32));
  }
  void* scr = nullptr;
  const size_t bbytes = sizeof(float) * bs.size();
  if (qc_status st = state_scratch(s, 256 + bbytes, &scr)) return st;
  int* status = reinterpret_cast<int*>(scr);
  float* dB = reinterpret_cast<float*>(static_cast<char*>(scr) + 256);
  if (qc_status st = check_cuda(cudaMemsetAsync(status, 0, sizeof(int), s->stream), "status reset")) return st;
  if (qc_status st = check_cuda(cudaMemcpyAsync(dB, bs.data(), bbytes, cudaMemcpyHostToDevice, s->stream), "B upload"))
    return st;
  if (qc_status st = check_cuda(cudaFuncSetAttribute(k_block_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem),
                                "tc smem"))
    return st;
  const uint64_t ntiles = (state_len(s) >> kTcK) / kTcRows;
  const unsigned grid = unsigned(std::min<uint64_t>(ntiles, uint64_t(device_sm_count()) * 2));
  QC_COUNT(), k_block_tc<<<grid, kTcRows, kTcSmem, s->stream>>>(reinterpret_cast<float*>(s->amps), ntiles, dB, status);
  if (qc_status st = check_launch("tensor-core block")) return st;
  int h = 0;
  if (qc_status st = check_cuda(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s->stream), "status"))
    return st;
  if (qc_status st = check_cuda(cudaStreamSynchronize(s->stream), "tensor-core block")) return st;
  return device_status(h, "tensor-core block");
}

}  // namespace qcgb
