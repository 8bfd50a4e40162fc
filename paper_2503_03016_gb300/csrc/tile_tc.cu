// Tile passes with tensor-core stages (QC_PREC_TF32X3, complex64).
//
// A tile of 2^12 amplitudes (the pass's bit set B, as for the CUDA-core passes) goes
// through the pass's stages in shared memory.  A stage owns 5 of the tile's bits (its
// slots); every op of the stage acts on, and is conditioned on, slot bits only, so the
// stage is one 32 x 32 block U_s = G_k ... G_1 (Sec. 3.2's U' of each gate, embedded
// on the slots and multiplied on the host in FP64).  With the 2^7 combinations of the
// tile's other bits as rows, a stage is the real GEMM D = A B of the fused-block
// kernel (A[r][2c + ri] = (re, im) of block index c in row r; B the real form of U_s^T),
// M = 128, N = K = 64, with the TF32 split a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi.
// Both splits round to nearest (hi = RN_tf32(a), lo = RN_tf32(a - hi)): the products
// then err in both directions, so a circuit's hundreds of stages do not drift in norm.
//
// Kernel: one 256-thread CTA per SM; thread t holds half of row t mod 128 (block index
// bit 4 = t / 128 selects the half, which is exactly one 32-column K slice of A).  Per
// stage: gather 16 amplitudes from the swizzled tile, split, store A_hi / A_lo in the
// K-major 128-byte-swizzled layout; one thread issues 3 x 8 tcgen05.mma (kind::tf32),
// each K step's three products into its own TMEM accumulator, and commits them to an
// mbarrier; every thread reads its half-row of the eight partial sums (tcgen05.ld),
// adds them and writes the result back into the tile.  The stages' B images (host-built,
// already in the swizzled layout, 32 KiB each) stream through two shared-memory
// buffers by bulk copies (cp.async.bulk, mbarrier transaction counts): the next
// stage's B lands while this stage computes.  Passes with one or two stages keep them
// resident.  Tiles are double-buffered with cp.async as in the CUDA-core passes.
// Every wait is bounded: on a timeout the kernel sets a status word, waits (bounded)
// for its copies and products in flight, frees its TMEM and returns.
#include <string.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "circuit.cuh"
#include "common.cuh"
#include "kernels.cuh"
#include "tc_common.cuh"
#include "tiles.cuh"

namespace qcgb {

constexpr int kTtM = 12;                        // tile bits
constexpr int kTtL = 4;                         // lowest index bits always in the tile
constexpr int kTtSB = 5;                        // stage (block) bits
constexpr int kTtRows = 1 << (kTtM - kTtSB);    // 128 rows = MMA M
constexpr int kTtThreads = 2 * kTtRows;         // two threads per row (one per K slice)
constexpr int kTtCols = 2 << kTtSB;             // 64 real columns (K = N)
constexpr int kTtAregion = kTtRows * 128;       // one 32-column K slice of A: 16 KiB
constexpr int kTtBregion = kTtCols * 128;       // one 32-column K slice of B: 8 KiB
constexpr int kTtAbytes = 2 * kTtAregion;       // A_hi (or A_lo): 32 KiB
constexpr int kTtBimg = 2 * 2 * kTtBregion;     // B_hi + B_lo of one stage: 32 KiB
constexpr int kTtImgFloats = kTtBimg / 4;
constexpr int kTtTileBytes = (1 << kTtM) * 8;   // complex64 tile: 32 KiB
constexpr int kTtMaxStages = kMaxPassOps;
constexpr int kTtHi = 1 << (kTtM - kTtL);       // 128-byte runs per tile

struct TcStage {
  int32_t img;         // index of the stage's B image
  int8_t slot_bit[5];  // local bit of block-index bit k
  int8_t lane_bit[7];  // local bit receiving bit k of the row index
};
static_assert(sizeof(TcStage) == 16, "TcStage must be 16 bytes");

constexpr size_t kTtSmem = 1024 /* alignment slack */ + 2 * kTtAbytes + 2 * kTtBimg + 2 * kTtTileBytes +
                           kTtHi * sizeof(uint64_t) + kTileNumberTab * sizeof(uint64_t) +
                           kTtMaxStages * sizeof(TcStage) + 64;

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < kTcSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// one bulk copy global -> shared, completion counted in bytes on `bar`
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__global__ void __launch_bounds__(kTtThreads, 1) k_tile_pass_tc(float* __restrict__ amps, const TilePass P,
                                                                 const TcStage* __restrict__ stages,
                                                                 const float* __restrict__ imgs,
                                                                 int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* a_hi = base;
  unsigned char* a_lo = a_hi + kTtAbytes;
  unsigned char* bbuf = a_lo + kTtAbytes;  // two stage images
  Cplx<float>* tiles = reinterpret_cast<Cplx<float>*>(bbuf + 2 * kTtBimg);
  uint64_t* hioff = reinterpret_cast<uint64_t*>(bbuf + 2 * kTtBimg + 2 * kTtTileBytes);
  uint64_t* tnt = hioff + kTtHi;  // tile number -> base
  TcStage* sst = reinterpret_cast<TcStage*>(tnt + kTileNumberTab);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sst + kTtMaxStages);  // products, B buffer 0, B buffer 1
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3);
  __shared__ int8_t sbits[16];
  const int tid = threadIdx.x, warp = tid >> 5;
  constexpr int m = kTtM, L = kTtL;
  constexpr uint32_t T = 1u << m;
  const int S = P.nstages;
  // The tensor cores truncate their FP32 accumulator toward zero after each product
  // step; in one accumulator for all 24 products the last steps, taken at the size of
  // the result, shrink every output a little and a circuit's stages compound it into a
  // norm loss (28-qubit brickwork ~4e-5).  So K step ks accumulates its three products
  // in its own 64 TMEM columns, small products first, and the eight partial sums are
  // added on the CUDA cores with round-to-nearest.
  constexpr int kTmemCols = 512;

  if (tid == 0) {
#pragma unroll
    for (int k = 0; k < 16; ++k) sbits[k] = P.bits[k];
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bars)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bars + 1)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bars + 2)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  for (int i = tid; i < S; i += kTtThreads) sst[i] = stages[P.stage0 + i];
  __syncthreads();
  for (int h = tid; h < kTtHi; h += kTtThreads) {
    uint64_t o = 0;
    for (int k = 0; k < m - L; ++k)
      if ((h >> k) & 1) o |= uint64_t(1) << sbits[L + k];
    hioff[h] = o;
  }
  build_tile_number_tables(tnt, sbits, m, __ffsll(static_cast<long long>(P.ntiles)) - 1);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t mbar = smem_u32(bars);
  const uint32_t bfull = smem_u32(bars + 1);  // buffer b: bfull + 8 b
  constexpr uint32_t idesc = tf32_idesc(kTtRows, kTtCols);

  // B images (thread 0): with one or two stages they stay resident, else buffer g & 1
  // serves stage execution g and the next execution's image is loaded into the other
  const bool resident = S <= 2;
  uint32_t bpar = 0;      // bit b: parity of buffer b's next completion
  uint32_t inflight = 0;  // bit b: a load into buffer b not waited for yet
  auto load_b = [&](int b, int s) {
    bulk_load(smem_u32(bbuf + b * kTtBimg), imgs + size_t(sst[s].img) * kTtImgFloats, kTtBimg, bfull + 8u * b);
    inflight |= 1u << b;
  };
  if (tid == 0 && S > 0) {
    load_b(0, 0);
    if (resident && S == 2) load_b(1, 1);
  }

  uint32_t mpar = 0;
  bool mma_pending = false;  // thread 0: products issued and not yet seen complete
  bool failed = false;
  uint64_t g = 0;
  const uint64_t G = gridDim.x;
  const int row = tid & (kTtRows - 1), half = tid >> 7;
  uint64_t t = blockIdx.x;
  if (t < P.ntiles) prefetch_tile<float>(tiles, amps, tile_base(t, tnt), hioff, L, T);
  cp_async_commit();
  for (int it = 0; t < P.ntiles && !failed; t += G, ++it) {
    Cplx<float>* tile = tiles + (it & 1) * T;
    const uint64_t tbase = tile_base(t, tnt);
    const uint64_t tn = t + G;
    if (tn < P.ntiles)
      prefetch_tile<float>(tiles + ((it + 1) & 1) * T, amps, tile_base(tn, tnt), hioff, L, T);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    for (int s = 0; s < S; ++s, ++g) {
      const TcStage& st = sst[s];
      uint32_t r0 = uint32_t(half) << st.slot_bit[4];
#pragma unroll
      for (int k = 0; k < 7; ++k) r0 |= uint32_t((row >> k) & 1) << st.lane_bit[k];
      uint32_t sw[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) sw[k] = tile_swz(1u << st.slot_bit[k]);
      const uint32_t p0 = tile_swz(r0);
      // this thread's 16 amplitudes (block index c = j + 16 half) -> TF32 hi / lo,
      // two amplitudes per 16-byte chunk of K slice `half`
#pragma unroll
      for (int c4 = 0; c4 < 8; ++c4) {
        const Cplx<float> u = tile[p0 ^ slot_xor<4>(2 * c4, sw)];
        const Cplx<float> v = tile[p0 ^ slot_xor<4>(2 * c4 + 1, sw)];
        const float4 h = make_float4(tf32_rna(u.re), tf32_rna(u.im), tf32_rna(v.re), tf32_rna(v.im));
        const float4 l =
            make_float4(tf32_rna(u.re - h.x), tf32_rna(u.im - h.y), tf32_rna(v.re - h.z), tf32_rna(v.im - h.w));
        const uint32_t o = sw128_offset(row, 32 * half + 4 * c4, kTtRows);
        *reinterpret_cast<float4*>(a_hi + o) = h;
        *reinterpret_cast<float4*>(a_lo + o) = l;
      }
      const int b = resident ? s : int(g & 1);
      bool bad = false;
      if (tid == 0 && ((inflight >> b) & 1u)) {
        bad = !mbar_wait_bounded(bfull + 8u * b, (bpar >> b) & 1u);
        if (!bad) {
          bpar ^= 1u << b;
          inflight &= ~(1u << b);
        }
      }
      // the generic-proxy stores of A become visible to the tensor cores
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      failed = __syncthreads_or(bad ? 1 : 0) != 0;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      if (failed) break;
      if (tid == 0) {
        const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo);
        const uint32_t bh = smem_u32(bbuf + b * kTtBimg), bl = bh + 2 * kTtBregion;
        for (int ks = 0; ks < kTtCols / 8; ++ks) {
          const uint32_t koff = uint32_t((ks & 3) * 32);
          const uint32_t aoff = (ks >> 2) * kTtAregion + koff, boff = (ks >> 2) * kTtBregion + koff;
          const uint32_t d = tmem + uint32_t(64 * ks);
          // the two small products first: only the last accumulation (adding a_hi b_hi)
          // is truncated at the size of the partial sum
          tc_mma(d, sw128_desc(ah + aoff, kTcAtom), sw128_desc(bl + boff, kTcAtom), idesc, 0u);
          tc_mma(d, sw128_desc(al + aoff, kTcAtom), sw128_desc(bh + boff, kTcAtom), idesc, 1u);
          tc_mma(d, sw128_desc(ah + aoff, kTcAtom), sw128_desc(bh + boff, kTcAtom), idesc, 1u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                     : "memory");
        mma_pending = true;
        // the other buffer's last readers (the previous stage's products) are done
        if (!resident) load_b(b ^ 1, s + 1 < S ? s + 1 : 0);
      }
      const bool done = mbar_wait_bounded(mbar, mpar);
      mpar ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      // this thread's half-row of D: TMEM lane `row`, columns 32 half .. 32 half + 31
      {
        const uint32_t ta = tmem + (uint32_t(32 * (warp & 3)) << 16) + uint32_t(32 * half);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          float y[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) y[i] = 0.0f;
#pragma unroll
          for (int ks = 0; ks < 8; ks += 2) {
            uint32_t pa[16], pb[16];  // partial sums of K steps ks and ks + 1
            tmem_ld16(ta + uint32_t(64 * ks + 16 * q), pa);
            tmem_ld16(ta + uint32_t(64 * (ks + 1) + 16 * q), pb);
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
            for (int i = 0; i < 16; ++i) y[i] += __uint_as_float(pa[i]) + __uint_as_float(pb[i]);
          }
#pragma unroll
          for (int j = 0; j < 8; ++j) tile[p0 ^ slot_xor<4>(8 * q + j, sw)] = Cplx<float>{y[2 * j], y[2 * j + 1]};
        }
      }
      // the tile is complete before the next stage gathers, and the TMEM reads are done
      // before the next products overwrite D
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      failed = __syncthreads_or(done ? 0 : 1) != 0;
      if (!failed && tid == 0) mma_pending = false;
      if (failed) break;
    }
    if (failed) break;
    for (uint32_t e = tid; e < T / 2; e += kTtThreads) {
      const uint32_t r = 2 * e;
      const uint64_t gi = tbase | hioff[r >> L] | (r & ((1u << L) - 1));
      const uint32_t p = tile_swz(r);
      st_amp2<float>(amps, gi, tile[p], tile[p ^ 1u]);
    }
    __syncthreads();  // this buffer is refilled two iterations later
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  if (tid == 0) {
    if (failed) atomicExch(status, 1);
    // copies and products still in flight finish before the block leaves (bounded)
    for (int b = 0; b < 2; ++b)
      if ((inflight >> b) & 1u) mbar_wait_bounded(bfull + 8u * b, (bpar >> b) & 1u);
    if (mma_pending) mbar_wait_bounded(mbar, mpar ^ 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
using cd = std::complex<double>;

// nearest TF32 value (ties to even) of a finite fp32 value of modest size
static float tf32_rne_host(float v) {
  uint32_t u;
  memcpy(&u, &v, 4);
  u += 0xFFFu + ((u >> 13) & 1u);
  u &= 0xFFFFE000u;
  float r;
  memcpy(&r, &u, 4);
  return r;
}

// The stages of one pass as 32 x 32 blocks and their B images; false if an op of a
// stage depends on a bit outside the stage's slots (a control or a phase bit elsewhere).
static bool tc_pass_blocks(const BuiltPass& bp, const std::vector<PlanOp>& pops, int n, std::vector<TcStage>& out,
                           std::vector<float>& imgs) {
  int local_of[64];
  for (int b = 0; b < 64; ++b) local_of[b] = -1;
  for (int i = 0; i < kTtM; ++i) local_of[bp.B[i]] = i;
  std::vector<std::vector<int>> takes, acts;
  split_stages(bp, pops, local_of, kTtSB, takes, acts, /*whole_ops=*/true);
  const std::vector<TileStage> recs = stage_layouts(acts, kTtM, kTtSB, 4);
  constexpr int D = 1 << kTtSB;
  for (size_t si = 0; si < takes.size(); ++si) {
    int slot_of_local[16];
    for (int k = 0; k < 16; ++k) slot_of_local[k] = -1;
    for (int k = 0; k < kTtSB; ++k) slot_of_local[recs[si].slot_bit[k]] = k;
    auto slot_of = [&](int gbit) { return local_of[gbit] < 0 ? -1 : slot_of_local[local_of[gbit]]; };
    std::vector<cd> U(D * D, cd(0.0, 0.0));  // U[row * D + col]
    for (int d = 0; d < D; ++d) U[d * D + d] = 1.0;
    for (int idx : takes[si]) {
      const PlanOp& p = pops[idx];
      uint32_t cm = 0, cv = 0;
      for (int b = 0; b < n; ++b) {
        if (!((p.cmask >> b) & 1)) continue;
        const int k = slot_of(b);
        if (k < 0) return false;
        cm |= 1u << k;
        if ((p.cval >> b) & 1) cv |= 1u << k;
      }
      if (p.phase) {
        std::vector<std::pair<int, double>> bs;
        for (const auto& be : p.beta) {
          const int k = slot_of(be.first);
          if (k < 0) return false;
          bs.push_back({k, be.second});
        }
        for (int d = 0; d < D; ++d) {
          if ((uint32_t(d) & cm) != cv) continue;
          double ang = p.c;
          for (const auto& be : bs) ang += ((d >> be.first) & 1) ? be.second : 0.0;
          const cd f = std::polar(1.0, ang);
          for (int c = 0; c < D; ++c) U[d * D + c] *= f;
        }
      } else if (p.nt == 1) {
        const int a = slot_of(p.tb[0]);
        if (a < 0) return false;
        const cd m00(p.m[0], p.m[1]), m01(p.m[2], p.m[3]), m10(p.m[4], p.m[5]), m11(p.m[6], p.m[7]);
        for (int d = 0; d < D; ++d) {
          if ((d >> a) & 1 || (uint32_t(d) & cm) != cv) continue;
          const int d1 = d | (1 << a);
          for (int c = 0; c < D; ++c) {
            const cd u0 = U[d * D + c], u1 = U[d1 * D + c];
            U[d * D + c] = m00 * u0 + m01 * u1;
            U[d1 * D + c] = m10 * u0 + m11 * u1;
          }
        }
      } else {
        const int a = slot_of(p.tb[0]), b2 = slot_of(p.tb[1]);  // row index 2 b_a + b_b
        if (a < 0 || b2 < 0) return false;
        cd M[16];
        for (int e = 0; e < 16; ++e) M[e] = cd(p.m[2 * e], p.m[2 * e + 1]);
        for (int d = 0; d < D; ++d) {
          if ((d >> a) & 1 || (d >> b2) & 1 || (uint32_t(d) & cm) != cv) continue;
          const int ix[4] = {d, d | (1 << b2), d | (1 << a), d | (1 << a) | (1 << b2)};
          for (int c = 0; c < D; ++c) {
            cd x[4];
            for (int i = 0; i < 4; ++i) x[i] = U[ix[i] * D + c];
            for (int i = 0; i < 4; ++i)
              U[ix[i] * D + c] = M[4 * i] * x[0] + M[4 * i + 1] * x[1] + M[4 * i + 2] * x[2] + M[4 * i + 3] * x[3];
          }
        }
      }
    }
    // B image: Bt[n][k] (n = output column, k = input column) of the real form,
    // y_d = sum_c U[d][c] x_c; hi region then lo region, each in the swizzled layout
    TcStage ts{};
    ts.img = int32_t(imgs.size() / kTtImgFloats);
    const size_t o0 = imgs.size();
    imgs.resize(o0 + kTtImgFloats, 0.0f);
    float* hi = imgs.data() + o0;
    float* lo = hi + kTtImgFloats / 2;
    for (int d = 0; d < D; ++d)
      for (int c = 0; c < D; ++c) {
        const double ur = U[d * D + c].real(), ui = U[d * D + c].imag();
        const double vals[4] = {ur, -ui, ui, ur};
        const int ns[4] = {2 * d, 2 * d, 2 * d + 1, 2 * d + 1};
        const int ks[4] = {2 * c, 2 * c + 1, 2 * c, 2 * c + 1};
        for (int e = 0; e < 4; ++e) {
          const float v = float(vals[e]), h = tf32_rne_host(v);
          const uint32_t off = sw128_offset(ns[e], ks[e], kTtCols) / 4;
          hi[off] = h;
          lo[off] = tf32_rne_host(v - h);
        }
      }
    for (int k = 0; k < kTtSB; ++k) ts.slot_bit[k] = recs[si].slot_bit[k];
    for (int k = 0; k < kTtM - kTtSB; ++k) ts.lane_bit[k] = recs[si].lane_bit[k];
    out.push_back(ts);
  }
  return true;
}

qc_status run_tiles_tc(qc_state* s, const std::vector<ResolvedOp>& rops, bool* handled) {
  *handled = false;
  const int n = s->n;
  if (s->dtype != QC_C64 || n < kTtM) return QC_OK;
  std::vector<PlanOp> pops;
  to_plan_ops(rops, pops);
  const std::vector<BuiltPass> bps = build_passes(pops, n, kTtM, kTtL);
  std::vector<TilePass> passes;
  std::vector<TcStage> stages;
  std::vector<float> imgs;
  for (const BuiltPass& bp : bps) {
    TilePass P{};
    P.m = kTtM;
    P.L = kTtL;
    for (int i = 0; i < kTtM; ++i) P.bits[i] = int8_t(bp.B[i]);
    P.ntiles = uint64_t(1) << (n - kTtM);
    P.stage0 = int(stages.size());
    if (!tc_pass_blocks(bp, pops, n, stages, imgs)) return QC_OK;  // the CUDA-core passes take it
    P.nstages = int(stages.size()) - P.stage0;
    if (P.nstages > kTtMaxStages) return QC_OK;
    passes.push_back(P);
  }
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t sb = al(stages.size() * sizeof(TcStage) + 1);
  const size_t ib = imgs.size() * sizeof(float);
  void* scr = nullptr;
  if (qc_status st = state_scratch(s, 256 + sb + ib, &scr)) return st;
  char* base = static_cast<char*>(scr);
  int* status = reinterpret_cast<int*>(base);
  const TcStage* dst = reinterpret_cast<const TcStage*>(base + 256);
  const float* dimg = reinterpret_cast<const float*>(base + 256 + sb);
  std::vector<char> host(sb + ib, 0);
  if (!stages.empty()) memcpy(host.data(), stages.data(), stages.size() * sizeof(TcStage));
  if (ib) memcpy(host.data() + sb, imgs.data(), ib);
  if (qc_status st = check_cuda(cudaMemsetAsync(status, 0, sizeof(int), s->stream), "status reset")) return st;
  if (qc_status st = check_cuda(cudaMemcpyAsync(base + 256, host.data(), host.size(), cudaMemcpyHostToDevice,
                                                s->stream),
                                "tensor-core plan upload"))
    return st;
  auto kern = k_tile_pass_tc;
  if (qc_status st = check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kTtSmem)),
                                "tensor-core tile pass shared memory"))
    return st;
  const uint64_t ntiles = uint64_t(1) << (n - kTtM);
  const unsigned grid = unsigned(std::min<uint64_t>(ntiles, uint64_t(device_sm_count())));
  float* a = reinterpret_cast<float*>(s->amps);
  for (const TilePass& P : passes) {
    QC_COUNT(), kern<<<grid, kTtThreads, kTtSmem, s->stream>>>(a, P, dst, dimg, status);
  }
  if (qc_status st = check_launch("tensor-core tile pass")) return st;
  int h = 0;
  if (qc_status st = check_cuda(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s->stream),
                                "status"))
    return st;
  if (qc_status st = check_cuda(cudaStreamSynchronize(s->stream), "tensor-core tile pass")) return st;
  if (h != 0) {
    set_error("tensor-core tile pass: a bounded wait for a copy or the products ran out");
    return QC_ERR_TIMEOUT;
  }
  g_last_pass_count = int(passes.size());
  g_last_fused_path = 2;
  g_last_stage_count = int(stages.size());
  *handled = true;
  return QC_OK;
}

}  // namespace qcgb
