// Fused reverse sweep of the adjoint gradient (qc_adjoint_grad).
//
// The reverse sweep applies U_L^dag, ..., U_1^dag to psi and lambda and records, just
// before a rotation U_l = exp(-i t_l G_l / 2) is undone, g_l = Im <lambda|G_l|psi>.  The
// daggered gates in reverse order form a circuit like any other, so the tile planner
// splits them into passes; this kernel runs a pass on BOTH states at once: it loads the
// same tile (the same index bits) of psi and of lambda, applies every gate of the pass
// to both in shared memory, and before each recorded rotation adds the tile's share of
// Im <lambda|G|psi> -- a sum over the tile's amplitudes -- to that rotation's sum.  A
// gate moved by the planner past gates it commutes with leaves the record unchanged:
// Im <A lambda|G|A psi> = Im <lambda|G|psi> when the unitary A commutes with G.  Both
// states then move once each way per pass instead of once per gate.
//
// Sums: each thread forms its share at the state's precision, a warp adds the 32
// shares at that precision too, and each warp keeps one running sum per recorded
// rotation in shared memory -- complex64: a pair of FP32 numbers (hi, lo) updated by
// Knuth's TwoSum (TAOCP Vol. 2, Sec. 4.2.2), so that the sum keeps about 48 bits
// without an FP64 instruction (GB300 runs FP64 at 2 operations per clock per SM);
// complex128: FP64.  At the end every block writes its per-rotation totals (FP64), which
// are reduced over blocks in a fixed order (deterministic).
#include <string.h>

#include <algorithm>
#include <vector>

#include "adjoint_tiles.cuh"
#include "circuit.cuh"
#include "common.cuh"
#include "kernels.cuh"
#include "tiles.cuh"
#include "tiles_df.cuh"

namespace qcgb {

// complex64 reverse passes: record shares kept pending per thread before their warp sums
constexpr int kAdjPend = 8;

// running per-warp sum of a recorded rotation's shares
template <typename R>
struct GradAcc;
template <>
struct GradAcc<float> {
  using T = float2;  // the sum is hi + lo
  __device__ static T zero() { return make_float2(0.0f, 0.0f); }
  __device__ static void add(T& a, float x) {
    const float s = __fadd_rn(a.x, x);
    const float bb = __fsub_rn(s, a.x);
    const float err = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    a.x = s;
    a.y = __fadd_rn(a.y, err);
  }
  __device__ static double value(T a) { return double(a.x) + double(a.y); }
};
template <>
struct GradAcc<double> {
  using T = double;
  __device__ static T zero() { return 0.0; }
  __device__ static void add(T& a, double x) { a += x; }
  __device__ static double value(T a) { return a; }
};

// Share of Im <w|Z_b|v> where bit b is register slot KS (>= 0) or reads `fixed` for
// every amplitude of the thread (KS = -1): the signs are known at compile time.
template <typename R, int SB, int KS>
__device__ __forceinline__ R grad_z(const Cplx<R> (&v)[1 << SB], const Cplx<R> (&w)[1 << SB], uint32_t fixed) {
  R pos = R(0), neg = R(0);
#pragma unroll
  for (int j = 0; j < (1 << SB); ++j) {
    const R x = im_conj_mul(w[j], v[j]);
    if (KS >= 0 && ((j >> KS) & 1))
      neg += x;
    else
      pos += x;
  }
  if (KS < 0) return fixed ? -pos : pos;
  return pos - neg;
}

template <typename R, int SB>
__device__ __forceinline__ R grad_z_at(int ks, const Cplx<R> (&v)[1 << SB], const Cplx<R> (&w)[1 << SB],
                                       uint32_t fixed) {
  switch (ks) {
    case 0: return grad_z<R, SB, 0>(v, w, fixed);
    case 1: return grad_z<R, SB, 1>(v, w, fixed);
    case 2:
      if constexpr (SB > 2) return grad_z<R, SB, 2>(v, w, fixed);
      return R(0);
    case 3:
      if constexpr (SB > 3) return grad_z<R, SB, 3>(v, w, fixed);
      return R(0);
    case 4:
      if constexpr (SB > 4) return grad_z<R, SB, 4>(v, w, fixed);
      return R(0);
    default: return grad_z<R, SB, -1>(v, w, fixed);
  }
}

// Im(conj(a) b)
template <typename R>
__device__ __forceinline__ R im_conj_mul(Cplx<R> a, Cplx<R> b) {
  return a.re * b.im - a.im * b.re;
}

// Share of Im <w|G|v> over the pairs along slot S0: G = X: (Gv)_0 = v_1, (Gv)_1 = v_0;
// G = Y: (Gv)_0 = -i v_1, (Gv)_1 = i v_0.
template <typename R, int SB, int S0>
__device__ __forceinline__ R grad_pairs(const Cplx<R> (&v)[1 << SB], const Cplx<R> (&w)[1 << SB], int gen) {
  R acc = R(0);
#pragma unroll
  for (int j = 0; j < (1 << SB); ++j) {
    if (j & (1 << S0)) continue;
    const int j1 = j | (1 << S0);
    if (gen == 0) {
      acc += im_conj_mul(w[j], v[j1]) + im_conj_mul(w[j1], v[j]);
    } else {
      const Cplx<R> g0{v[j1].im, -v[j1].re}, g1{-v[j].im, v[j].re};
      acc += im_conj_mul(w[j], g0) + im_conj_mul(w[j1], g1);
    }
  }
  return acc;
}

template <typename R, int SB>
__device__ __forceinline__ R grad_pairs_at(int s0, const Cplx<R> (&v)[1 << SB], const Cplx<R> (&w)[1 << SB],
                                           int gen) {
  switch (s0) {
    case 0: return grad_pairs<R, SB, 0>(v, w, gen);
    case 1: return grad_pairs<R, SB, 1>(v, w, gen);
    case 2: return grad_pairs<R, SB, 2>(v, w, gen);
    case 3:
      if constexpr (SB > 3) return grad_pairs<R, SB, 3>(v, w, gen);
      return R(0);
    default:
      if constexpr (SB > 4) return grad_pairs<R, SB, 4>(v, w, gen);
      return R(0);
  }
}

// The warp's sums of its kAdjPend pending record shares (this thread's share of record
// k at pend[k * NT + thread]; record k's slot among the pass's records in slots[k]; the
// first cnt are valid), added into the warp's running sums acc[slot].  A transposing
// reduction: at offset 16 each lane keeps the half of the records its lane bit 4 names
// and adds its partner's copy of that half, then at 8 and 4 the same on the halves left,
// and the single record a lane then holds (k = lane / 4) is summed over offsets 2 and 1.
template <int NT>
__device__ __forceinline__ void flush_records_impl(const float* pend, const int16_t* slots, int cnt, int lane,
                                                   float2* acc) {
  __syncwarp();
  const int tid = threadIdx.x;
  float x[kAdjPend];
#pragma unroll
  for (int k = 0; k < kAdjPend; ++k) x[k] = k < cnt ? pend[k * NT + tid] : 0.0f;
  const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0, b2 = (lane & 4) != 0;
  float y[4], z[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float keep = b4 ? x[4 + i] : x[i], send = b4 ? x[i] : x[4 + i];
    y[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float keep = b3 ? y[2 + i] : y[i], send = b3 ? y[i] : y[2 + i];
    z[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  float u = (b2 ? z[1] : z[0]) + __shfl_xor_sync(0xffffffffu, b2 ? z[0] : z[1], 4);
  u += __shfl_xor_sync(0xffffffffu, u, 2);
  u += __shfl_xor_sync(0xffffffffu, u, 1);
  const int k = lane >> 2;
  if ((lane & 3) == 0 && k < cnt) GradAcc<float>::add(acc[slots[k]], u);
  __syncwarp();
}

template <typename R, int NT, int SB>
__global__ void __launch_bounds__(NT, 1) k_adj_pass(R* __restrict__ psi, R* __restrict__ lam, const TilePass P,
                                                    const TileStage* __restrict__ stages,
                                                    const TileOp* __restrict__ ops, const R* __restrict__ pool,
                                                    const R* __restrict__ mats, double* __restrict__ gpart) {
  constexpr int NA = 1 << SB;
  constexpr int NW = NT / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = P.m, L = P.L;
  const uint32_t T = 1u << m;
  Cplx<R>* bufs = reinterpret_cast<Cplx<R>*>(smem_raw);  // psi: 2 x T, lambda: 2 x T
  uint64_t* hioff = reinterpret_cast<uint64_t*>(smem_raw + 4 * sizeof(Cplx<R>) * T);
  const int nhi = m - L;
  uint64_t* tnt = hioff + (1u << nhi);  // tile number -> base
  TileStage* sst = reinterpret_cast<TileStage*>(tnt + kTileNumberTab);
  TileOp* sop = reinterpret_cast<TileOp*>(sst + P.nstages);
  R* smat = reinterpret_cast<R*>(sop + P.nops);
  using GA = GradAcc<R>;
  typename GA::T* sacc = reinterpret_cast<typename GA::T*>(smat + ((P.nmat + 1) & ~1));  // NW x ngrad
  // complex64: each thread's shares of up to kAdjPend records, summed over the warp
  // together (a transposing reduction: 9 shuffles for 8 records instead of 40)
  float* pend = reinterpret_cast<float*>(sacc + NW * P.ngrad);  // kAdjPend x NT
  __shared__ int16_t pslot[NW][kAdjPend];
  int npend = 0;  // warp-uniform: every thread of a warp takes the same records
  __shared__ int8_t sbits[16];
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 16; ++k) sbits[k] = P.bits[k];
  }
  __syncthreads();
  for (uint32_t h = threadIdx.x; h < (1u << nhi); h += blockDim.x) {
    uint64_t o = 0;
    for (int k = 0; k < nhi; ++k)
      if ((h >> k) & 1) o |= uint64_t(1) << sbits[L + k];
    hioff[h] = o;
  }
  build_tile_number_tables(tnt, sbits, m, __ffsll(static_cast<long long>(P.ntiles)) - 1);
  for (int i = threadIdx.x; i < P.nstages; i += blockDim.x) sst[i] = stages[P.stage0 + i];
  for (int i = threadIdx.x; i < P.nops; i += blockDim.x) sop[i] = ops[P.op0 + i];
  for (int i = threadIdx.x; i < P.nmat; i += blockDim.x) smat[i] = mats[P.mat0 + i];
  for (int i = threadIdx.x; i < NW * P.ngrad; i += blockDim.x) sacc[i] = GA::zero();
  __syncthreads();
  const uint32_t lowmask = (1u << L) - 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Cplx<R>* cpool = reinterpret_cast<const Cplx<R>*>(pool);
  uint64_t t = blockIdx.x;
  if (t < P.ntiles) {
    const uint64_t b0 = tile_base(t, tnt);
    prefetch_tile<R>(bufs, psi, b0, hioff, L, T);
    prefetch_tile<R>(bufs + 2 * T, lam, b0, hioff, L, T);
  }
  cp_async_commit();
  for (int it = 0; t < P.ntiles; t += gridDim.x, ++it) {
    Cplx<R>* tp = bufs + (it & 1) * T;
    Cplx<R>* tl = bufs + 2 * T + (it & 1) * T;
    const uint64_t base = tile_base(t, tnt);
    const uint64_t tn = t + gridDim.x;
    if (tn < P.ntiles) {
      const uint64_t bn = tile_base(tn, tnt);
      prefetch_tile<R>(bufs + ((it + 1) & 1) * T, psi, bn, hioff, L, T);
      prefetch_tile<R>(bufs + 2 * T + ((it + 1) & 1) * T, lam, bn, hioff, L, T);
    }
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    for (int s = 0; s < P.nstages; ++s) {
      const TileStage& st = sst[s];
      uint32_t r0 = 0;
#pragma unroll
      for (int k = 0; k < 16; ++k)
        if (k < m - SB) r0 |= ((threadIdx.x >> k) & 1u) << st.lane_bit[k];
      uint32_t sw[SB];
#pragma unroll
      for (int k = 0; k < SB; ++k) sw[k] = tile_swz(1u << st.slot_bit[k]);
      const uint32_t p0 = tile_swz(r0);
      Cplx<R> v[NA], w[NA];
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        const uint32_t a = p0 ^ slot_xor<SB>(j, sw);
        v[j] = tp[a];
        w[j] = tl[a];
      }
      for (int q = 0; q < st.nops; ++q) {
        const TileOp op = sop[st.op0 + q];  // one copy into registers (the loop writes shared memory)
        if (op.grad >= 0) {
          // recorded rotations carry no condition: every thread takes part
          R share;
          if (op.gen == 2) {
            // Z on bit zloc (in the tile) or zglob (fixed by the tile number)
            int ks = -1;
#pragma unroll
            for (int k = 0; k < SB; ++k)
              if (st.slot_bit[k] == op.zloc) ks = k;
            const uint32_t fixed = op.zloc >= 0 ? ((r0 >> op.zloc) & 1u) : uint32_t((base >> op.zglob) & 1u);
            if constexpr (sizeof(R) == 4) {
              // the signs of the slot combinations as compile-time constants
              share = grad_z_at<R, SB>(ks, v, w, fixed);
            } else {
              // (complex128: the selecting form keeps the FP64 pass's register allocation)
              share = R(0);
#pragma unroll
              for (int j = 0; j < NA; ++j) {
                const uint32_t b = ks >= 0 ? uint32_t((j >> ks) & 1) : fixed;
                const R x = im_conj_mul(w[j], v[j]);
                share += b ? -x : x;
              }
            }
          } else {
            share = grad_pairs_at<R, SB>(op.s0, v, w, op.gen);
          }
          if constexpr (sizeof(R) == 4) {
            pend[npend * NT + threadIdx.x] = share;
            if (lane == 0) pslot[warp][npend] = int16_t(op.gslot);
            if (++npend == kAdjPend) {
              flush_records_impl<NT>(pend, pslot[warp], npend, lane, reinterpret_cast<float2*>(sacc + warp * P.ngrad));
              npend = 0;
            }
          } else {
            // warp sum at the state's precision (32 shares), then one update of the
            // warp's running sum
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) share += __shfl_xor_sync(0xffffffffu, share, o);
            if (lane == 0) GA::add(sacc[warp * P.ngrad + op.gslot], share);
          }
        }
        if ((base & op.gmask) != op.gval) continue;  // condition on bits outside the tile
        if ((r0 & op.lmask) != op.lval) continue;    // ... on the thread's lane bits
        if (op.type == TOP_DENSE1) {
          apply_dense1<R, SB>(op.s0, v, smat + op.mat, op.jmask);
          apply_dense1<R, SB>(op.s0, w, smat + op.mat, op.jmask);
        } else if (op.type == TOP_REAL1) {
          apply_real1<R, SB>(op.s0, v, smat + op.mat, op.jmask);
          apply_real1<R, SB>(op.s0, w, smat + op.mat, op.jmask);
        } else if (op.type == TOP_DENSE2) {
          apply_dense2<R, SB>(op.s0, op.s1, v, smat + op.mat);
          apply_dense2<R, SB>(op.s0, op.s1, w, smat + op.mat);
        } else if (op.type == TOP_PHASE1) {
          const uint32_t fixed =
              op.s0 >= 0 ? 0u : op.zloc >= 0 ? (r0 >> op.zloc) & 1u : uint32_t((base >> op.zglob) & 1u);
          apply_phase1<R, SB>(v, smat + op.mat, op.s0, fixed, op.jmask);
          apply_phase1<R, SB>(w, smat + op.mat, op.s0, fixed, op.jmask);
        } else if (op.type == TOP_CZSET) {
          const uint32_t flip = czset_flips<R, SB>(smat + op.mat, op.s0, r0, base);
#pragma unroll
          for (int j = 0; j < NA; ++j)
            if ((flip >> j) & 1u) {
              v[j] = Cplx<R>{-v[j].re, -v[j].im};
              w[j] = Cplx<R>{-w[j].re, -w[j].im};
            }
        } else {
          // exp(i (c + sum beta_p b_p)), the same factor on both states
          const Cplx<R>* jt = reinterpret_cast<const Cplx<R>*>(smat + op.mat);
          const Cplx<R>* l0 = cpool + op.tab;
          const Cplx<R>* l1 = l0 + (1 << P.c0);
          const Cplx<R>* g0 = l1 + (1 << (m - P.c0));
          const uint32_t gn = 1u << P.cg, gm = gn - 1;
          Cplx<R> f = cmul(cmul(g0[t & gm], g0[gn + ((t >> P.cg) & gm)]), g0[2 * gn + ((t >> (2 * P.cg)) & gm)]);
          f = cmul(f, cmul(l0[r0 & ((1u << P.c0) - 1)], l1[r0 >> P.c0]));
#pragma unroll
          for (int j = 0; j < NA; ++j) {
            if (!((op.jmask >> j) & 1u)) continue;  // ... on the slot bits
            const Cplx<R> z = cmul(f, jt[j]);
            v[j] = cmul(v[j], z);
            w[j] = cmul(w[j], z);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        const uint32_t a = p0 ^ slot_xor<SB>(j, sw);
        tp[a] = v[j];
        tl[a] = w[j];
      }
      if (st.warp_local)
        __syncwarp();  // the next stage gives this warp the same amplitudes
      else
        __syncthreads();
    }
    for (uint32_t e = threadIdx.x; e < T / 2; e += blockDim.x) {
      const uint32_t r = 2 * e;
      const uint64_t gi = base | hioff[r >> L] | (r & lowmask);
      const uint32_t p = tile_swz(r);
      st_amp2<R>(psi, gi, tp[p], tp[p ^ 1u]);
      st_amp2<R>(lam, gi, tl[p], tl[p ^ 1u]);
    }
    __syncthreads();  // this buffer is refilled two iterations later
  }
  if constexpr (sizeof(R) == 4) {
    if (npend > 0)
      flush_records_impl<NT>(pend, pslot[warp], npend, lane, reinterpret_cast<float2*>(sacc + warp * P.ngrad));
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  // this block's total for each recorded rotation, warps added in a fixed order
  for (int i = threadIdx.x; i < P.nops; i += blockDim.x) {
    const TileOp& op = sop[i];
    if (op.grad < 0) continue;
    double a = 0.0;
    for (int k = 0; k < NW; ++k) a += GA::value(sacc[k * P.ngrad + op.gslot]);
    gpart[size_t(op.grad) * gridDim.x + blockIdx.x] = a;
  }
}

// ---------------------------------------------------------------------------
// complex128 in double-float arithmetic (states of 2^kDfMinQubits amplitudes or more)
// ---------------------------------------------------------------------------
// the sum of the two lanes of a packed double-float result
__device__ __forceinline__ float2 df_lane_total(const DF2& r) {
  return dfs_add(make_float2(r.hi.x, r.lo.x), make_float2(r.hi.y, r.lo.y));
}
// one packed product term c x (c's hi, lo; its -hi formed here) into the accumulator
__device__ __forceinline__ void dfg_term(DF2Acc& a, bool first, float2 ch, float2 cl, const DF2& x) {
  const float2 cn = make_float2(-ch.x, -ch.y);
  if (first)
    df2_first(a, ch, cn, cl, x);
  else
    df2_mac(a, ch, cn, cl, x);
}

// Im <w|Z_b|v> with bit b the register slot KS (>= 0) or reading `fixed` (KS = -1):
// lanes (w.re, -w.im) * (v.im, v.re), the sign of each slot combination at compile time
template <int SB, int KS>
__device__ __forceinline__ float2 dfgrad_z(const DFC (&v)[1 << SB], const DFC (&w)[1 << SB], uint32_t fixed) {
  DF2Acc a;
#pragma unroll
  for (int j = 0; j < (1 << SB); ++j) {
    float2 ch = make_float2(w[j].hi.x, -w[j].hi.y), cl = make_float2(w[j].lo.x, -w[j].lo.y);
    if (KS >= 0 && ((j >> KS) & 1)) {
      ch = make_float2(-ch.x, -ch.y);
      cl = make_float2(-cl.x, -cl.y);
    }
    dfg_term(a, j == 0, ch, cl, dfc_sw(v[j]));
  }
  const float2 t = df_lane_total(df2_result(a));
  return (KS < 0 && fixed) ? make_float2(-t.x, -t.y) : t;
}

template <int SB>
__device__ __forceinline__ float2 dfgrad_z_at(int ks, const DFC (&v)[1 << SB], const DFC (&w)[1 << SB],
                                              uint32_t fixed) {
  switch (ks) {
    case 0: return dfgrad_z<SB, 0>(v, w, fixed);
    case 1: return dfgrad_z<SB, 1>(v, w, fixed);
    case 2:
      if constexpr (SB > 2) return dfgrad_z<SB, 2>(v, w, fixed);
      return make_float2(0.0f, 0.0f);
    case 3:
      if constexpr (SB > 3) return dfgrad_z<SB, 3>(v, w, fixed);
      return make_float2(0.0f, 0.0f);
    default: return dfgrad_z<SB, -1>(v, w, fixed);
  }
}

// Im <w|G|v> over the pairs along slot S0: G = X (gen 0):
//   (w0.re, -w0.im) * (v1.im, v1.re) + (w1.re, -w1.im) * (v0.im, v0.re);
// G = Y (gen 1): Im(conj(w0) (-i v1)) + Im(conj(w1) (i v0)) =
//   (w1.re, w1.im) * (v0.re, v0.im) - (w0.re, w0.im) * (v1.re, v1.im)
template <int SB, int S0>
__device__ __forceinline__ float2 dfgrad_pairs(const DFC (&v)[1 << SB], const DFC (&w)[1 << SB], int gen) {
  DF2Acc a;
  bool first = true;
#pragma unroll
  for (int j = 0; j < (1 << SB); ++j) {
    if (j & (1 << S0)) continue;
    const int j1 = j | (1 << S0);
    if (gen == 0) {
      dfg_term(a, first, make_float2(w[j].hi.x, -w[j].hi.y), make_float2(w[j].lo.x, -w[j].lo.y), dfc_sw(v[j1]));
      dfg_term(a, false, make_float2(w[j1].hi.x, -w[j1].hi.y), make_float2(w[j1].lo.x, -w[j1].lo.y),
               dfc_sw(v[j]));
    } else {
      dfg_term(a, first, w[j1].hi, w[j1].lo, dfc_x(v[j]));
      dfg_term(a, false, make_float2(-w[j].hi.x, -w[j].hi.y), make_float2(-w[j].lo.x, -w[j].lo.y), dfc_x(v[j1]));
    }
    first = false;
  }
  return df_lane_total(df2_result(a));
}

template <int SB>
__device__ __forceinline__ float2 dfgrad_pairs_at(int s0, const DFC (&v)[1 << SB], const DFC (&w)[1 << SB],
                                                  int gen) {
  switch (s0) {
    case 0: return dfgrad_pairs<SB, 0>(v, w, gen);
    case 1: return dfgrad_pairs<SB, 1>(v, w, gen);
    case 2:
      if constexpr (SB > 2) return dfgrad_pairs<SB, 2>(v, w, gen);
      return make_float2(0.0f, 0.0f);
    default:
      if constexpr (SB > 3) return dfgrad_pairs<SB, 3>(v, w, gen);
      return make_float2(0.0f, 0.0f);
  }
}

// The reverse pass of k_adj_pass for complex128 in double-float arithmetic: both tiles
// split in place after their load, every op's double-float body applied to psi and
// lambda, each record's share a double-float sum, summed over the warp with TwoSum and
// kept per warp and rotation as (hi, lo); the matrices and tables are double-float slots.
template <int NT, int SB>
__global__ void __launch_bounds__(NT, 1) k_adj_pass_df(double* __restrict__ psi, double* __restrict__ lam,
                                                       const TilePass P, const TileStage* __restrict__ stages,
                                                       const TileOp* __restrict__ ops, const double* __restrict__ pool,
                                                       const double* __restrict__ mats, double* __restrict__ gpart) {
  constexpr int NA = 1 << SB;
  constexpr int NW = NT / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = P.m, L = P.L;
  const uint32_t T = 1u << m;
  Cplx<double>* bufs = reinterpret_cast<Cplx<double>*>(smem_raw);  // psi: 2 x T, lambda: 2 x T
  uint64_t* hioff = reinterpret_cast<uint64_t*>(smem_raw + 4 * sizeof(Cplx<double>) * T);
  const int nhi = m - L;
  uint64_t* tnt = hioff + (1u << nhi);
  TileStage* sst = reinterpret_cast<TileStage*>(tnt + kTileNumberTab);
  TileOp* sop = reinterpret_cast<TileOp*>(sst + P.nstages);
  double* smat = reinterpret_cast<double*>(sop + P.nops);
  float2* sacc = reinterpret_cast<float2*>(smat + ((P.nmat + 1) & ~1));  // NW x ngrad
  __shared__ int8_t sbits[16];
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 16; ++k) sbits[k] = P.bits[k];
  }
  __syncthreads();
  for (uint32_t h = threadIdx.x; h < (1u << nhi); h += blockDim.x) {
    uint64_t o = 0;
    for (int k = 0; k < nhi; ++k)
      if ((h >> k) & 1) o |= uint64_t(1) << sbits[L + k];
    hioff[h] = o;
  }
  build_tile_number_tables(tnt, sbits, m, __ffsll(static_cast<long long>(P.ntiles)) - 1);
  for (int i = threadIdx.x; i < P.nstages; i += blockDim.x) sst[i] = stages[P.stage0 + i];
  for (int i = threadIdx.x; i < P.nops; i += blockDim.x) sop[i] = ops[P.op0 + i];
  for (int i = threadIdx.x; i < P.nmat; i += blockDim.x) smat[i] = mats[P.mat0 + i];
  for (int i = threadIdx.x; i < NW * P.ngrad; i += blockDim.x) sacc[i] = make_float2(0.0f, 0.0f);
  __syncthreads();
  const uint32_t lowmask = (1u << L) - 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint64_t t = blockIdx.x;
  if (t < P.ntiles) {
    const uint64_t b0 = tile_base(t, tnt);
    prefetch_tile<double>(bufs, psi, b0, hioff, L, T);
    prefetch_tile<double>(bufs + 2 * T, lam, b0, hioff, L, T);
  }
  cp_async_commit();
  for (int it = 0; t < P.ntiles; t += gridDim.x, ++it) {
    Cplx<double>* dp = bufs + (it & 1) * T;
    Cplx<double>* dl = bufs + 2 * T + (it & 1) * T;
    float4* tp = reinterpret_cast<float4*>(dp);
    float4* tl = reinterpret_cast<float4*>(dl);
    const uint64_t base = tile_base(t, tnt);
    const uint64_t tn = t + gridDim.x;
    if (tn < P.ntiles) {
      const uint64_t bn = tile_base(tn, tnt);
      prefetch_tile<double>(bufs + ((it + 1) & 1) * T, psi, bn, hioff, L, T);
      prefetch_tile<double>(bufs + 2 * T + ((it + 1) & 1) * T, lam, bn, hioff, L, T);
    }
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    for (uint32_t p = threadIdx.x; p < T; p += blockDim.x) {
      const Cplx<double> a = dp[p], b = dl[p];
      float rh, rl, ih, il;
      df_split(a.re, rh, rl);
      df_split(a.im, ih, il);
      tp[p] = make_float4(rh, ih, rl, il);
      df_split(b.re, rh, rl);
      df_split(b.im, ih, il);
      tl[p] = make_float4(rh, ih, rl, il);
    }
    __syncthreads();
    for (int s = 0; s < P.nstages; ++s) {
      const TileStage& st = sst[s];
      uint32_t r0 = 0;
#pragma unroll
      for (int k = 0; k < 16; ++k)
        if (k < m - SB) r0 |= ((threadIdx.x >> k) & 1u) << st.lane_bit[k];
      uint32_t sw[SB];
#pragma unroll
      for (int k = 0; k < SB; ++k) sw[k] = tile_swz(1u << st.slot_bit[k]);
      const uint32_t p0 = tile_swz(r0);
      DFC v[NA], w[NA];
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        const uint32_t a = p0 ^ slot_xor<SB>(j, sw);
        v[j] = dfc_ld(tp, a);
        w[j] = dfc_ld(tl, a);
      }
      for (int q = 0; q < st.nops; ++q) {
        const TileOp op = sop[st.op0 + q];
        if (op.grad >= 0) {
          float2 share;
          if (op.gen == 2) {
            int ks = -1;
#pragma unroll
            for (int k = 0; k < SB; ++k)
              if (st.slot_bit[k] == op.zloc) ks = k;
            const uint32_t fixed = op.zloc >= 0 ? ((r0 >> op.zloc) & 1u) : uint32_t((base >> op.zglob) & 1u);
            share = dfgrad_z_at<SB>(ks, v, w, fixed);
          } else {
            share = dfgrad_pairs_at<SB>(op.s0, v, w, op.gen);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1)
            share = dfs_add(share, make_float2(__shfl_xor_sync(0xffffffffu, share.x, o),
                                               __shfl_xor_sync(0xffffffffu, share.y, o)));
          if (lane == 0) sacc[warp * P.ngrad + op.gslot] = dfs_add(sacc[warp * P.ngrad + op.gslot], share);
        }
        if ((base & op.gmask) != op.gval) continue;
        if ((r0 & op.lmask) != op.lval) continue;
        const double* mm = smat + op.mat;
        if (op.type == TOP_DENSE1) {
          df_apply_dense1<SB>(op.s0, v, mm, op.jmask);
          df_apply_dense1<SB>(op.s0, w, mm, op.jmask);
        } else if (op.type == TOP_REAL1) {
          df_apply_real1<SB>(op.s0, v, mm, op.jmask);
          df_apply_real1<SB>(op.s0, w, mm, op.jmask);
        } else if (op.type == TOP_DENSE2) {
          df_apply_dense2<SB>(op.s0, op.s1, v, mm);
          df_apply_dense2<SB>(op.s0, op.s1, w, mm);
        } else if (op.type == TOP_PHASE1) {
          const uint32_t fixed =
              op.s0 >= 0 ? 0u : op.zloc >= 0 ? (r0 >> op.zloc) & 1u : uint32_t((base >> op.zglob) & 1u);
          df_apply_phase1<SB>(v, mm, op.s0, fixed, op.jmask);
          df_apply_phase1<SB>(w, mm, op.s0, fixed, op.jmask);
        } else if (op.type == TOP_CZSET) {
          const uint32_t flip = czset_flips<double, SB>(mm, op.s0, r0, base);
#pragma unroll
          for (int j = 0; j < NA; ++j)
            if ((flip >> j) & 1u) {
              v[j].hi = make_float2(-v[j].hi.x, -v[j].hi.y);
              v[j].lo = make_float2(-v[j].lo.x, -v[j].lo.y);
              w[j].hi = make_float2(-w[j].hi.x, -w[j].hi.y);
              w[j].lo = make_float2(-w[j].lo.x, -w[j].lo.y);
            }
        } else {
          // exp(i (c + sum beta_p b_p)), the same factor on both states
          const double* l0 = pool + 2 * op.tab;
          const double* l1 = l0 + 2 * (1 << P.c0);
          const double* g0 = l1 + 2 * (1 << (m - P.c0));
          const uint32_t gn = 1u << P.cg, gm = gn - 1;
          DFC f = dfc_mul(dfc_slots(g0 + 2 * (t & gm)), dfc_slots(g0 + 2 * (gn + ((t >> P.cg) & gm))));
          f = dfc_mul(dfc_slots(g0 + 2 * (2 * gn + ((t >> (2 * P.cg)) & gm))), f);
          f = dfc_mul(dfc_slots(l0 + 2 * (r0 & ((1u << P.c0) - 1))), f);
          f = dfc_mul(dfc_slots(l1 + 2 * (r0 >> P.c0)), f);
          const DFPair pf = df_pairs(f);
#pragma unroll
          for (int j = 0; j < NA; ++j) {
            if (!((op.jmask >> j) & 1u)) continue;
            DF2Acc a;
            dfc_first(a, pf, dfc_slots(mm + 2 * j));
            const DFPair pz = df_pairs(dfc_res(a));
            DF2Acc b0, b1;
            dfc_first(b0, pz, v[j]);
            dfc_first(b1, pz, w[j]);
            v[j] = dfc_res(b0);
            w[j] = dfc_res(b1);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        const uint32_t a = p0 ^ slot_xor<SB>(j, sw);
        dfc_st(tp, a, v[j]);
        dfc_st(tl, a, w[j]);
      }
      if (st.warp_local)
        __syncwarp();
      else
        __syncthreads();
    }
    for (uint32_t e = threadIdx.x; e < T / 2; e += blockDim.x) {
      const uint32_t r = 2 * e;
      const uint64_t gi = base | hioff[r >> L] | (r & lowmask);
      const uint32_t p = tile_swz(r);
      const float4 a0 = tp[p], a1 = tp[p ^ 1u], b0 = tl[p], b1 = tl[p ^ 1u];
      st_amp2<double>(psi, gi, Cplx<double>{df_join(a0.x, a0.z), df_join(a0.y, a0.w)},
                      Cplx<double>{df_join(a1.x, a1.z), df_join(a1.y, a1.w)});
      st_amp2<double>(lam, gi, Cplx<double>{df_join(b0.x, b0.z), df_join(b0.y, b0.w)},
                      Cplx<double>{df_join(b1.x, b1.z), df_join(b1.y, b1.w)});
    }
    __syncthreads();
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  for (int i = threadIdx.x; i < P.nops; i += blockDim.x) {
    const TileOp& op = sop[i];
    if (op.grad < 0) continue;
    double a = 0.0;
    for (int k = 0; k < NW; ++k) {
      const float2 x = sacc[k * P.ngrad + op.gslot];
      a += double(x.x) + double(x.y);
    }
    gpart[size_t(op.grad) * gridDim.x + blockIdx.x] = a;
  }
}

// Tile shape of the fused sweep per precision: two states x two buffers of 2^m
// amplitudes in shared memory (4 x 32 KiB), register stages of SB bits per state.
template <typename R>
struct AdjShape;
template <>
struct AdjShape<float> {
  static constexpr int M = 12, L = 4, SB = 3, NT = 512;
};
template <>
struct AdjShape<double> {
  static constexpr int M = 11, L = 3, SB = 3, NT = 256;
};

// complex128 in double-float arithmetic: the same tiles, 2-bit register stages per
// state with 512 threads (3-bit stages with 256 threads: 90 against 81 ms per 24-qubit
// gradient call; the register cap of 512 threads costs a 152-byte spill)
constexpr int kAdjDfSB = 2, kAdjDfNT = 512;

int adjoint_tiles_min_qubits() { return 12; }

template <typename R>
qc_status adjoint_reverse_tiles(int n, const std::vector<ResolvedOp>& rev, const std::vector<int>& grad,
                                const std::vector<int>& gen, R* psi, R* lam, cudaStream_t stream, AdjPlanBuf* buf,
                                double* gpart, int* grid_out) {
  using S = AdjShape<R>;
  const int m = S::M, L = S::L;
  if (n < m) {
    set_error("fused adjoint sweep needs n >= %d", m);
    return QC_ERR_UNSUPPORTED;
  }
  const bool df = sizeof(R) == 8 && n >= kDfMinQubits;
  const int sbw = df ? kAdjDfSB : S::SB, ntw = df ? kAdjDfNT : S::NT;
  std::vector<PlanOp> pops;
  to_plan_ops(rev, pops, &grad, &gen);
  // psi and lambda take every op together, so a global phase of an op multiplies both
  // and cancels in Im<lambda|G|psi>: leave it out (a Z rotation then changes only the
  // amplitudes whose bit reads 1)
  drop_global_phases(pops);
  const std::vector<BuiltPass> bps = build_passes(pops, n, m, L);
  HostPlan<R> hp;
  for (const BuiltPass& bp : bps)
    emit_pass<R>(bp, pops, n, m, L, sbw, hp, /*swap_ops=*/false, /*phase1_ops=*/true, /*relabel_swaps=*/false,
                 /*bfly_ops=*/false, /*real1_ops=*/true);
  g_last_pass_count = int(hp.passes.size());
  if constexpr (sizeof(R) == 8) {
    if (df) encode_df_slots(hp);
  }
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t sb = al(hp.stages.size() * sizeof(TileStage));
  const size_t ob = al(hp.ops.size() * sizeof(TileOp));
  const size_t pb = al(hp.pool.size() * sizeof(R));
  const size_t mb = al(hp.mats.size() * sizeof(R));
  const size_t total = sb + ob + pb + mb + 256;
  if (buf->bytes < total) {
    if (buf->p) {
      cudaStreamSynchronize(stream);
      cudaFree(buf->p);
      buf->p = nullptr;
      buf->bytes = 0;
    }
    if (qc_status st = check_cuda(cudaMalloc(&buf->p, total), "adjoint plan")) return st;
    buf->bytes = total;
  }
  buf->host.assign(sb + ob + pb + mb, 0);
  char* h = buf->host.data();
  if (!hp.stages.empty()) memcpy(h, hp.stages.data(), hp.stages.size() * sizeof(TileStage));
  if (!hp.ops.empty()) memcpy(h + sb, hp.ops.data(), hp.ops.size() * sizeof(TileOp));
  if (!hp.pool.empty()) memcpy(h + sb + ob, hp.pool.data(), hp.pool.size() * sizeof(R));
  if (!hp.mats.empty()) memcpy(h + sb + ob + pb, hp.mats.data(), hp.mats.size() * sizeof(R));
  char* base = static_cast<char*>(buf->p);
  if (qc_status st = check_cuda(cudaMemcpyAsync(base, h, buf->host.size(), cudaMemcpyHostToDevice, stream),
                                "adjoint plan upload"))
    return st;
  size_t plan_max = 0;
  for (const TilePass& P : hp.passes)
    plan_max = std::max(plan_max, P.nstages * sizeof(TileStage) + P.nops * sizeof(TileOp) +
                                      ((P.nmat + 1) & ~1) * sizeof(R) + size_t(ntw / 32) * P.ngrad * sizeof(double) +
                                      (sizeof(R) == 4 ? size_t(kAdjPend) * ntw * sizeof(float) : 0));
  const size_t smem = 4 * sizeof(Cplx<R>) * (size_t(1) << m) + sizeof(uint64_t) * (size_t(1) << (m - L)) +
                      sizeof(uint64_t) * kTileNumberTab + plan_max;
  auto kern = k_adj_pass<R, S::NT, S::SB>;
  if constexpr (sizeof(R) == 8) {
    if (df) kern = k_adj_pass_df<kAdjDfNT, kAdjDfSB>;
  }
  if (qc_status st = check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)),
                                "adjoint pass shared memory"))
    return st;
  const uint64_t ntiles = uint64_t(1) << (n - m);
  const unsigned grid = unsigned(std::min<uint64_t>(ntiles, uint64_t(device_sm_count())));
  const TileStage* dst = reinterpret_cast<const TileStage*>(base);
  const TileOp* dop = reinterpret_cast<const TileOp*>(base + sb);
  const R* dpool = reinterpret_cast<const R*>(base + sb + ob);
  const R* dmats = reinterpret_cast<const R*>(base + sb + ob + pb);
  const unsigned threads = 1u << (m - sbw);
  for (const TilePass& P : hp.passes)
    QC_COUNT(), kern<<<grid, threads, smem, stream>>>(psi, lam, P, dst, dop, dpool, dmats, gpart);
  *grid_out = int(grid);
  return check_launch("adjoint pass");
}

template qc_status adjoint_reverse_tiles<float>(int, const std::vector<ResolvedOp>&, const std::vector<int>&,
                                                const std::vector<int>&, float*, float*, cudaStream_t, AdjPlanBuf*,
                                                double*, int*);
template qc_status adjoint_reverse_tiles<double>(int, const std::vector<ResolvedOp>&, const std::vector<int>&,
                                                 const std::vector<int>&, double*, double*, cudaStream_t,
                                                 AdjPlanBuf*, double*, int*);

}  // namespace qcgb

// ---------------------------------------------------------------------------
// host emulation of the fused reverse sweep's plan (a check of its logic)
// ---------------------------------------------------------------------------
namespace qcgb {

// The reverse sweep's plan for `rev` (the daggered gates in reverse order; grad/gen: the
// rotation recorded just before each op, or -1) applied on the host in FP64 to psi and
// lambda, each record's shares summed into rec[grad]: the plan adjoint_reverse_tiles
// launches, the same passes, stages, op conditions and record positions
template <typename R>
static void emulate_reverse(int n, const std::vector<ResolvedOp>& rev, const std::vector<int>& grad,
                            const std::vector<int>& gen, std::complex<double>* psi, std::complex<double>* lam,
                            double* rec) {
  using cd = std::complex<double>;
  using S = AdjShape<R>;
  const int m = S::M, L = S::L;
  const bool df = sizeof(R) == 8 && n >= kDfMinQubits;
  const int sb = df ? kAdjDfSB : S::SB;
  std::vector<PlanOp> pops;
  to_plan_ops(rev, pops, &grad, &gen);
  drop_global_phases(pops);
  const std::vector<BuiltPass> bps = build_passes(pops, n, m, L);
  HostPlan<double> hp;
  for (const BuiltPass& bp : bps)
    emit_pass<double>(bp, pops, n, m, L, sb, hp, /*swap_ops=*/false, /*phase1_ops=*/true, /*relabel_swaps=*/false,
                      /*bfly_ops=*/false, /*real1_ops=*/true);
  const uint32_t T = 1u << m, NA = 1u << sb;
  const uint64_t ntiles = uint64_t(1) << (n - m);
  const cd* cpool = reinterpret_cast<const cd*>(hp.pool.data());
  std::vector<cd> tp(T), tl(T), v(NA), w(NA);
  std::vector<uint32_t> pos(NA);
  for (const TilePass& P : hp.passes) {
    bool in[64] = {false};
    for (int k = 0; k < m; ++k) in[P.bits[k]] = true;
    std::vector<int> tnb;
    for (int b = 0; b < n; ++b)
      if (!in[b]) tnb.push_back(b);
    const double* mats = hp.mats.data() + P.mat0;
    for (uint64_t t = 0; t < ntiles; ++t) {
      uint64_t base = 0;
      for (size_t i = 0; i < tnb.size(); ++i)
        if ((t >> i) & 1) base |= uint64_t(1) << tnb[i];
      auto addr = [&](uint32_t u) {
        uint64_t g = base;
        for (int k = 0; k < m; ++k)
          if ((u >> k) & 1) g |= uint64_t(1) << P.bits[k];
        return g;
      };
      for (uint32_t u = 0; u < T; ++u) {
        tp[u] = psi[addr(u)];
        tl[u] = lam[addr(u)];
      }
      for (int s = 0; s < P.nstages; ++s) {
        const TileStage& st = hp.stages[size_t(P.stage0 + s)];
        for (uint32_t th = 0; th < (1u << (m - sb)); ++th) {
          uint32_t r0 = 0;
          for (int k = 0; k < m - sb; ++k) r0 |= ((th >> k) & 1u) << st.lane_bit[k];
          for (uint32_t j = 0; j < NA; ++j) {
            uint32_t u = r0;
            for (int k = 0; k < sb; ++k)
              if ((j >> k) & 1) u |= 1u << st.slot_bit[k];
            pos[j] = u;
            v[j] = tp[u];
            w[j] = tl[u];
          }
          for (int q = 0; q < st.nops; ++q) {
            const TileOp& op = hp.ops[size_t(P.op0 + st.op0 + q)];
            if (op.grad >= 0) {  // the record: Im <lambda|G|psi> over this thread's amplitudes
              double share = 0.0;
              if (op.gen == 2) {
                int ks = -1;
                for (int k = 0; k < sb; ++k)
                  if (st.slot_bit[k] == op.zloc) ks = k;
                const uint32_t fixed =
                    op.zloc >= 0 ? ((r0 >> op.zloc) & 1u) : uint32_t((base >> op.zglob) & 1u);
                for (uint32_t j = 0; j < NA; ++j) {
                  const uint32_t b = ks >= 0 ? (j >> ks) & 1u : fixed;
                  const double x = std::imag(std::conj(w[j]) * v[j]);
                  share += b ? -x : x;
                }
              } else {  // X or Y on slot s0
                for (uint32_t j = 0; j < NA; ++j) {
                  if ((j >> op.s0) & 1) continue;
                  const uint32_t j1 = j | (1u << op.s0);
                  const cd g0 = op.gen == 0 ? v[j1] : cd(0.0, -1.0) * v[j1];
                  const cd g1 = op.gen == 0 ? v[j] : cd(0.0, 1.0) * v[j];
                  share += std::imag(std::conj(w[j]) * g0) + std::imag(std::conj(w[j1]) * g1);
                }
              }
              rec[op.grad] += share;
            }
            if ((base & op.gmask) != op.gval) continue;
            if ((r0 & op.lmask) != op.lval) continue;
            emulate_tile_op(op, mats, P, cpool, m, t, base, r0, v);
            emulate_tile_op(op, mats, P, cpool, m, t, base, r0, w);
          }
          for (uint32_t j = 0; j < NA; ++j) {
            tp[pos[j]] = v[j];
            tl[pos[j]] = w[j];
          }
        }
      }
      for (uint32_t u = 0; u < T; ++u) {
        psi[addr(u)] = tp[u];
        lam[addr(u)] = tl[u];
      }
    }
  }
}

}  // namespace qcgb

extern "C" qc_status qc_adjoint_emulate(const qc_circuit* c, const double* params, qc_dtype dtype, double* psi,
                                        double* lam, double* records, int nrec) {
  using namespace qcgb;
  clear_error();
  if (!c || !psi || !lam || !records || c->n < AdjShape<float>::M || c->n > 24 || (c->nops > 0 && !c->ops) ||
      (dtype != QC_C64 && dtype != QC_C128)) {
    set_error("qc_adjoint_emulate: invalid arguments (%d <= n <= 24)", AdjShape<float>::M);
    return QC_ERR_INVALID_ARG;
  }
  // the rotations in order (RX, RY, RZ with a parameter) and the reverse circuit with its
  // records, as the gradient builds them
  std::vector<ResolvedOp> rops(size_t(c->nops));
  std::vector<int> gen(size_t(c->nops), -1);
  int nrot = 0;
  for (int i = 0; i < c->nops; ++i) {
    const qc_op& op = c->ops[i];
    if (qc_status st = resolve_op(c, op, params, &rops[size_t(i)])) return st;
    if (op.param >= 0) {
      if (op.kind != QC_GATE_RX && op.kind != QC_GATE_RY && op.kind != QC_GATE_RZ) {
        set_error("qc_adjoint_emulate: parameterised op %d must be RX, RY or RZ", i);
        return QC_ERR_UNSUPPORTED;
      }
      gen[size_t(i)] = op.kind == QC_GATE_RX ? 0 : op.kind == QC_GATE_RY ? 1 : 2;
      ++nrot;
    }
  }
  if (nrec < nrot) {
    set_error("qc_adjoint_emulate: %d records needed", nrot);
    return QC_ERR_INVALID_ARG;
  }
  std::vector<ResolvedOp> rev;
  std::vector<int> rgrad, rgen;
  int r = nrot;
  for (int i = c->nops - 1; i >= 0; --i) {
    ResolvedOp ud = rops[size_t(i)];
    const int dim = ud.form == FORM_2Q ? 4 : 2;
    double t[32];
    for (int a = 0; a < dim; ++a)
      for (int b = 0; b < dim; ++b) {
        t[2 * (a * dim + b)] = ud.m[2 * (b * dim + a)];
        t[2 * (a * dim + b) + 1] = -ud.m[2 * (b * dim + a) + 1];
      }
    memcpy(ud.m, t, sizeof(double) * 2 * dim * dim);
    rev.push_back(ud);
    rgrad.push_back(gen[size_t(i)] >= 0 ? --r : -1);
    rgen.push_back(gen[size_t(i)]);
  }
  for (int k = 0; k < nrot; ++k) records[k] = 0.0;
  auto* ps = reinterpret_cast<std::complex<double>*>(psi);
  auto* ls = reinterpret_cast<std::complex<double>*>(lam);
  if (dtype == QC_C64)
    emulate_reverse<float>(c->n, rev, rgrad, rgen, ps, ls, records);
  else
    emulate_reverse<double>(c->n, rev, rgrad, rgen, ps, ls, records);
  return QC_OK;
}
