// Fused execution of a circuit: shared-memory tile passes (QC_RUN_FUSED).
//
// The product of the paper's per-gate maps (Sec. 3.2) is unchanged by grouping
// gates that act on disjoint index bits, or by moving a gate past gates it commutes
// with.  A pass loads a tile of 2^m amplitudes -- every combination of the m index
// bits in the tile's bit set B (always including the lowest L bits, so that each
// contiguous run is 2^L amplitudes), the other bits fixed by the tile number --
// applies every gate of the pass to it in shared memory, and writes it back: one
// read and one write of the state per pass instead of one per gate.
//
// Gates a pass can hold: dense 1- and 2-qubit gates whose targets lie in B (controls
// anywhere: outside B they are a per-tile condition), and diagonal gates on any bits
// (the phase of an amplitude depends only on its index).  Runs of diagonal gates with
// the same condition are merged into one phase op exp(i (c + sum_p beta_p b_p)).
//
// Inside a pass the gates are split into stages; in a stage every thread holds 2^SB
// amplitudes spanning SB of the tile's bits in registers (SB = 5 for complex64, 4 for
// complex128) and applies all of the stage's gates to them before writing back to
// shared memory.  Shared memory is
// addressed through an XOR swizzle so that the strided accesses of a stage do not
// collide in the same bank.
#include <string.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "circuit.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace qcgb {

constexpr int kMaxStageBits = 5;  // amplitudes a thread holds per stage: 2^SB, SB <= 5

enum TileOpType : int32_t { TOP_DENSE1 = 0, TOP_DENSE2 = 1, TOP_PHASE = 2 };

struct TileOp {
  int32_t type;
  int32_t s0, s1;        // stage slots of the targets (DENSE2: s0 = first qubit = row MSB)
  uint32_t lmask, lval;  // condition on the amplitude's local (in-tile) index
  int32_t pad;
  uint64_t gmask, gval;  // condition on the index bits outside the tile
  int64_t mat;           // DENSE: matrix / PHASE: 2^SB-entry slot table, offset (R values)
                         // in the pass's matrix block
  int64_t tab;           // PHASE: offset (complex entries) of its other tables in the pool
  int64_t pad2;          // 64-byte record: keeps the staged matrices 16-byte aligned
};
static_assert(sizeof(TileOp) == 64, "TileOp must be 64 bytes");

struct TileStage {
  int32_t op0, nops;
  int8_t slot_bit[8];   // local bit of each slot (SB used)
  int8_t lane_bit[16];  // local bit receiving bit k of the thread index (the m-SB non-slot
                        // bits; the first ones cover distinct bit positions mod 4 so that
                        // a half warp's shared-memory accesses fall in distinct banks)
};
static_assert(sizeof(TileStage) == 32, "TileStage must be 32 bytes");

struct TilePass {
  int32_t m, L;
  int32_t stage0, nstages;
  int32_t op0, nops;    // the pass's ops (staged in shared memory)
  int32_t mat0, nmat;   // the pass's dense matrices and phase slot tables (R values)
  int8_t bits[16];   // B ascending (global bit positions); bits[0..L) = 0..L-1
  int32_t c0, c1;    // local phase-table chunks: local bits [0,c0) and [c0,m)
  int32_t cg;        // tile-index phase-table chunk width (3 chunks)
  uint64_t ntiles;
};

// ---------------------------------------------------------------------------
// device side
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t tile_swz(uint32_t r) {
  uint32_t x = r >> 4;
  return r ^ ((x ^ (x >> 4) ^ (x >> 8)) & 15u);
}

// offset of slot combination j: OR of the slot masks selected by j's bits
template <int SB>
__device__ __forceinline__ uint32_t slot_off(int j, const uint32_t (&sm)[SB]) {
  uint32_t o = 0;
#pragma unroll
  for (int k = 0; k < SB; ++k)
    if ((j >> k) & 1) o |= sm[k];
  return o;
}

// swizzled address offset of slot combination j: XOR of the swizzled slot masks
// (the swizzle is linear over XOR, but swizzled masks may share bits)
template <int SB>
__device__ __forceinline__ uint32_t slot_xor(int j, const uint32_t (&sw)[SB]) {
  uint32_t o = 0;
#pragma unroll
  for (int k = 0; k < SB; ++k)
    if ((j >> k) & 1) o ^= sw[k];
  return o;
}

// NV values of a 16-byte-aligned shared-memory matrix into registers
template <typename R, int NV>
__device__ __forceinline__ void load_mat(R (&um)[NV], const R* __restrict__ u) {
  if (sizeof(R) == 4) {
    const float4* q = reinterpret_cast<const float4*>(u);
#pragma unroll
    for (int i = 0; i < NV / 4; ++i) {
      const float4 t = q[i];
      um[4 * i] = R(t.x); um[4 * i + 1] = R(t.y); um[4 * i + 2] = R(t.z); um[4 * i + 3] = R(t.w);
    }
  } else {
    const double2* q = reinterpret_cast<const double2*>(u);
#pragma unroll
    for (int i = 0; i < NV / 2; ++i) {
      const double2 t = q[i];
      um[2 * i] = R(t.x); um[2 * i + 1] = R(t.y);
    }
  }
}

// Complex64 gates on packed pairs.  For complex64 the planner stores each matrix entry
// u = (ur, ui) as the two pairs (ur, ur) and (-ui, ui), so that u x is
// (ur, ur) * (xr, xi) + (-ui, ui) * (xi, xr): two paired FMAs (one instruction each on
// sm_100 and later) in place of four scalar ones.

template <int NE>
__device__ __forceinline__ void load_packed(float2 (&a)[NE], float2 (&b)[NE], const float* __restrict__ u) {
  const float4* q = reinterpret_cast<const float4*>(u);
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    const float4 t = q[e];
    a[e] = make_float2(t.x, t.y);
    b[e] = make_float2(t.z, t.w);
  }
}

template <typename R, int SB, int S0>
__device__ __forceinline__ void dense1(Cplx<R> (&v)[1 << SB], const R* __restrict__ u, uint32_t r0,
                                       const uint32_t (&sm)[SB], uint32_t lmask, uint32_t lval) {
  if constexpr (sizeof(R) == 4) {
    float2 a[4], b[4];
    load_packed<4>(a, b, u);
#pragma unroll
    for (int j = 0; j < (1 << SB); ++j) {
      if (j & (1 << S0)) continue;
      const int j1 = j | (1 << S0);
      if (((r0 | slot_off<SB>(j, sm)) & lmask) != lval) continue;
      const float2 x = f2(v[j]), xs = f2swap(v[j]), y = f2(v[j1]), ys = f2swap(v[j1]);
      v[j] = c2(__ffma2_rn(b[1], ys, __ffma2_rn(a[1], y, __ffma2_rn(b[0], xs, __fmul2_rn(a[0], x)))));
      v[j1] = c2(__ffma2_rn(b[3], ys, __ffma2_rn(a[3], y, __ffma2_rn(b[2], xs, __fmul2_rn(a[2], x)))));
    }
  } else {
    R um[8];
    load_mat<R, 8>(um, u);
    const Cplx<R> u00{um[0], um[1]}, u01{um[2], um[3]}, u10{um[4], um[5]}, u11{um[6], um[7]};
#pragma unroll
    for (int j = 0; j < (1 << SB); ++j) {
      if (j & (1 << S0)) continue;
      const int j1 = j | (1 << S0);
      if (((r0 | slot_off<SB>(j, sm)) & lmask) != lval) continue;
      const Cplx<R> x = v[j], y = v[j1];
      v[j] = cmul2(u00, x, u01, y);
      v[j1] = cmul2(u10, x, u11, y);
    }
  }
}

template <typename R, int SB, int S0, int S1>
__device__ __forceinline__ void dense2(Cplx<R> (&v)[1 << SB], const R* __restrict__ us) {
  if constexpr (sizeof(R) == 4) {
    float2 a[16], b[16];
    load_packed<16>(a, b, us);
    // the four output rows are independent chains: step them together so that each
    // packed FMA's result is not needed by the next instruction
#pragma unroll
    for (int j = 0; j < (1 << SB); ++j) {
      if (j & ((1 << S0) | (1 << S1))) continue;
      const int i[4] = {j, j | (1 << S1), j | (1 << S0), j | (1 << S0) | (1 << S1)};
      float2 x[4], xs[4], o[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        x[c] = f2(v[i[c]]);
        xs[c] = f2swap(v[i[c]]);
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) o[r] = __fmul2_rn(a[4 * r], x[0]);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (c > 0) {
#pragma unroll
          for (int r = 0; r < 4; ++r) o[r] = __ffma2_rn(a[4 * r + c], x[c], o[r]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) o[r] = __ffma2_rn(b[4 * r + c], xs[c], o[r]);
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) v[i[r]] = c2(o[r]);
    }
    return;
  }
  R u[32];
  load_mat<R, 32>(u, us);
#pragma unroll
  for (int j = 0; j < (1 << SB); ++j) {
    if (j & ((1 << S0) | (1 << S1))) continue;
    const int i0 = j, i1 = j | (1 << S1), i2 = j | (1 << S0), i3 = j | (1 << S0) | (1 << S1);
    const Cplx<R> x0 = v[i0], x1 = v[i1], x2 = v[i2], x3 = v[i3];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const R* ur = u + 8 * r;
      Cplx<R> o;
      o.re = fma(ur[0], x0.re, fma(-ur[1], x0.im, fma(ur[2], x1.re, fma(-ur[3], x1.im,
             fma(ur[4], x2.re, fma(-ur[5], x2.im, fma(ur[6], x3.re, -ur[7] * x3.im)))))));
      o.im = fma(ur[0], x0.im, fma(ur[1], x0.re, fma(ur[2], x1.im, fma(ur[3], x1.re,
             fma(ur[4], x2.im, fma(ur[5], x2.re, fma(ur[6], x3.im, ur[7] * x3.re)))))));
      if (r == 0) v[i0] = o;
      else if (r == 1) v[i1] = o;
      else if (r == 2) v[i2] = o;
      else v[i3] = o;
    }
  }
}

template <typename R, int SB>
__device__ __forceinline__ void apply_dense1(int s0, Cplx<R> (&v)[1 << SB], const R* u, uint32_t r0,
                                             const uint32_t (&sm)[SB], uint32_t lmask, uint32_t lval) {
  switch (s0) {
    case 0: dense1<R, SB, 0>(v, u, r0, sm, lmask, lval); break;
    case 1: dense1<R, SB, 1>(v, u, r0, sm, lmask, lval); break;
    case 2: dense1<R, SB, 2>(v, u, r0, sm, lmask, lval); break;
    case 3: dense1<R, SB, 3>(v, u, r0, sm, lmask, lval); break;
    default:
      if constexpr (SB > 4) dense1<R, SB, 4>(v, u, r0, sm, lmask, lval);
      break;
  }
}

#define QC_D2(A, B) \
  case (A) * 8 + (B): dense2<R, SB, A, B>(v, u); return;
template <typename R, int SB>
__device__ __forceinline__ void apply_dense2(int s0, int s1, Cplx<R> (&v)[1 << SB], const R* u) {
  switch (s0 * 8 + s1) {
    // the planner orders every two-qubit gate so that s0 < s1
    QC_D2(0, 1) QC_D2(0, 2) QC_D2(0, 3) QC_D2(1, 2) QC_D2(1, 3) QC_D2(2, 3)
    default: break;
  }
  if constexpr (SB > 4) {
    switch (s0 * 8 + s1) {
      QC_D2(0, 4) QC_D2(1, 4) QC_D2(2, 4) QC_D2(3, 4)
      default: break;
    }
  }
}
#undef QC_D2

// Asynchronous global -> shared copy of one amplitude (8 or 16 bytes).
template <typename R>
__device__ __forceinline__ void cp_async_amp(Cplx<R>* dst, const R* src) {
  const uint32_t d = uint32_t(__cvta_generic_to_shared(dst));
  if (sizeof(R) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <typename R>
__device__ __forceinline__ void prefetch_tile(Cplx<R>* buf, const R* amps, uint64_t base, const uint64_t* hioff,
                                              int L, uint32_t T) {
  const uint32_t lowmask = (1u << L) - 1;
  for (uint32_t r = threadIdx.x; r < T; r += blockDim.x) {
    const uint64_t gi = base | hioff[r >> L] | (r & lowmask);
    cp_async_amp<R>(buf + tile_swz(r), amps + 2 * gi);
  }
}

// One launch = one pass over all tiles; blockDim = 2^(m-SB), one block per SM with
// two tile buffers: the next tile is fetched (cp.async) while this one is computed.
template <typename R, int NT, int SB>
__global__ void __launch_bounds__(NT, 1) k_tile_pass(R* __restrict__ amps, const TilePass P,
                                                     const TileStage* __restrict__ stages,
                                                     const TileOp* __restrict__ ops, const R* __restrict__ pool,
                                                     const R* __restrict__ mats) {
  constexpr int NA = 1 << SB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = P.m, L = P.L;
  const uint32_t T = 1u << m;
  Cplx<R>* bufs = reinterpret_cast<Cplx<R>*>(smem_raw);  // 2 x T
  uint64_t* hioff = reinterpret_cast<uint64_t*>(smem_raw + 2 * sizeof(Cplx<R>) * T);
  const int nhi = m - L;
  // the pass's plan, copied once into shared memory: stages, ops, matrices
  TileStage* sst = reinterpret_cast<TileStage*>(hioff + (1u << nhi));
  TileOp* sop = reinterpret_cast<TileOp*>(sst + P.nstages);
  R* smat = reinterpret_cast<R*>(sop + P.nops);
  // the tile's bit positions in shared memory (a dynamically indexed kernel parameter
  // array would be copied to local memory)
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
  for (int i = threadIdx.x; i < P.nstages; i += blockDim.x) sst[i] = stages[P.stage0 + i];
  for (int i = threadIdx.x; i < P.nops; i += blockDim.x) sop[i] = ops[P.op0 + i];
  for (int i = threadIdx.x; i < P.nmat; i += blockDim.x) smat[i] = mats[P.mat0 + i];
  __syncthreads();
  const uint32_t lowmask = (1u << L) - 1;
  const Cplx<R>* cpool = reinterpret_cast<const Cplx<R>*>(pool);
  uint64_t t = blockIdx.x;
  if (t < P.ntiles) prefetch_tile<R>(bufs, amps, insert_zero_bits(t, sbits, m), hioff, L, T);
  cp_async_commit();
  for (int it = 0; t < P.ntiles; t += gridDim.x, ++it) {
    Cplx<R>* tile = bufs + (it & 1) * T;
    const uint64_t base = insert_zero_bits(t, sbits, m);
    const uint64_t tn = t + gridDim.x;
    if (tn < P.ntiles) prefetch_tile<R>(bufs + ((it + 1) & 1) * T, amps, insert_zero_bits(tn, sbits, m), hioff, L, T);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    for (int s = 0; s < P.nstages; ++s) {
      const TileStage& st = sst[s];
      uint32_t r0 = 0;
#pragma unroll
      for (int k = 0; k < 16; ++k)
        if (k < m - SB) r0 |= ((threadIdx.x >> k) & 1u) << st.lane_bit[k];
      uint32_t sm[SB], sw[SB];
#pragma unroll
      for (int k = 0; k < SB; ++k) {
        sm[k] = 1u << st.slot_bit[k];
        sw[k] = tile_swz(sm[k]);  // the swizzle is linear over XOR: swz(a^b) = swz(a)^swz(b)
      }
      const uint32_t p0 = tile_swz(r0);
      Cplx<R> v[NA];
#pragma unroll
      for (int j = 0; j < NA; ++j) v[j] = tile[p0 ^ slot_xor<SB>(j, sw)];
      for (int q = 0; q < st.nops; ++q) {
        const TileOp& op = sop[st.op0 + q];
        if ((base & op.gmask) != op.gval) continue;
        if (op.type == TOP_DENSE1) {
          apply_dense1<R, SB>(op.s0, v, smat + op.mat, r0, sm, op.lmask, op.lval);
        } else if (op.type == TOP_DENSE2) {
          apply_dense2<R, SB>(op.s0, op.s1, v, smat + op.mat);
        } else {
          // exp(i (c + sum beta_p b_p)) factorised over: tile-index chunks (3), the
          // thread's inactive local bits (2 chunks) and the 2^SB slot combinations
          const Cplx<R>* jt = reinterpret_cast<const Cplx<R>*>(smat + op.mat);
          const Cplx<R>* l0 = cpool + op.tab;
          const Cplx<R>* l1 = l0 + (1 << P.c0);
          const Cplx<R>* g0 = l1 + (1 << (m - P.c0));
          const uint32_t gn = 1u << P.cg, gm = gn - 1;
          Cplx<R> w = cmul(cmul(g0[t & gm], g0[gn + ((t >> P.cg) & gm)]), g0[2 * gn + ((t >> (2 * P.cg)) & gm)]);
          w = cmul(w, cmul(l0[r0 & ((1u << P.c0) - 1)], l1[r0 >> P.c0]));
#pragma unroll
          for (int j = 0; j < NA; ++j) {
            if (((r0 | slot_off<SB>(j, sm)) & op.lmask) != op.lval) continue;
            v[j] = cmul(v[j], cmul(w, jt[j]));
          }
        }
      }
#pragma unroll
      for (int j = 0; j < NA; ++j) tile[p0 ^ slot_xor<SB>(j, sw)] = v[j];
      __syncthreads();
    }
    for (uint32_t e = threadIdx.x; e < T / 2; e += blockDim.x) {
      const uint32_t r = 2 * e;
      const uint64_t gi = base | hioff[r >> L] | (r & lowmask);
      const uint32_t p = tile_swz(r);
      st_amp2<R>(amps, gi, tile[p], tile[p ^ 1u]);
    }
    __syncthreads();  // this buffer is refilled two iterations later
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// ---------------------------------------------------------------------------
// host planner
// ---------------------------------------------------------------------------
using cd = std::complex<double>;

struct PlanOp {
  // dense: 1 or 2 target bits, matrix, control mask/values (global bits)
  // phase: condition mask/values (global), constant angle and per-bit coefficients
  bool phase;
  int nt;
  int tb[2];
  double m[32];
  uint64_t cmask, cval;
  double c;
  std::vector<std::pair<int, double>> beta;  // (bit, coefficient)
  uint64_t touched;                          // every bit the op reads or writes
};

static bool near_unit(cd z) { return std::abs(std::abs(z) - 1.0) < 1e-12; }

// Converts resolved gates to plan ops; diagonal gates become phase ops.
static void to_plan_ops(const std::vector<ResolvedOp>& in, std::vector<PlanOp>& out) {
  for (const ResolvedOp& r : in) {
    PlanOp p{};
    p.cmask = p.cval = 0;
    if (r.form == FORM_2Q) {
      const cd d0(r.m[0], r.m[1]), d1(r.m[10], r.m[11]), d2(r.m[20], r.m[21]), d3(r.m[30], r.m[31]);
      bool diag = true;
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j)
          if (i != j && (r.m[2 * (4 * i + j)] != 0.0 || r.m[2 * (4 * i + j) + 1] != 0.0)) diag = false;
      if (diag && near_unit(d0) && near_unit(d1) && near_unit(d2) && near_unit(d3)) {
        // theta(ba, bb) = t00 + (t10-t00) ba + (t01-t00) bb + (t11-t10-t01+t00) ba bb
        const double t00 = std::arg(d0), t01 = std::arg(d1), t10 = std::arg(d2), t11 = std::arg(d3);
        const int a = r.bits[0], b = r.bits[1];
        PlanOp q{};
        q.phase = true;
        q.c = t00;
        q.beta = {{a, t10 - t00}, {b, t01 - t00}};
        q.touched = (uint64_t(1) << a) | (uint64_t(1) << b);
        out.push_back(q);
        const double quad = t11 - t10 - t01 + t00;
        if (quad != 0.0) {
          PlanOp w{};
          w.phase = true;
          w.cmask = w.cval = uint64_t(1) << a;
          w.c = 0.0;
          w.beta = {{b, quad}};
          w.touched = q.touched;
          out.push_back(w);
        }
        continue;
      }
      p.phase = false;
      p.nt = 2;
      p.tb[0] = r.bits[0];
      p.tb[1] = r.bits[1];
      memcpy(p.m, r.m, sizeof(double) * 32);
      p.touched = (uint64_t(1) << r.bits[0]) | (uint64_t(1) << r.bits[1]);
      out.push_back(p);
      continue;
    }
    const int nc = r.form == FORM_CTRL ? r.nq - 1 : 0;
    const int tgt = r.bits[nc];
    for (int j = 0; j < nc; ++j) {
      p.cmask |= uint64_t(1) << r.bits[j];
      if ((r.cstate >> j) & 1) p.cval |= uint64_t(1) << r.bits[j];
    }
    p.touched = p.cmask | (uint64_t(1) << tgt);
    const cd d0(r.m[0], r.m[1]), d1(r.m[6], r.m[7]);
    const bool diag = r.m[2] == 0 && r.m[3] == 0 && r.m[4] == 0 && r.m[5] == 0;
    if (diag && near_unit(d0) && near_unit(d1)) {
      p.phase = true;
      if (nc == 1 && r.m[0] == 1.0 && r.m[1] == 0.0) {
        // a singly controlled phase diag(1, e^{i phi}) is symmetric in its two qubits:
        // key it on the target bit so that phases sharing a target (e.g. the ladder of
        // controlled phases in a Fourier transform) merge into one phase op
        const int cb = r.bits[0];
        const bool cv = (r.cstate & 1) != 0;
        p.cmask = p.cval = uint64_t(1) << tgt;
        p.c = 0.0;
        const double phi = std::arg(d1);
        // control state 1: phi * b_c; control state 0: phi * (1 - b_c)
        if (cv) {
          p.beta = {{cb, phi}};
        } else {
          p.c = phi;
          p.beta = {{cb, -phi}};
        }
      } else {
        p.c = std::arg(d0);
        p.beta = {{tgt, std::arg(d1) - std::arg(d0)}};
      }
    } else {
      p.phase = false;
      p.nt = 1;
      p.tb[0] = tgt;
      memcpy(p.m, r.m, sizeof(double) * 8);
    }
    out.push_back(p);
  }
}

constexpr int kMaxPassOps = 128;  // bounds the plan staged in shared memory per pass

struct BuiltPass {
  std::vector<int> B;       // ascending
  std::vector<int> ops;     // indices into plan ops, in order
};

// One pass over `remaining` in order.  With `fixed` set, B is exactly `B0` (ops whose
// dense targets are outside it are skipped); otherwise B starts as B0 and grows to m
// bits with the targets of the first ops that need them.  An op is taken unless it
// meets a skipped op it may not commute with (shared bits; two diagonal ops commute).
static void greedy_pass(const std::vector<PlanOp>& ops, const std::vector<int>& remaining, int m, uint64_t B0,
                        bool fixed, BuiltPass* bp, std::vector<int>* excluded, uint64_t* Bout, double* score) {
  uint64_t Bmask = B0;
  int Bcount = __builtin_popcountll(B0);
  uint64_t blocked_all = 0;   // bits of skipped non-diagonal ops
  uint64_t blocked_diag = 0;  // bits of skipped diagonal ops
  double sc = 0.0;
  for (int idx : remaining) {
    const PlanOp& p = ops[idx];
    bool ok = (p.touched & blocked_all) == 0 && int(bp->ops.size()) < kMaxPassOps;
    if (ok && !p.phase) ok = (p.touched & blocked_diag) == 0;
    if (ok && !p.phase) {
      uint64_t need = 0;
      for (int k = 0; k < p.nt; ++k) need |= uint64_t(1) << p.tb[k];
      need &= ~Bmask;
      const int add = __builtin_popcountll(need);
      if (add == 0) {
      } else if (!fixed && Bcount + add <= m) {
        Bmask |= need;
        Bcount += add;
      } else {
        ok = false;
      }
    }
    if (ok) {
      bp->ops.push_back(idx);
      sc += p.phase ? 0.1 : double(p.nt);  // rough cost of the work the pass absorbs
    } else {
      excluded->push_back(idx);
      if (p.phase)
        blocked_diag |= p.touched;
      else
        blocked_all |= p.touched;
    }
  }
  *Bout = Bmask;
  *score = sc;
}

static std::vector<BuiltPass> build_passes(const std::vector<PlanOp>& ops, int n, int m, int L) {
  std::vector<int> remaining(ops.size());
  for (size_t i = 0; i < ops.size(); ++i) remaining[i] = int(i);
  std::vector<BuiltPass> passes;
  const uint64_t low = (uint64_t(1) << L) - 1;
  const int w = m - L;  // free tile bits
  while (!remaining.empty()) {
    // candidates: the growing greedy, and every contiguous window of w index bits next
    // to the always-present low bits (neighbouring qubits interact in most circuits)
    BuiltPass best;
    std::vector<int> best_ex;
    uint64_t bestB = 0;
    double best_score = -1.0;
    for (int cand = -1; cand <= n - w - L; ++cand) {
      BuiltPass bp;
      std::vector<int> ex;
      uint64_t Bm = 0;
      double sc = 0.0;
      if (cand < 0) {
        greedy_pass(ops, remaining, m, low, false, &bp, &ex, &Bm, &sc);
      } else {
        const uint64_t win = ((uint64_t(1) << w) - 1) << (L + cand);
        greedy_pass(ops, remaining, m, low | win, true, &bp, &ex, &Bm, &sc);
      }
      if (sc > best_score + 1e-9) {
        best_score = sc;
        best = bp;
        best_ex = ex;
        bestB = Bm;
      }
    }
    // fill B up to m bits with the lowest free bits (a full tile)
    int Bcount = __builtin_popcountll(bestB);
    for (int b = 0; Bcount < m && b < n; ++b)
      if (!((bestB >> b) & 1)) {
        bestB |= uint64_t(1) << b;
        ++Bcount;
      }
    for (int b = 0; b < n; ++b)
      if ((bestB >> b) & 1) best.B.push_back(b);
    passes.push_back(best);
    remaining.swap(best_ex);
  }
  return passes;
}

// Device plan assembled on the host.
template <typename R>
struct HostPlan {
  std::vector<TilePass> passes;
  std::vector<TileStage> stages;
  std::vector<TileOp> ops;
  std::vector<R> pool;  // phase tables read per thread (global memory)
  std::vector<R> mats;  // per-pass matrices and slot tables (staged in shared memory)
};

template <typename R>
static void emit_pass(const BuiltPass& bp, const std::vector<PlanOp>& pops, int n, int m, int L, int sb,
                      HostPlan<R>& hp) {
  TilePass P{};
  P.m = m;
  P.L = L;
  for (int i = 0; i < m; ++i) P.bits[i] = int8_t(bp.B[i]);
  P.ntiles = uint64_t(1) << (n - m);
  P.c0 = m / 2;
  P.c1 = m - P.c0;
  P.cg = (n - m + 2) / 3;
  if (P.cg < 1) P.cg = 1;
  P.stage0 = int(hp.stages.size());
  P.op0 = int(hp.ops.size());
  P.mat0 = int(hp.mats.size());
  int local_of[64];
  for (int b = 0; b < 64; ++b) local_of[b] = -1;
  for (int i = 0; i < m; ++i) local_of[bp.B[i]] = i;
  // tile-index bit of each global bit outside B
  int tbit_of[64];
  {
    int k = 0;
    for (int b = 0; b < n; ++b) tbit_of[b] = local_of[b] >= 0 ? -1 : k++;
  }
  // stages: each takes, in order, every remaining op of the pass whose dense targets
  // fit in <= 4 active local bits and that no skipped op it fails to commute with
  // precedes (same rule as for passes); skipped ops go to later stages in order.
  std::vector<int> rest = bp.ops;
  while (!rest.empty()) {
    std::vector<int> act;
    std::vector<int> take, skip;
    uint64_t blocked_all = 0, blocked_diag = 0;
    for (int idx : rest) {
      const PlanOp& p = pops[idx];
      bool ok = (p.touched & blocked_all) == 0;
      if (ok && !p.phase) ok = (p.touched & blocked_diag) == 0;
      if (ok && !p.phase) {
        std::vector<int> nw = act;
        for (int k = 0; k < p.nt; ++k) {
          const int lb = local_of[p.tb[k]];
          if (std::find(nw.begin(), nw.end(), lb) == nw.end()) nw.push_back(lb);
        }
        if (int(nw.size()) > sb)
          ok = false;
        else
          act = nw;
      }
      if (ok) {
        take.push_back(idx);
      } else {
        skip.push_back(idx);
        if (p.phase)
          blocked_diag |= p.touched;
        else
          blocked_all |= p.touched;
      }
    }
    // pad with unused local bits (lowest first)
    for (int b = 0; int(act.size()) < sb && b < m; ++b)
      if (std::find(act.begin(), act.end(), b) == act.end()) act.push_back(b);
    TileStage st{};
    for (int k = 0; k < sb; ++k) st.slot_bit[k] = int8_t(act[k]);
    {
      // thread-index bits -> non-slot local bits; first one bit per residue mod 4
      // (4 residues: 8-byte elements, half-warp banks; 3: 16-byte elements)
      std::vector<int> rest_bits;
      for (int b = 0; b < m; ++b)
        if (std::find(act.begin(), act.end(), b) == act.end()) rest_bits.push_back(b);
      std::vector<int> order;
      const int nres = sizeof(R) == 4 ? 4 : 3;
      for (int res = 0; res < nres; ++res)
        for (int b : rest_bits)
          if (b % 4 == res && std::find(order.begin(), order.end(), b) == order.end()) {
            order.push_back(b);
            break;
          }
      for (int b : rest_bits)
        if (std::find(order.begin(), order.end(), b) == order.end()) order.push_back(b);
      for (size_t k = 0; k < order.size() && k < 16; ++k) st.lane_bit[k] = int8_t(order[k]);
    }
    st.op0 = int(hp.ops.size()) - P.op0;
    const size_t j = take.size();
    for (size_t q = 0; q < j; ++q) {
      const PlanOp& p = pops[take[q]];
      TileOp op{};
      op.lmask = op.lval = 0;
      op.gmask = op.gval = 0;
      for (int b = 0; b < n; ++b) {
        if (!((p.cmask >> b) & 1)) continue;
        const bool v = (p.cval >> b) & 1;
        if (local_of[b] >= 0) {
          op.lmask |= 1u << local_of[b];
          if (v) op.lval |= 1u << local_of[b];
        } else {
          op.gmask |= uint64_t(1) << b;
          if (v) op.gval |= uint64_t(1) << b;
        }
      }
      if (!p.phase) {
        op.type = p.nt == 1 ? TOP_DENSE1 : TOP_DENSE2;
        auto slot = [&](int gbit) {
          const int lb = local_of[gbit];
          for (int k = 0; k < sb; ++k)
            if (st.slot_bit[k] == lb) return k;
          return -1;
        };
        op.s0 = slot(p.tb[0]);
        op.s1 = p.nt == 2 ? slot(p.tb[1]) : 0;
        op.mat = int64_t(hp.mats.size()) - P.mat0;
        // entry (re, im); complex64 stores it as the pairs (re, re), (-im, im)
        auto entry = [&](double re, double im) {
          hp.mats.push_back(R(re));
          if (sizeof(R) == 4) {
            hp.mats.push_back(R(re));
            hp.mats.push_back(R(-im));
          }
          hp.mats.push_back(R(im));
        };
        if (p.nt == 2 && op.s0 > op.s1) {
          // the same gate with its qubits listed in the other order: row/column index
          // 2a+b -> 2b+a
          std::swap(op.s0, op.s1);
          for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) {
              const int rr = ((r & 1) << 1) | (r >> 1), cc = ((c & 1) << 1) | (c >> 1);
              entry(p.m[2 * (4 * rr + cc)], p.m[2 * (4 * rr + cc) + 1]);
            }
        } else {
          for (int e = 0; e < (p.nt == 1 ? 4 : 16); ++e) entry(p.m[2 * e], p.m[2 * e + 1]);
        }
      } else {
        // merge following phase ops with the same condition (they commute)
        op.type = TOP_PHASE;
        double c = p.c;
        std::vector<double> beta(64, 0.0);
        for (auto& be : p.beta) beta[be.first] += be.second;
        while (q + 1 < j) {
          const PlanOp& nx = pops[take[q + 1]];
          if (!nx.phase || nx.cmask != p.cmask || nx.cval != p.cval) break;
          c += nx.c;
          for (auto& be : nx.beta) beta[be.first] += be.second;
          ++q;
        }
        // tables: [16 slot combos][2^c0 low local][2^c1 high local][3 x 2^cg tile index]
        while (hp.pool.size() % 2) hp.pool.push_back(R(0));
        op.tab = int64_t(hp.pool.size() / 2);
        auto push = [&](double ang) {
          hp.pool.push_back(R(std::cos(ang)));
          hp.pool.push_back(R(std::sin(ang)));
        };
        op.mat = int64_t(hp.mats.size()) - P.mat0;
        for (int jj = 0; jj < (1 << sb); ++jj) {
          double a = 0;
          for (int k = 0; k < sb; ++k)
            if ((jj >> k) & 1) a += beta[bp.B[st.slot_bit[k]]];
          hp.mats.push_back(R(std::cos(a)));
          hp.mats.push_back(R(std::sin(a)));
        }
        // inactive local bits only (slot bits are zero in r0)
        for (int x = 0; x < (1 << P.c0); ++x) {
          double a = 0;
          for (int k = 0; k < P.c0; ++k)
            if ((x >> k) & 1) a += beta[bp.B[k]];
          push(a);
        }
        for (int x = 0; x < (1 << P.c1); ++x) {
          double a = 0;
          for (int k = 0; k < P.c1; ++k)
            if ((x >> k) & 1) a += beta[bp.B[P.c0 + k]];
          push(a);
        }
        for (int ch = 0; ch < 3; ++ch)
          for (int x = 0; x < (1 << P.cg); ++x) {
            double a = ch == 0 ? c : 0.0;
            for (int k = 0; k < P.cg; ++k) {
              const int tb = ch * P.cg + k;
              if (!((x >> k) & 1)) continue;
              for (int b = 0; b < n; ++b)
                if (tbit_of[b] == tb) a += beta[b];
            }
            push(a);
          }
      }
      hp.ops.push_back(op);
    }
    st.nops = int(hp.ops.size()) - P.op0 - st.op0;
    hp.stages.push_back(st);
    rest.swap(skip);
  }
  P.nstages = int(hp.stages.size()) - P.stage0;
  P.nops = int(hp.ops.size()) - P.op0;
  P.nmat = int(hp.mats.size()) - P.mat0;
  hp.passes.push_back(P);
}

static int g_last_pass_count = 0;

// Register stage width SB (a thread holds 2^SB amplitudes) and block size of the tile
// pass per precision: blockDim = 2^(m - SB) <= NT with m = 13 (complex64) / 12.
template <typename R>
struct TileShape;
template <>
struct TileShape<float> {
  static constexpr int SB = 5, NT = 256;
};
template <>
struct TileShape<double> {
  static constexpr int SB = 4, NT = 256;
};

template <typename R>
static qc_status run_tiles(qc_state* s, const std::vector<ResolvedOp>& rops, int m) {
  const int n = s->n;
  const int L = sizeof(R) == 4 ? 4 : 3;
  constexpr int SB = TileShape<R>::SB;
  std::vector<PlanOp> pops;
  to_plan_ops(rops, pops);
  std::vector<BuiltPass> bps = build_passes(pops, n, m, L);
  HostPlan<R> hp;
  for (const BuiltPass& bp : bps) emit_pass<R>(bp, pops, n, m, L, SB, hp);
  g_last_pass_count = int(hp.passes.size());
  // upload stages, ops, tables and matrices into the state's scratch (stream ordered)
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t sb = al(hp.stages.size() * sizeof(TileStage));
  const size_t ob = al(hp.ops.size() * sizeof(TileOp));
  const size_t pb = al(hp.pool.size() * sizeof(R));
  const size_t mb = al(hp.mats.size() * sizeof(R));
  void* scr = nullptr;
  if (qc_status st = state_scratch(s, sb + ob + pb + mb + 256, &scr)) return st;
  char* base = static_cast<char*>(scr);
  std::vector<char> host(sb + ob + pb + mb, 0);
  if (!hp.stages.empty()) memcpy(host.data(), hp.stages.data(), hp.stages.size() * sizeof(TileStage));
  if (!hp.ops.empty()) memcpy(host.data() + sb, hp.ops.data(), hp.ops.size() * sizeof(TileOp));
  if (!hp.pool.empty()) memcpy(host.data() + sb + ob, hp.pool.data(), hp.pool.size() * sizeof(R));
  if (!hp.mats.empty()) memcpy(host.data() + sb + ob + pb, hp.mats.data(), hp.mats.size() * sizeof(R));
  if (qc_status st = check_cuda(cudaMemcpyAsync(base, host.data(), host.size(), cudaMemcpyHostToDevice, s->stream),
                                "plan upload"))
    return st;
  const TileStage* dst = reinterpret_cast<const TileStage*>(base);
  const TileOp* dop = reinterpret_cast<const TileOp*>(base + sb);
  const R* dpool = reinterpret_cast<const R*>(base + sb + ob);
  const R* dmats = reinterpret_cast<const R*>(base + sb + ob + pb);
  const int threads = 1 << (m - SB);
  size_t plan_max = 0;
  for (const TilePass& P : hp.passes)
    plan_max = std::max(plan_max, P.nstages * sizeof(TileStage) + P.nops * sizeof(TileOp) + P.nmat * sizeof(R));
  const size_t smem = 2 * sizeof(Cplx<R>) * (size_t(1) << m) + sizeof(uint64_t) * (size_t(1) << (m - L)) + plan_max;
  constexpr int NT = TileShape<R>::NT;
  if (qc_status st = check_cuda(
          cudaFuncSetAttribute(k_tile_pass<R, NT, SB>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)),
          "tile pass shared memory"))
    return st;
  const uint64_t ntiles = uint64_t(1) << (n - m);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_pass<R, NT, SB>, threads, smem);
  if (per_sm < 1) per_sm = 1;
  const uint64_t cap = uint64_t(device_sm_count()) * per_sm;
  const unsigned grid = unsigned(ntiles < cap ? ntiles : cap);
  R* a = reinterpret_cast<R*>(s->amps);
  for (const TilePass& P : hp.passes) {
    QC_COUNT(), k_tile_pass<R, NT, SB><<<grid, threads, smem, s->stream>>>(a, P, dst, dop, dpool, dmats);
  }
  return check_launch("tile pass");
}

int tile_bits_for(const qc_state* s) {
  const int want = s->dtype == QC_C64 ? 13 : 12;
  return std::min(want, s->n);
}

qc_status run_fused(qc_state* s, const qc_circuit* c, const double* params, qc_prec prec) {
  (void)prec;
  std::vector<ResolvedOp> rops(c->nops);
  for (int i = 0; i < c->nops; ++i)
    if (qc_status st = resolve_op(c, c->ops[i], params, &rops[i])) return st;
  const int m = tile_bits_for(s);
  if (s->n < 10 || m < kMaxStageBits + 4) return run_per_gate(s, c, params);
  return s->dtype == QC_C64 ? run_tiles<float>(s, rops, m) : run_tiles<double>(s, rops, m);
}

template <typename R>
static void plan_stats(int n, const std::vector<ResolvedOp>& rops, int m, int* passes, int* stages, int* ops) {
  const int L = sizeof(R) == 4 ? 4 : 3;
  constexpr int SB = TileShape<R>::SB;
  std::vector<PlanOp> pops;
  to_plan_ops(rops, pops);
  std::vector<BuiltPass> bps = build_passes(pops, n, m, L);
  HostPlan<R> hp;
  for (const BuiltPass& bp : bps) emit_pass<R>(bp, pops, n, m, L, SB, hp);
  *passes = int(hp.passes.size());
  *stages = int(hp.stages.size());
  *ops = int(hp.ops.size());
}

}  // namespace qcgb

using namespace qcgb;

extern "C" int qc_last_pass_count(void) { return qcgb::g_last_pass_count; }

extern "C" qc_status qc_plan_info(const qc_circuit* c, const double* params, qc_dtype dtype, int* passes,
                                  int* stages, int* ops) {
  clear_error();
  if (!c || c->n < 1 || c->n > 34 || (c->nops > 0 && !c->ops) || !passes || !stages || !ops ||
      (dtype != QC_C64 && dtype != QC_C128)) {
    set_error("qc_plan_info: invalid arguments");
    return QC_ERR_INVALID_ARG;
  }
  std::vector<ResolvedOp> rops(c->nops);
  for (int i = 0; i < c->nops; ++i)
    if (qc_status st = resolve_op(c, c->ops[i], params, &rops[i])) return st;
  const int m = std::min(dtype == QC_C64 ? 13 : 12, c->n);
  if (c->n < 10) {
    *passes = *stages = *ops = 0;
    return QC_OK;
  }
  if (dtype == QC_C64)
    plan_stats<float>(c->n, rops, m, passes, stages, ops);
  else
    plan_stats<double>(c->n, rops, m, passes, stages, ops);
  return QC_OK;
}
