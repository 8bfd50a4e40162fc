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
// Inside a pass the gates are split into stages; in a stage every thread holds 16
// amplitudes spanning 4 of the tile's bits in registers and applies all of the
// stage's gates to them before writing back to shared memory.  Shared memory is
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

constexpr int kStageBits = 4;
constexpr int kStageAmps = 1 << kStageBits;

enum TileOpType : int32_t { TOP_DENSE1 = 0, TOP_DENSE2 = 1, TOP_PHASE = 2 };

struct TileOp {
  int32_t type;
  int32_t s0, s1;        // stage slots of the targets (DENSE2: s0 = first qubit = row MSB)
  uint32_t lmask, lval;  // condition on the amplitude's local (in-tile) index
  int32_t pad;
  uint64_t gmask, gval;  // condition on the index bits outside the tile
  int64_t mat;           // DENSE: matrix / PHASE: 16-entry slot table, offset (R values) in
                         // the pass's matrix block
  int64_t tab;           // PHASE: offset (complex entries) of its other tables in the pool
};

struct TileStage {
  int32_t op0, nops;
  int8_t slot_bit[kStageBits];  // local bit of each slot
  int8_t sorted[kStageBits];    // the same bits ascending (zero-insertion order)
};

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
__device__ __forceinline__ uint32_t slot_off(int j, const uint32_t (&sm)[kStageBits]) {
  uint32_t o = 0;
#pragma unroll
  for (int k = 0; k < kStageBits; ++k)
    if ((j >> k) & 1) o |= sm[k];
  return o;
}

// swizzled address offset of slot combination j: XOR of the swizzled slot masks
// (the swizzle is linear over XOR, but swizzled masks may share bits)
__device__ __forceinline__ uint32_t slot_xor(int j, const uint32_t (&sw)[kStageBits]) {
  uint32_t o = 0;
#pragma unroll
  for (int k = 0; k < kStageBits; ++k)
    if ((j >> k) & 1) o ^= sw[k];
  return o;
}

template <typename R, int S0>
__device__ __forceinline__ void dense1(Cplx<R> (&v)[kStageAmps], const R* __restrict__ u, uint32_t r0,
                                       const uint32_t (&sm)[kStageBits], uint32_t lmask, uint32_t lval) {
  const Cplx<R> u00{u[0], u[1]}, u01{u[2], u[3]}, u10{u[4], u[5]}, u11{u[6], u[7]};
#pragma unroll
  for (int j = 0; j < kStageAmps; ++j) {
    if (j & (1 << S0)) continue;
    const int j1 = j | (1 << S0);
    if (((r0 | slot_off(j, sm)) & lmask) != lval) continue;
    const Cplx<R> x = v[j], y = v[j1];
    v[j] = cmul2(u00, x, u01, y);
    v[j1] = cmul2(u10, x, u11, y);
  }
}

template <typename R, int S0, int S1>
__device__ __forceinline__ void dense2(Cplx<R> (&v)[kStageAmps], const R* __restrict__ u) {
#pragma unroll
  for (int j = 0; j < kStageAmps; ++j) {
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

template <typename R>
__device__ __forceinline__ void apply_dense1(int s0, Cplx<R> (&v)[kStageAmps], const R* u, uint32_t r0,
                                             const uint32_t (&sm)[kStageBits], uint32_t lmask, uint32_t lval) {
  switch (s0) {
    case 0: dense1<R, 0>(v, u, r0, sm, lmask, lval); break;
    case 1: dense1<R, 1>(v, u, r0, sm, lmask, lval); break;
    case 2: dense1<R, 2>(v, u, r0, sm, lmask, lval); break;
    default: dense1<R, 3>(v, u, r0, sm, lmask, lval); break;
  }
}

template <typename R>
__device__ __forceinline__ void apply_dense2(int s0, int s1, Cplx<R> (&v)[kStageAmps], const R* u) {
  switch (s0 * 4 + s1) {
    case 1: dense2<R, 0, 1>(v, u); break;
    case 2: dense2<R, 0, 2>(v, u); break;
    case 3: dense2<R, 0, 3>(v, u); break;
    case 4: dense2<R, 1, 0>(v, u); break;
    case 6: dense2<R, 1, 2>(v, u); break;
    case 7: dense2<R, 1, 3>(v, u); break;
    case 8: dense2<R, 2, 0>(v, u); break;
    case 9: dense2<R, 2, 1>(v, u); break;
    case 11: dense2<R, 2, 3>(v, u); break;
    case 12: dense2<R, 3, 0>(v, u); break;
    case 13: dense2<R, 3, 1>(v, u); break;
    case 14: dense2<R, 3, 2>(v, u); break;
    default: break;
  }
}

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

// One launch = one pass over all tiles; blockDim = 2^(m-4), one block per SM with
// two tile buffers: the next tile is fetched (cp.async) while this one is computed.
template <typename R, int NT>
__global__ void __launch_bounds__(NT, 1) k_tile_pass(R* __restrict__ amps, const TilePass P,
                                                      const TileStage* __restrict__ stages,
                                                      const TileOp* __restrict__ ops, const R* __restrict__ pool,
                                                      const R* __restrict__ mats) {
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
  for (uint32_t h = threadIdx.x; h < (1u << nhi); h += blockDim.x) {
    uint64_t o = 0;
    for (int k = 0; k < nhi; ++k)
      if ((h >> k) & 1) o |= uint64_t(1) << P.bits[L + k];
    hioff[h] = o;
  }
  for (int i = threadIdx.x; i < P.nstages; i += blockDim.x) sst[i] = stages[P.stage0 + i];
  for (int i = threadIdx.x; i < P.nops; i += blockDim.x) sop[i] = ops[P.op0 + i];
  for (int i = threadIdx.x; i < P.nmat; i += blockDim.x) smat[i] = mats[P.mat0 + i];
  __syncthreads();
  const uint32_t lowmask = (1u << L) - 1;
  const Cplx<R>* cpool = reinterpret_cast<const Cplx<R>*>(pool);
  uint64_t t = blockIdx.x;
  if (t < P.ntiles) prefetch_tile<R>(bufs, amps, insert_zero_bits(t, P.bits, m), hioff, L, T);
  cp_async_commit();
  for (int it = 0; t < P.ntiles; t += gridDim.x, ++it) {
    Cplx<R>* tile = bufs + (it & 1) * T;
    const uint64_t base = insert_zero_bits(t, P.bits, m);
    const uint64_t tn = t + gridDim.x;
    if (tn < P.ntiles) prefetch_tile<R>(bufs + ((it + 1) & 1) * T, amps, insert_zero_bits(tn, P.bits, m), hioff, L, T);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    for (int s = 0; s < P.nstages; ++s) {
      const TileStage st = sst[s];
      const uint32_t r0 = uint32_t(insert_zero_bits(threadIdx.x, st.sorted, kStageBits));
      uint32_t sm[kStageBits], sw[kStageBits];
#pragma unroll
      for (int k = 0; k < kStageBits; ++k) {
        sm[k] = 1u << st.slot_bit[k];
        sw[k] = tile_swz(sm[k]);  // the swizzle is linear over XOR: swz(a^b) = swz(a)^swz(b)
      }
      const uint32_t p0 = tile_swz(r0);
      Cplx<R> v[kStageAmps];
#pragma unroll
      for (int j = 0; j < kStageAmps; ++j) v[j] = tile[p0 ^ slot_xor(j, sw)];
      for (int q = 0; q < st.nops; ++q) {
        const TileOp& op = sop[st.op0 + q];
        if ((base & op.gmask) != op.gval) continue;
        if (op.type == TOP_DENSE1) {
          apply_dense1<R>(op.s0, v, smat + op.mat, r0, sm, op.lmask, op.lval);
        } else if (op.type == TOP_DENSE2) {
          apply_dense2<R>(op.s0, op.s1, v, smat + op.mat);
        } else {
          // exp(i (c + sum beta_p b_p)) factorised over: tile-index chunks (3), the
          // thread's inactive local bits (2 chunks) and the 16 slot combinations
          const Cplx<R>* jt = reinterpret_cast<const Cplx<R>*>(smat + op.mat);
          const Cplx<R>* l0 = cpool + op.tab;
          const Cplx<R>* l1 = l0 + (1 << P.c0);
          const Cplx<R>* g0 = l1 + (1 << (m - P.c0));
          const uint32_t gn = 1u << P.cg, gm = gn - 1;
          Cplx<R> w = cmul(cmul(g0[t & gm], g0[gn + ((t >> P.cg) & gm)]), g0[2 * gn + ((t >> (2 * P.cg)) & gm)]);
          w = cmul(w, cmul(l0[r0 & ((1u << P.c0) - 1)], l1[r0 >> P.c0]));
#pragma unroll
          for (int j = 0; j < kStageAmps; ++j) {
            if (((r0 | slot_off(j, sm)) & op.lmask) != op.lval) continue;
            v[j] = cmul(v[j], cmul(w, jt[j]));
          }
        }
      }
#pragma unroll
      for (int j = 0; j < kStageAmps; ++j) tile[p0 ^ slot_xor(j, sw)] = v[j];
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
      p.c = std::arg(d0);
      p.beta = {{tgt, std::arg(d1) - std::arg(d0)}};
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

static std::vector<BuiltPass> build_passes(const std::vector<PlanOp>& ops, int n, int m, int L) {
  std::vector<int> remaining(ops.size());
  for (size_t i = 0; i < ops.size(); ++i) remaining[i] = int(i);
  std::vector<BuiltPass> passes;
  while (!remaining.empty()) {
    BuiltPass bp;
    uint64_t Bmask = (uint64_t(1) << L) - 1;
    int Bcount = L;
    uint64_t blocked_all = 0;   // bits of excluded non-diagonal ops
    uint64_t blocked_diag = 0;  // bits of excluded diagonal ops
    std::vector<int> excluded;
    for (int idx : remaining) {
      const PlanOp& p = ops[idx];
      bool ok = (p.touched & blocked_all) == 0 && int(bp.ops.size()) < kMaxPassOps;
      if (ok && !p.phase) ok = (p.touched & blocked_diag) == 0;
      if (ok && !p.phase) {
        uint64_t need = 0;
        for (int k = 0; k < p.nt; ++k) need |= uint64_t(1) << p.tb[k];
        need &= ~Bmask;
        const int add = __builtin_popcountll(need);
        if (Bcount + add <= m) {
          Bmask |= need;
          Bcount += add;
        } else {
          ok = false;
        }
      }
      if (ok) {
        bp.ops.push_back(idx);
      } else {
        excluded.push_back(idx);
        if (p.phase)
          blocked_diag |= p.touched;
        else
          blocked_all |= p.touched;
      }
    }
    // fill B up to m bits with the lowest free bits (a full tile)
    for (int b = 0; Bcount < m && b < n; ++b)
      if (!((Bmask >> b) & 1)) {
        Bmask |= uint64_t(1) << b;
        ++Bcount;
      }
    for (int b = 0; b < n; ++b)
      if ((Bmask >> b) & 1) bp.B.push_back(b);
    passes.push_back(bp);
    remaining.swap(excluded);
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
static void emit_pass(const BuiltPass& bp, const std::vector<PlanOp>& pops, int n, int m, int L, HostPlan<R>& hp) {
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
        if (int(nw.size()) > kStageBits)
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
    for (int b = 0; int(act.size()) < kStageBits && b < m; ++b)
      if (std::find(act.begin(), act.end(), b) == act.end()) act.push_back(b);
    TileStage st{};
    for (int k = 0; k < kStageBits; ++k) st.slot_bit[k] = int8_t(act[k]);
    std::vector<int> srt = act;
    std::sort(srt.begin(), srt.end());
    for (int k = 0; k < kStageBits; ++k) st.sorted[k] = int8_t(srt[k]);
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
          for (int k = 0; k < kStageBits; ++k)
            if (st.slot_bit[k] == lb) return k;
          return -1;
        };
        op.s0 = slot(p.tb[0]);
        op.s1 = p.nt == 2 ? slot(p.tb[1]) : 0;
        op.mat = int64_t(hp.mats.size()) - P.mat0;
        for (int e = 0; e < (p.nt == 1 ? 8 : 32); ++e) hp.mats.push_back(R(p.m[e]));
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
        for (int jj = 0; jj < kStageAmps; ++jj) {
          double a = 0;
          for (int k = 0; k < kStageBits; ++k)
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

template <typename R>
static qc_status run_tiles(qc_state* s, const std::vector<ResolvedOp>& rops, int m) {
  const int n = s->n;
  const int L = sizeof(R) == 4 ? 4 : 3;
  std::vector<PlanOp> pops;
  to_plan_ops(rops, pops);
  std::vector<BuiltPass> bps = build_passes(pops, n, m, L);
  HostPlan<R> hp;
  for (const BuiltPass& bp : bps) emit_pass<R>(bp, pops, n, m, L, hp);
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
  const int threads = 1 << (m - kStageBits);
  size_t plan_max = 0;
  for (const TilePass& P : hp.passes)
    plan_max = std::max(plan_max, P.nstages * sizeof(TileStage) + P.nops * sizeof(TileOp) + P.nmat * sizeof(R));
  const size_t smem = 2 * sizeof(Cplx<R>) * (size_t(1) << m) + sizeof(uint64_t) * (size_t(1) << (m - L)) + plan_max;
  constexpr int NT = sizeof(R) == 4 ? 512 : 256;
  cudaFuncSetAttribute(k_tile_pass<R, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  const uint64_t ntiles = uint64_t(1) << (n - m);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_pass<R, NT>, threads, smem);
  if (per_sm < 1) per_sm = 1;
  const uint64_t cap = uint64_t(device_sm_count()) * per_sm;
  const unsigned grid = unsigned(ntiles < cap ? ntiles : cap);
  R* a = reinterpret_cast<R*>(s->amps);
  for (const TilePass& P : hp.passes) {
    QC_COUNT(), k_tile_pass<R, NT><<<grid, threads, smem, s->stream>>>(a, P, dst, dop, dpool, dmats);
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
  if (s->n < 10 || m < kStageBits + 4) return run_per_gate(s, c, params);
  return s->dtype == QC_C64 ? run_tiles<float>(s, rops, m) : run_tiles<double>(s, rops, m);
}

}  // namespace qcgb

extern "C" int qc_last_pass_count(void) { return qcgb::g_last_pass_count; }
