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
// amplitudes spanning SB of the tile's bits in registers (SB = 4 for both precisions;
// 3 for the double-float complex128 passes) and applies all of the stage's gates to them before writing back to
// shared memory.  Shared memory is
// addressed through an XOR swizzle so that the strided accesses of a stage do not
// collide in the same bank.
#include <string.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <mutex>
#include <map>
#include <string>
#include <unordered_map>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "circuit.cuh"
#include "common.cuh"
#include "kernels.cuh"
#include "tiles.cuh"

namespace qcgb {

// One launch = one pass over all tiles; blockDim = 2^(m-SB), one block per SM with
// two tile buffers: the next tile is fetched (cp.async) while this one is computed.
// EXTOPS: the plan contains CZ sign ops or single-bit phase ops (a second instantiation
// without them keeps the gate bodies' code generation unchanged for plans that have
// none, e.g. circuits of dense two-qubit gates)
template <typename R, int NT, int SB, bool EXTOPS>
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
  // write-out gather after relabeled swaps: tile position of output local index u is
  // rlo[u mod 2^L] | rhi[u >> L]
  uint32_t* rhi = reinterpret_cast<uint32_t*>(hioff + (1u << nhi));
  uint64_t* tnt = reinterpret_cast<uint64_t*>(rhi + (1u << nhi));  // tile number -> base
  // the pass's plan, copied once into shared memory: stages, ops, matrices
  TileStage* sst = reinterpret_cast<TileStage*>(tnt + kTileNumberTab);
  TileOp* sop = reinterpret_cast<TileOp*>(sst + P.nstages);
  R* smat = reinterpret_cast<R*>(sop + P.nops);
  // the pass's phase tables (16-byte aligned after the matrices), when they fit
  R* spool = reinterpret_cast<R*>(smat + ((P.nmat + 3) & ~3));
  // the tile's bit positions in shared memory (a dynamically indexed kernel parameter
  // array would be copied to local memory)
  __shared__ int8_t sbits[16], srbit[16];
  __shared__ uint32_t rlo[16];
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      sbits[k] = P.bits[k];
      srbit[k] = P.rbit[k];
    }
  }
  __syncthreads();
  for (uint32_t h = threadIdx.x; h < (1u << nhi); h += blockDim.x) {
    uint64_t o = 0;
    for (int k = 0; k < nhi; ++k)
      if ((h >> k) & 1) o |= uint64_t(1) << sbits[L + k];
    hioff[h] = o;
  }
  if constexpr (EXTOPS) {
    for (uint32_t h = threadIdx.x; h < (1u << nhi); h += blockDim.x) {
      uint32_t q = 0;
      for (int k = 0; k < nhi; ++k)
        if ((h >> k) & 1) q |= 1u << srbit[L + k];
      rhi[h] = q;
    }
    if (threadIdx.x < (1u << L)) {
      uint32_t q = 0;
      for (int k = 0; k < L; ++k)
        if ((threadIdx.x >> k) & 1) q |= 1u << srbit[k];
      rlo[threadIdx.x] = q;
    }
  }
  build_tile_number_tables(tnt, sbits, m, __ffsll(static_cast<long long>(P.ntiles)) - 1);
  for (int i = threadIdx.x; i < P.nstages; i += blockDim.x) sst[i] = stages[P.stage0 + i];
  for (int i = threadIdx.x; i < P.nops; i += blockDim.x) sop[i] = ops[P.op0 + i];
  for (int i = threadIdx.x; i < P.nmat; i += blockDim.x) smat[i] = mats[P.mat0 + i];
  if (P.spool)
    for (int i = threadIdx.x; i < P.npool; i += blockDim.x) spool[i] = pool[P.pool0 + i];
  __syncthreads();
  const uint32_t lowmask = (1u << L) - 1;
  // table offsets (op.tab) count complex entries from the start of the pool
  const Cplx<R>* cpool = P.spool ? reinterpret_cast<const Cplx<R>*>(spool) - P.pool0 / 2
                                 : reinterpret_cast<const Cplx<R>*>(pool);
  uint64_t t = blockIdx.x;
  if (t < P.ntiles) prefetch_tile<R>(bufs, amps, tile_base(t, tnt), hioff, L, T);
  cp_async_commit();
  for (int it = 0; t < P.ntiles; t += gridDim.x, ++it) {
    Cplx<R>* tile = bufs + (it & 1) * T;
    const uint64_t base = tile_base(t, tnt);
    const uint64_t tn = t + gridDim.x;
    if (tn < P.ntiles) prefetch_tile<R>(bufs + ((it + 1) & 1) * T, amps, tile_base(tn, tnt), hioff, L, T);
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
      for (int k = 0; k < SB; ++k)
        sw[k] = tile_swz(1u << st.slot_bit[k]);  // the swizzle is linear over XOR: swz(a^b) = swz(a)^swz(b)
      const uint32_t p0 = tile_swz(r0);
      Cplx<R> v[NA];
#pragma unroll
      for (int j = 0; j < NA; ++j) v[j] = tile[p0 ^ slot_xor<SB>(j, sw)];
      for (int q = 0; q < st.nops; ++q) {
        const TileOp op = sop[st.op0 + q];  // one copy into registers
        if ((base & op.gmask) != op.gval) continue;  // condition on bits outside the tile
        if ((r0 & op.lmask) != op.lval) continue;    // ... on the thread's lane bits
        if (op.type == TOP_DENSE1) {
          apply_dense1<R, SB>(op.s0, v, smat + op.mat, op.jmask);
        } else if (op.type == TOP_DENSE2) {
          apply_dense2<R, SB>(op.s0, op.s1, v, smat + op.mat);
        } else if (sizeof(R) == 8 && op.type == TOP_SWAP) {
          if constexpr (sizeof(R) == 8) apply_swap<R, SB>(op.s0, op.s1, v);
        } else if (EXTOPS && op.type == TOP_CZSET) {
          if constexpr (EXTOPS) {
            const uint32_t flip = czset_flips<R, SB>(smat + op.mat, op.s0, r0, base);
#pragma unroll
            for (int j = 0; j < NA; ++j)
              if ((flip >> j) & 1u) v[j] = Cplx<R>{-v[j].re, -v[j].im};
          }
        } else if (sizeof(R) == 8 && EXTOPS && op.type == TOP_BFLY) {
          if constexpr (sizeof(R) == 8 && EXTOPS) apply_bfly<R, SB>(op.s0, v, smat + op.mat, op.jmask);
        } else if (sizeof(R) == 8 && EXTOPS && op.type == TOP_REAL1) {
          if constexpr (sizeof(R) == 8 && EXTOPS) apply_real1<R, SB>(op.s0, v, smat + op.mat, op.jmask);
        } else if (EXTOPS && op.type == TOP_PHASE1) {
          if constexpr (EXTOPS) {
            const uint32_t fixed =
                op.s0 >= 0 ? 0u : op.zloc >= 0 ? (r0 >> op.zloc) & 1u : uint32_t((base >> op.zglob) & 1u);
            apply_phase1<R, SB>(v, smat + op.mat, op.s0, fixed, op.jmask);
          }
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
            if (!((op.jmask >> j) & 1u)) continue;  // ... on the slot bits
            v[j] = cmul(v[j], cmul(w, jt[j]));
          }
        }
      }
#pragma unroll
      for (int j = 0; j < NA; ++j) tile[p0 ^ slot_xor<SB>(j, sw)] = v[j];
      if (st.warp_local)
        __syncwarp();  // the next stage gives this warp the same amplitudes
      else
        __syncthreads();
    }
    if constexpr (EXTOPS) {
      // (identity tables unless the pass relabeled swaps; plans with relabeled swaps
      // run this variant)
      for (uint32_t e = threadIdx.x; e < T / 2; e += blockDim.x) {
        const uint32_t u = 2 * e;
        const uint64_t gi = base | hioff[u >> L] | (u & lowmask);
        const uint32_t hi = rhi[u >> L];
        st_amp2<R>(amps, gi, tile[tile_swz(hi | rlo[u & lowmask])], tile[tile_swz(hi | rlo[(u | 1u) & lowmask])]);
      }
    } else {
      for (uint32_t e = threadIdx.x; e < T / 2; e += blockDim.x) {
        const uint32_t r = 2 * e;
        const uint64_t gi = base | hioff[r >> L] | (r & lowmask);
        const uint32_t p = tile_swz(r);
        st_amp2<R>(amps, gi, tile[p], tile[p ^ 1u]);
      }
    }
    __syncthreads();  // this buffer is refilled two iterations later
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// ---------------------------------------------------------------------------
// host planner
// ---------------------------------------------------------------------------
using cd = std::complex<double>;

static bool near_unit(cd z) { return std::abs(std::abs(z) - 1.0) < 1e-12; }

// Converts resolved gates to plan ops; diagonal gates become phase ops.
void to_plan_ops(const std::vector<ResolvedOp>& in, std::vector<PlanOp>& out, const std::vector<int>* grad,
                 const std::vector<int>* gen) {
  for (size_t i = 0; i < in.size(); ++i) {
    const ResolvedOp& r = in[i];
    PlanOp p{};
    p.cmask = p.cval = 0;
    if (grad && (*grad)[i] >= 0) {
      // a recorded rotation: X/Y generators stay dense 2x2 (even where the matrix
      // happens to be diagonal), Z rotations are phase ops on their own bit
      const int tgt = r.bits[0];
      p.grad = (*grad)[i];
      p.gen = (*gen)[i];
      p.touched = uint64_t(1) << tgt;
      if (p.gen == 2) {
        p.phase = true;
        p.c = std::arg(cd(r.m[0], r.m[1]));
        p.beta = {{tgt, std::arg(cd(r.m[6], r.m[7])) - std::arg(cd(r.m[0], r.m[1]))}};
      } else {
        p.phase = false;
        p.nt = 1;
        p.tb[0] = tgt;
        memcpy(p.m, r.m, sizeof(double) * 8);
      }
      out.push_back(p);
      continue;
    }
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
        if (t00 != 0.0 || t10 != t00 || t01 != t00) out.push_back(q);  // skip the identity
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



// One pass over `remaining` in order.  With `fixed` set, B is exactly `B0` (ops whose
// dense targets are outside it are skipped); otherwise B starts as B0 and grows to m
// bits with the targets of the first ops that need them.  An op is taken unless it
// meets a skipped op it may not commute with (shared bits; two diagonal ops commute).
static void greedy_pass(const std::vector<PlanOp>& ops, const std::vector<int>& remaining, int m, uint64_t B0,
                        bool fixed, bool cond_in_tile, BuiltPass* bp, std::vector<int>* excluded, uint64_t* Bout,
                        double* score) {
  uint64_t Bmask = B0;
  int Bcount = __builtin_popcountll(B0);
  uint64_t blocked_all = 0;   // bits of skipped non-diagonal ops
  uint64_t blocked_diag = 0;  // bits of skipped diagonal ops
  double sc = 0.0;
  for (int idx : remaining) {
    const PlanOp& p = ops[idx];
    bool ok = (p.touched & blocked_all) == 0 && int(bp->ops.size()) < kMaxPassOps;
    if (ok && !p.phase) ok = (p.touched & blocked_diag) == 0;
    if (ok && (!p.phase || (cond_in_tile && p.cmask))) {
      uint64_t need = cond_in_tile ? p.cmask : 0;
      if (!p.phase)
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

static std::vector<BuiltPass> build_passes_uncached(const std::vector<PlanOp>& ops, int n, int m, int L,
                                                    bool cond_in_tile) {
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
        greedy_pass(ops, remaining, m, low, false, cond_in_tile, &bp, &ex, &Bm, &sc);
      } else {
        const uint64_t win = ((uint64_t(1) << w) - 1) << (L + cand);
        greedy_pass(ops, remaining, m, low | win, true, cond_in_tile, &bp, &ex, &Bm, &sc);
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

// The pass structure depends only on each op's kind, targets and touched bits -- not on
// its matrix or angles -- so it is reused when a circuit is run again with other
// parameters (training loops, repeated gradients).  A few recent structures are kept.
struct PassCacheEntry {
  std::vector<int64_t> key;
  std::vector<BuiltPass> passes;
};
static std::mutex g_pass_cache_mu;
static std::vector<PassCacheEntry> g_pass_cache;  // most recent last
constexpr size_t kPassCacheEntries = 8;

std::vector<BuiltPass> build_passes(const std::vector<PlanOp>& ops, int n, int m, int L, bool cond_in_tile) {
  std::vector<int64_t> key;
  key.reserve(4 + 5 * ops.size());
  key.push_back(n);
  key.push_back(m);
  key.push_back(L);
  key.push_back(cond_in_tile ? 1 : 0);
  for (const PlanOp& p : ops) {
    key.push_back(p.phase ? -1 : p.nt);
    key.push_back(p.phase ? 0 : p.tb[0]);
    key.push_back(!p.phase && p.nt == 2 ? p.tb[1] : 0);
    key.push_back(int64_t(p.touched));
    if (cond_in_tile) key.push_back(int64_t(p.cmask));
  }
  {
    std::lock_guard<std::mutex> lock(g_pass_cache_mu);
    for (size_t e = 0; e < g_pass_cache.size(); ++e)
      if (g_pass_cache[e].key == key) {
        PassCacheEntry hit = std::move(g_pass_cache[e]);
        g_pass_cache.erase(g_pass_cache.begin() + long(e));
        g_pass_cache.push_back(std::move(hit));
        return g_pass_cache.back().passes;
      }
  }
  std::vector<BuiltPass> passes = build_passes_uncached(ops, n, m, L, cond_in_tile);
  std::lock_guard<std::mutex> lock(g_pass_cache_mu);
  if (g_pass_cache.size() >= kPassCacheEntries) g_pass_cache.erase(g_pass_cache.begin());
  g_pass_cache.push_back(PassCacheEntry{std::move(key), passes});
  return passes;
}


// Slot and thread-index bits of each stage of a pass.  acts[s] holds the local bits
// stage s's gates act on (at most sb); it is padded to sb slot bits, and the other
// m - sb local bits receive the thread-index bits: the first ones (lanes) one local bit
// per residue mod nres, so that a half warp's shared-memory accesses fall in distinct
// banks; the bits from 5 up pick the warp, so they fix the set of amplitudes a warp
// holds.  Those warp bits are kept the same over runs of consecutive stages (disjoint
// from every slot of the run), chosen greedily to make each run as long as possible
// (which gives the fewest runs): inside a run a warp only exchanges amplitudes with
// itself, and a warp barrier replaces the block barrier between its stages.
// Register stages of a pass: each takes, in order, every remaining op of the pass whose
// dense targets fit in <= sb active local bits and that no skipped op it fails to
// commute with precedes (same rule as for passes); skipped ops go to later stages in
// order.  takes[s]: the ops of stage s; acts[s]: the local bits their targets occupy.
// With whole_ops, an op's in-tile control and phase bits count as active bits too (a
// stage applied as one block must see every bit its ops depend on).
// One stage over `rest` (in order): an op is taken if the local bits it needs join the
// stage's set without exceeding sb bits (with `fixed` >= 0: stay inside that set of
// local bits) and no skipped op it fails to commute with precedes it.
static void stage_sweep(const std::vector<int>& rest, const std::vector<PlanOp>& pops, const int* local_of, int sb,
                        int whole_ops, int64_t fixed, std::vector<int>& take, std::vector<int>& skip,
                        std::vector<int>& act) {
  take.clear();
  skip.clear();
  // the stage's local bits in the order they joined (av) and as a mask; an op's trial set
  // is built in nv / nmask and kept if it fits
  int av[64], nv[64];
  int na = 0;
  uint64_t amask = 0;
  uint64_t blocked_all = 0, blocked_diag = 0;
  // mode 2: condition bits of phase ops whose other bits may be deferred past the stage;
  // a dense op on one of them would not commute with that deferred part
  uint64_t dblock = 0;
  for (int idx : rest) {
    const PlanOp& p = pops[idx];
    bool ok = (p.touched & blocked_all) == 0;
    if (ok && !p.phase) ok = (p.touched & blocked_diag) == 0;
    if (ok && !p.phase && whole_ops == 2)
      for (int k = 0; k < p.nt; ++k)
        if ((dblock >> p.tb[k]) & 1) ok = false;
    if (ok && (whole_ops || !p.phase)) {
      int nn = na;
      uint64_t nmask = amask;
      for (int i = 0; i < na; ++i) nv[i] = av[i];
      bool outside = false;
      auto add = [&](int gbit) {
        const int lb = local_of[gbit];
        if (lb < 0) return;
        if (fixed >= 0 && !((fixed >> lb) & 1)) outside = true;
        if (!((nmask >> lb) & 1)) {
          nmask |= uint64_t(1) << lb;
          nv[nn++] = lb;
        }
      };
      if (!p.phase)
        for (int k = 0; k < p.nt; ++k) add(p.tb[k]);
      if (whole_ops) {
        for (uint64_t cm = p.cmask; cm; cm &= cm - 1) add(__builtin_ctzll(cm));
        // mode 2: the phase bits of an op conditioned on at most one bit need no slot
        // (that part of the op is deferred to the end of the stage)
        if (whole_ops == 1 || !p.phase || __builtin_popcountll(p.cmask) >= 2)
          for (const auto& be : p.beta) add(be.first);
      }
      if (outside || nn > sb) {
        ok = false;
      } else {
        for (int i = na; i < nn; ++i) av[i] = nv[i];
        na = nn;
        amask = nmask;
      }
      if (ok && whole_ops == 2 && p.phase && __builtin_popcountll(p.cmask) == 1)
        for (const auto& be : p.beta) {
          const int lb = local_of[be.first];
          if (lb < 0 || !((amask >> lb) & 1)) dblock |= p.cmask;
        }
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
  act.assign(av, av + na);
}

void split_stages(const BuiltPass& bp, const std::vector<PlanOp>& pops, const int* local_of, int sb,
                  std::vector<std::vector<int>>& takes, std::vector<std::vector<int>>& acts, int whole_ops) {
  int m = 0;
  for (int b = 0; b < 64; ++b) m = std::max(m, local_of[b] + 1);
  std::vector<int> rest = bp.ops;
  std::vector<int> take, skip, act, btake, bskip, bact;
  while (!rest.empty()) {
    // candidates: the growing first-fit set, and every window of sb neighbouring local
    // bits; the one that takes the most ops wins (the first-fit set on ties)
    stage_sweep(rest, pops, local_of, sb, whole_ops, -1, btake, bskip, bact);
    for (int w = 0; w + sb <= m; ++w) {
      stage_sweep(rest, pops, local_of, sb, whole_ops, ((int64_t(1) << sb) - 1) << w, take, skip, act);
      if (take.size() > btake.size()) {
        btake.swap(take);
        bskip.swap(skip);
        bact.swap(act);
      }
    }
    takes.push_back(btake);
    acts.push_back(bact);
    rest.swap(bskip);
  }
}

// The candidate stages over `rest` (the growing first-fit set and every window of sb
// neighbouring local bits), without repeats
struct StageCand {
  std::vector<int> take, skip, act;
};
static std::vector<StageCand> stage_candidates(const std::vector<int>& rest, const std::vector<PlanOp>& pops,
                                               const int* local_of, int sb, int whole_ops, int m) {
  std::vector<StageCand> out;
  auto push = [&](int64_t fixed) {
    StageCand c;
    stage_sweep(rest, pops, local_of, sb, whole_ops, fixed, c.take, c.skip, c.act);
    if (c.take.empty()) return;
    for (const StageCand& o : out)
      if (o.take == c.take) return;
    out.push_back(std::move(c));
  };
  push(-1);
  for (int w = 0; w + sb <= m; ++w) push(((int64_t(1) << sb) - 1) << w);
  return out;
}

// Greedy stage counts of op sets met during one search: the greedy cuts from different
// branches run into the same remaining sets, so each set is cut once
struct OpSetHash {
  size_t operator()(const std::vector<int>& v) const {
    uint64_t h = 1469598103934665603ull;  // FNV-style: one 32-bit index per step
    for (int x : v) {
      h ^= uint32_t(x);
      h *= 1099511628211ull;
    }
    return size_t(h);
  }
};
using GreedyMemo = std::unordered_map<std::vector<int>, int, OpSetHash>;
constexpr int kNoCut = 1 << 20;  // some op fits no stage

// stages the greedy cut (most ops per stage; the first such candidate) needs for `rest`;
// kNoCut if it reaches ops that fit no stage
static int greedy_stage_count(const std::vector<int>& rest, const std::vector<PlanOp>& pops, const int* local_of,
                              int sb, int whole_ops, int m, GreedyMemo& memo) {
  std::vector<std::vector<int>> chain;  // the sets the cut walks through, not yet known
  std::vector<int> cur = rest;
  int tail;
  while (true) {
    if (cur.empty()) {
      tail = 0;
      break;
    }
    const auto it = memo.find(cur);
    if (it != memo.end()) {
      tail = it->second;
      break;
    }
    std::vector<StageCand> cs = stage_candidates(cur, pops, local_of, sb, whole_ops, m);
    if (cs.empty()) {
      memo.emplace(cur, kNoCut);
      tail = kNoCut;
      break;
    }
    size_t best = 0;
    for (size_t i = 1; i < cs.size(); ++i)
      if (cs[i].take.size() > cs[best].take.size()) best = i;
    chain.push_back(std::move(cur));
    cur = std::move(cs[best].skip);
  }
  int v = tail;
  for (size_t i = chain.size(); i-- > 0;) {
    v = v == kNoCut ? kNoCut : v + 1;
    memo.emplace(std::move(chain[i]), v);
  }
  return v;
}

// stages needed for `rest` when the next `depth` stages are chosen by search and the
// rest greedily
static int lookahead_stage_count(const std::vector<int>& rest, const std::vector<PlanOp>& pops, const int* local_of,
                                 int sb, int whole_ops, int m, int depth, GreedyMemo& memo) {
  if (rest.empty()) return 0;
  if (depth == 0) return greedy_stage_count(rest, pops, local_of, sb, whole_ops, m, memo);
  int best = kNoCut;
  for (const StageCand& c : stage_candidates(rest, pops, local_of, sb, whole_ops, m))
    best = std::min(best, 1 + lookahead_stage_count(c.skip, pops, local_of, sb, whole_ops, m, depth - 1, memo));
  return best;
}

void split_stages_search(const BuiltPass& bp, const std::vector<PlanOp>& pops, const int* local_of, int sb,
                         std::vector<std::vector<int>>& takes, std::vector<std::vector<int>>& acts, int whole_ops,
                         int depth);

// The searched cuts depend only on the pass's structure -- each op's kind, bits, condition
// and phase bits, the tile's local bits -- not on matrices or angles, so they are kept
// for reuse when a circuit runs again with other parameters (a training loop): the
// search costs far more than the rest of the plan.  Cuts are stored as positions in
// bp.ops; a bounded number of recent ones are kept.
struct StageCutEntry {
  std::vector<int64_t> key;
  std::vector<std::vector<int>> takes, acts;  // takes: positions in bp.ops
};
static std::mutex g_cut_mu;
static std::vector<StageCutEntry> g_cuts;  // most recent last
constexpr size_t kStageCutEntries = 512;

static std::vector<int64_t> stage_cut_key(const BuiltPass& bp, const std::vector<PlanOp>& pops, const int* local_of,
                                          int sb, int whole_ops, int depth) {
  std::vector<int64_t> key = {sb, whole_ops, depth};
  for (int b : bp.B) key.push_back(int64_t(b) * 64 + local_of[b]);
  for (int idx : bp.ops) {
    const PlanOp& p = pops[size_t(idx)];
    key.push_back(p.phase ? -1 : p.nt);
    key.push_back(p.phase ? 0 : int64_t(p.tb[0]) * 64 + (p.nt == 2 ? p.tb[1] : 0));
    key.push_back(int64_t(p.touched));
    key.push_back(int64_t(p.cmask));
    key.push_back(int64_t(p.cval));
    uint64_t bb = 0;
    for (const auto& be : p.beta) bb |= uint64_t(1) << be.first;
    key.push_back(int64_t(bb));
  }
  return key;
}

void split_stages_lookahead(const BuiltPass& bp, const std::vector<PlanOp>& pops, const int* local_of, int sb,
                            std::vector<std::vector<int>>& takes, std::vector<std::vector<int>>& acts, int whole_ops,
                            int depth) {
  const std::vector<int64_t> key = stage_cut_key(bp, pops, local_of, sb, whole_ops, depth);
  {
    std::lock_guard<std::mutex> lock(g_cut_mu);
    for (size_t e = 0; e < g_cuts.size(); ++e)
      if (g_cuts[e].key == key) {
        for (const std::vector<int>& t : g_cuts[e].takes) {
          takes.emplace_back();
          for (int pos : t) takes.back().push_back(bp.ops[size_t(pos)]);
        }
        for (const std::vector<int>& a : g_cuts[e].acts) acts.push_back(a);
        return;
      }
  }
  const size_t t0 = takes.size(), a0 = acts.size();
  split_stages_search(bp, pops, local_of, sb, takes, acts, whole_ops, depth);
  StageCutEntry ent;
  ent.key = key;
  for (size_t i = t0; i < takes.size(); ++i) {
    ent.takes.emplace_back();
    for (int idx : takes[i]) {
      const auto it = std::find(bp.ops.begin(), bp.ops.end(), idx);
      ent.takes.back().push_back(int(it - bp.ops.begin()));
    }
  }
  for (size_t i = a0; i < acts.size(); ++i) ent.acts.push_back(acts[i]);
  std::lock_guard<std::mutex> lock(g_cut_mu);
  if (g_cuts.size() >= kStageCutEntries) g_cuts.erase(g_cuts.begin());
  g_cuts.push_back(std::move(ent));
}

void split_stages_search(const BuiltPass& bp, const std::vector<PlanOp>& pops, const int* local_of, int sb,
                         std::vector<std::vector<int>>& takes, std::vector<std::vector<int>>& acts, int whole_ops,
                         int depth) {
  int m = 0;
  for (int b = 0; b < 64; ++b) m = std::max(m, local_of[b] + 1);
  std::vector<int> rest = bp.ops;
  GreedyMemo memo;
  while (!rest.empty()) {
    std::vector<StageCand> cs = stage_candidates(rest, pops, local_of, sb, whole_ops, m);
    if (cs.empty()) {  // (no op fits: leave them to the caller's checks, as the greedy cut does)
      split_stages(BuiltPass{bp.B, rest}, pops, local_of, sb, takes, acts, whole_ops);
      return;
    }
    size_t best = 0;
    int best_n = kNoCut;
    for (size_t i = 0; i < cs.size(); ++i) {
      const int nst = 1 + lookahead_stage_count(cs[i].skip, pops, local_of, sb, whole_ops, m, depth - 1, memo);
      if (nst < best_n || (nst == best_n && cs[i].take.size() > cs[best].take.size())) {
        best_n = nst;
        best = i;
      }
    }
    takes.push_back(cs[best].take);
    acts.push_back(cs[best].act);
    rest = cs[best].skip;
  }
}

std::vector<TileStage> stage_layouts(const std::vector<std::vector<int>>& acts, int m, int sb, int nres) {
  const int nthr = m - sb;
  const int nl = std::min(nthr, 5), nw = nthr - nl;
  const int need = std::min(nres, nl);
  const uint32_t all = (1u << m) - 1;
  auto resmask = [&](int r) {
    uint32_t mk = 0;
    for (int b = r; b < m; b += 4) mk |= 1u << b;
    return mk;
  };
  std::vector<uint32_t> amask(acts.size(), 0);
  for (size_t s = 0; s < acts.size(); ++s)
    for (int b : acts[s]) amask[s] |= 1u << b;
  // stage s can take warp bits W: W misses its active bits and the remaining bits hold
  // every residue the lanes need (padding then takes only surplus bits)
  auto fits = [&](size_t s, uint32_t W) {
    if (W & amask[s]) return false;
    const uint32_t rest = all & ~(amask[s] | W);
    for (int r = 0; r < need; ++r)
      if (!(rest & resmask(r))) return false;
    return true;
  };
  std::vector<uint32_t> wsets;
  for (uint32_t W = all;; W = (W - 1) & all) {  // descending: high bits first on ties
    if (__builtin_popcount(W) == nw) wsets.push_back(W);
    if (W == 0) break;
  }
  std::vector<TileStage> recs(acts.size());
  size_t s = 0;
  while (s < acts.size()) {
    uint32_t best = 0;
    size_t best_len = 0;
    for (uint32_t W : wsets) {
      size_t len = 0;
      while (s + len < acts.size() && fits(s + len, W)) ++len;
      if (len > best_len) {
        best_len = len;
        best = W;
      }
    }
    const bool run = best_len > 0;
    if (!run) best_len = 1;  // no choice covers the lanes' residues: the plain layout
    for (size_t k = 0; k < best_len; ++k) {
      TileStage& st = recs[s + k];
      std::vector<int> act = acts[s + k];
      const uint32_t W = run ? best : 0;
      uint32_t used = amask[s + k] | W;
      // pad the slots: bits whose residue keeps another free bit first, lowest first
      while (int(act.size()) < sb) {
        int pick = -1;
        for (int b = 0; b < m && pick < 0; ++b)
          if (!((used >> b) & 1) && __builtin_popcount(all & ~used & resmask(b % 4)) > 1) pick = b;
        for (int b = 0; b < m && pick < 0; ++b)
          if (!((used >> b) & 1)) pick = b;
        act.push_back(pick);
        used |= 1u << pick;
      }
      for (int q = 0; q < sb; ++q) st.slot_bit[q] = int8_t(act[q]);
      std::vector<int> order;
      for (int r = 0; r < nres; ++r)
        for (int b = r; b < m; b += 4)
          if (!((used >> b) & 1)) {
            order.push_back(b);
            used |= 1u << b;
            break;
          }
      for (int b = 0; b < m; ++b)
        if (!((used >> b) & 1)) order.push_back(b);
      for (int b = 0; b < m; ++b)
        if ((W >> b) & 1) order.push_back(b);
      for (size_t q = 0; q < order.size() && q < 16; ++q) st.lane_bit[q] = int8_t(order[q]);
      st.warp_local = int8_t(run && k + 1 < best_len ? 1 : 0);
    }
    s += best_len;
  }
  return recs;
}

// exactly the SWAP permutation (rows 0, 2, 1, 3 of the identity), no condition
bool is_exact_swap(const PlanOp& p) {
  if (p.phase || p.nt != 2 || p.cmask != 0 || p.grad >= 0) return false;
  for (int e = 0; e < 16; ++e) {
    const int r = e >> 2, c = e & 3;
    const int want_c = r == 1 ? 2 : r == 2 ? 1 : r;
    if (p.m[2 * e] != (c == want_c ? 1.0 : 0.0) || p.m[2 * e + 1] != 0.0) return false;
  }
  return true;
}

// an op with its global bits renamed: bit b -> ren[b]
PlanOp renamed(const PlanOp& p, const int* ren) {
  PlanOp q = p;
  for (int k = 0; k < p.nt && !p.phase; ++k) q.tb[k] = ren[p.tb[k]];
  auto map_mask = [&](uint64_t mk) {
    uint64_t o = 0;
    for (int b = 0; b < 64; ++b)
      if ((mk >> b) & 1) o |= uint64_t(1) << ren[b];
    return o;
  };
  q.cmask = map_mask(p.cmask);
  q.cval = map_mask(p.cval);
  q.touched = map_mask(p.touched);
  for (auto& be : q.beta) be.first = ren[be.first];
  return q;
}

template <typename R>
void emit_pass(const BuiltPass& bp0, const std::vector<PlanOp>& pops0, int n, int m, int L, int sb,
               HostPlan<R>& hp, bool swap_ops, bool phase1_ops, bool relabel_swaps, bool bfly_ops,
               bool real1_ops) {
  TilePass P{};
  P.m = m;
  P.L = L;
  for (int i = 0; i < m; ++i) P.bits[i] = int8_t(bp0.B[i]);
  for (int i = 0; i < 16; ++i) P.rbit[i] = int8_t(i);
  // The pass's ops, in order.  An exact SWAP of two tile bits moves no data: from there
  // on the data of either qubit sits where the other's was, so the pass's later ops are
  // renamed (ren[b]: where the data of global bit b sits in the tile as loaded), and the
  // write-out takes the amplitude for local index u (bit k of u = global bit B[k]) from
  // the tile position whose bit rbit[k] is bit k of u.
  std::vector<PlanOp> pops;
  BuiltPass bp;
  bp.B = bp0.B;
  {
    int ren[64], loc[64];
    for (int b = 0; b < 64; ++b) {
      ren[b] = b;
      loc[b] = -1;
    }
    for (int i = 0; i < m; ++i) loc[bp0.B[i]] = i;
    for (int idx : bp0.ops) {
      const PlanOp& p = pops0[idx];
      if (relabel_swaps && is_exact_swap(p) && loc[ren[p.tb[0]]] >= 0 && loc[ren[p.tb[1]]] >= 0) {
        std::swap(ren[p.tb[0]], ren[p.tb[1]]);
        P.permuted = 1;
        continue;
      }
      bp.ops.push_back(int(pops.size()));
      pops.push_back(renamed(p, ren));
    }
    if (P.permuted)
      for (int k = 0; k < m; ++k) P.rbit[k] = int8_t(loc[ren[bp0.B[k]]]);
  }
  P.ntiles = uint64_t(1) << (n - m);
  P.c0 = m / 2;
  P.c1 = m - P.c0;
  P.cg = (n - m + 2) / 3;
  if (P.cg < 1) P.cg = 1;
  P.stage0 = int(hp.stages.size());
  P.op0 = int(hp.ops.size());
  P.mat0 = int(hp.mats.size());
  while (hp.pool.size() % 2) hp.pool.push_back(R(0));
  P.pool0 = int(hp.pool.size());
  int local_of[64];
  for (int b = 0; b < 64; ++b) local_of[b] = -1;
  for (int i = 0; i < m; ++i) local_of[bp.B[i]] = i;
  // global bit of each tile-index bit (the bits outside B, ascending)
  int gbit_of_tb[64];
  {
    int k = 0;
    for (int b = 0; b < n; ++b)
      if (local_of[b] < 0) gbit_of_tb[k++] = b;
  }
  std::vector<std::vector<int>> takes, acts;
  split_stages(bp, pops, local_of, sb, takes, acts);
  // 4 residues: 8-byte elements, half-warp banks; 3: 16-byte elements
  const std::vector<TileStage> recs = stage_layouts(acts, m, sb, sizeof(R) == 4 ? 4 : 3);
  for (size_t si = 0; si < takes.size(); ++si) {
    const std::vector<int>& take = takes[si];
    TileStage st = recs[si];
    st.op0 = int(hp.ops.size()) - P.op0;
    const size_t j = take.size();
    // a CZ: the phase pi (or -pi: the same factor -1, e.g. a daggered CZ whose matrix
    // carries -0 imaginary parts) on b_t b_c keyed on its target t (no constant, no tag)
    auto is_cz = [&](const PlanOp& o) {
      return o.phase && o.grad < 0 && o.c == 0.0 && o.beta.size() == 1 &&
             (o.beta[0].second == M_PI || o.beta[0].second == -M_PI) && o.cmask == o.cval &&
             __builtin_popcountll(o.cmask) == 1;
    };
    // code of one end of a CZ pair in this stage: 0x80 | slot, a lane bit (< 16), or
    // 0x40 | global bit for a bit fixed by the tile number
    auto cz_end = [&](int gbit) -> uint32_t {
      const int lb = local_of[gbit];
      if (lb < 0) return 0x40u | uint32_t(gbit);
      for (int k = 0; k < sb; ++k)
        if (st.slot_bit[k] == lb) return 0x80u | uint32_t(k);
      return uint32_t(lb);
    };
    for (size_t q = 0; q < j; ++q) {
      const PlanOp& p = pops[take[q]];
      TileOp op{};
      op.lmask = op.lval = 0;
      op.gmask = op.gval = 0;
      op.grad = p.grad;
      op.gslot = -1;
      if (is_cz(p)) {
        // a run of CZs (they commute) becomes one sign op: the amplitude's sign is the
        // parity of sum over pairs b_t b_c; the pair codes go into the matrix block
        op.type = TOP_CZSET;
        op.jmask = 0xFFFFFFFFu;
        op.mat = int64_t(hp.mats.size()) - P.mat0;
        int np = 0;
        for (;;) {
          const PlanOp& c = pops[take[q]];
          const uint32_t code = cz_end(__builtin_ctzll(c.cmask)) | (cz_end(c.beta[0].first) << 8);
          R word{};
          memcpy(&word, &code, sizeof(code));  // a small bit pattern: never a NaN
          hp.mats.push_back(word);
          ++np;
          if (q + 1 >= j || !is_cz(pops[take[q + 1]])) break;
          ++q;
        }
        // keep the block's later matrices 16-byte aligned (they are read as 16-byte words)
        while ((hp.mats.size() - size_t(P.mat0)) * sizeof(R) % 16) hp.mats.push_back(R(0));
        op.s0 = np;
        hp.ops.push_back(op);
        continue;
      }
      if (p.grad >= 0) {
        op.gen = int8_t(p.gen);
        op.gslot = P.ngrad++;
        op.zglob = int8_t(p.touched ? __builtin_ctzll(p.touched) : 0);
        op.zloc = int8_t(local_of[op.zglob]);
      }
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
      {
        // split the in-tile condition: slot bits -> a table over the 2^sb slot
        // combinations (jmask), the rest stays a per-thread test on the lane bits
        uint32_t slotmask = 0;
        for (int k = 0; k < sb; ++k) slotmask |= 1u << st.slot_bit[k];
        const uint32_t ls = op.lmask & slotmask, lvs = op.lval & slotmask;
        op.jmask = 0;
        for (int jj = 0; jj < (1 << sb); ++jj) {
          uint32_t loc = 0;
          for (int k = 0; k < sb; ++k)
            if ((jj >> k) & 1) loc |= 1u << st.slot_bit[k];
          if ((loc & ls) == lvs) op.jmask |= 1u << jj;
        }
        op.lmask &= ~slotmask;
        op.lval &= ~slotmask;
      }
      // exactly the SWAP permutation (rows 0, 2, 1, 3 of the identity): a register
      // permutation in the stage, symmetric in its two slots
      bool is_swap = swap_ops && !p.phase && p.nt == 2;
      for (int e = 0; is_swap && e < 16; ++e) {
        const int r = e >> 2, c = e & 3;
        const int want_c = r == 1 ? 2 : r == 2 ? 1 : r;
        if (p.m[2 * e] != (c == want_c ? 1.0 : 0.0) || p.m[2 * e + 1] != 0.0) is_swap = false;
      }
      auto slot = [&](int gbit) {
        const int lb = local_of[gbit];
        for (int k = 0; k < sb; ++k)
          if (st.slot_bit[k] == lb) return k;
        return -1;
      };
      if (is_swap) {
        op.type = TOP_SWAP;
        op.s0 = std::min(slot(p.tb[0]), slot(p.tb[1]));
        op.s1 = std::max(slot(p.tb[0]), slot(p.tb[1]));
        op.mat = 0;
      } else if (bfly_ops && !p.phase && p.nt == 1 && p.m[1] == 0.0 && p.m[3] == 0.0 && p.m[5] == 0.0 &&
                 p.m[7] == 0.0 && p.m[2] == p.m[0] && p.m[4] == p.m[0] && p.m[6] == -p.m[0]) {
        // s [[1, 1], [1, -1]]: a butterfly
        op.type = TOP_BFLY;
        op.s0 = slot(p.tb[0]);
        op.s1 = 0;
        op.mat = int64_t(hp.mats.size()) - P.mat0;
        const R sv = R(p.m[0]);
        hp.mats.push_back(sv);
        hp.mats.push_back(sv);
        hp.mats.push_back(-sv);
        hp.mats.push_back(-sv);
      } else if (real1_ops && !p.phase && p.nt == 1 && p.m[1] == 0.0 && p.m[3] == 0.0 && p.m[5] == 0.0 &&
                 p.m[7] == 0.0) {
        // a real 2x2 matrix
        op.type = TOP_REAL1;
        op.s0 = slot(p.tb[0]);
        op.s1 = 0;
        op.mat = int64_t(hp.mats.size()) - P.mat0;
        for (int e = 0; e < 4; ++e) {
          hp.mats.push_back(R(p.m[2 * e]));
          if (sizeof(R) == 4) hp.mats.push_back(R(p.m[2 * e]));
        }
      } else if (!p.phase) {
        op.type = p.nt == 1 ? TOP_DENSE1 : TOP_DENSE2;
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
          // a recorded rotation starts its own op: its record must see the state
          // before it (a tagged op may absorb the untagged ones after it)
          if (!nx.phase || nx.cmask != p.cmask || nx.cval != p.cval || nx.grad >= 0) break;
          c += nx.c;
          for (auto& be : nx.beta) beta[be.first] += be.second;
          ++q;
        }
        int nbeta = 0, bbit = -1;
        for (int b = 0; b < 64; ++b)
          if (beta[b] != 0.0) {
            ++nbeta;
            bbit = b;
          }
        if (phase1_ops && nbeta <= 1) {
          // exp(i (c + beta b)) on at most one bit: the two factors e^{ic}, e^{i(c+beta)}
          // go into the matrix block; the bit is a register slot (s0), a lane bit (zloc)
          // or a bit fixed by the tile number (zglob)
          op.type = TOP_PHASE1;
          if (bbit < 0) bbit = 0;  // a constant phase: both factors equal
          op.mat = int64_t(hp.mats.size()) - P.mat0;
          const cd z0 = std::polar(1.0, c), z1 = std::polar(1.0, c + beta[bbit]);
          hp.mats.push_back(R(z0.real()));
          hp.mats.push_back(R(z0.imag()));
          hp.mats.push_back(R(z1.real()));
          hp.mats.push_back(R(z1.imag()));
          const int lb = local_of[bbit];
          op.s0 = -1;
          for (int k = 0; k < sb; ++k)
            if (lb >= 0 && st.slot_bit[k] == lb) op.s0 = k;
          if (p.grad < 0) {  // a recorded Z rotation already carries its own bit here
            op.zloc = int8_t(lb);
            op.zglob = int8_t(bbit);
          }
          if (c == 0.0 && nbeta == 1 && !((p.cmask >> bbit) & 1)) {
            // e^{ic} = 1: only the amplitudes whose bit reads 1 change (a further
            // condition on that bit: its slot combinations, its lane, or the tile number)
            if (op.s0 >= 0) {
              uint32_t keep = 0;
              for (int jj = 0; jj < (1 << sb); ++jj)
                if ((jj >> op.s0) & 1) keep |= 1u << jj;
              op.jmask &= keep;
            } else if (lb >= 0) {
              op.lmask |= 1u << lb;
              op.lval |= 1u << lb;
            } else {
              op.gmask |= uint64_t(1) << bbit;
              op.gval |= uint64_t(1) << bbit;
            }
          }
          hp.ops.push_back(op);
          continue;
        }
        // tables: [2^sb slot combos][2^c0 low local][2^c1 high local][3 x 2^cg tile index].
        // Entry x of a table over bits g_0..g_{k-1} is exp(i sum_{x_j = 1} beta_{g_j}),
        // built by doubling: entry x = entry(x without its top bit) * exp(i beta_top)
        // (one complex product per entry; k <= 8 products deep, ~1e-15 relative).
        auto table = [&](const std::vector<int>& gbits, double c0) {
          std::vector<cd> t(size_t(1) << gbits.size());
          t[0] = std::polar(1.0, c0);
          for (size_t k = 0; k < gbits.size(); ++k) {
            const cd f = std::polar(1.0, gbits[k] >= 0 ? beta[gbits[k]] : 0.0);
            const size_t h = size_t(1) << k;
            for (size_t x = 0; x < h; ++x) t[h + x] = t[x] * f;
          }
          return t;
        };
        while (hp.pool.size() % 2) hp.pool.push_back(R(0));
        op.tab = int64_t(hp.pool.size() / 2);
        auto push_all = [&](std::vector<R>& dst, const std::vector<cd>& t) {
          for (const cd& z : t) {
            dst.push_back(R(z.real()));
            dst.push_back(R(z.imag()));
          }
        };
        op.mat = int64_t(hp.mats.size()) - P.mat0;
        std::vector<int> gb;
        for (int k = 0; k < sb; ++k) gb.push_back(bp.B[st.slot_bit[k]]);
        push_all(hp.mats, table(gb, 0.0));
        // inactive local bits only (slot bits are zero in r0)
        gb.clear();
        for (int k = 0; k < P.c0; ++k) gb.push_back(bp.B[k]);
        push_all(hp.pool, table(gb, 0.0));
        gb.clear();
        for (int k = 0; k < P.c1; ++k) gb.push_back(bp.B[P.c0 + k]);
        push_all(hp.pool, table(gb, 0.0));
        for (int ch = 0; ch < 3; ++ch) {
          gb.clear();
          for (int k = 0; k < P.cg; ++k) {
            const int tb = ch * P.cg + k;
            gb.push_back(tb < n - m ? gbit_of_tb[tb] : -1);  // past the last tile bit: no bit
          }
          push_all(hp.pool, table(gb, ch == 0 ? c : 0.0));
        }
      }
      hp.ops.push_back(op);
    }
    st.nops = int(hp.ops.size()) - P.op0 - st.op0;
    hp.stages.push_back(st);
  }
  P.nstages = int(hp.stages.size()) - P.stage0;
  P.nops = int(hp.ops.size()) - P.op0;
  P.nmat = int(hp.mats.size()) - P.mat0;
  P.npool = int(hp.pool.size()) - P.pool0;
  hp.passes.push_back(P);
}

template void emit_pass<float>(const BuiltPass&, const std::vector<PlanOp>&, int, int, int, int, HostPlan<float>&,
                               bool, bool, bool, bool, bool);
template void emit_pass<double>(const BuiltPass&, const std::vector<PlanOp>&, int, int, int, int, HostPlan<double>&,
                                bool, bool, bool, bool, bool);

void encode_df_slots(HostPlan<double>& hp) {
  auto enc = [](double x) {
    const float h = float(x), l = float(x - double(h));  // x - h is exact in binary64
    uint32_t hb, lb;
    memcpy(&hb, &h, 4);
    memcpy(&lb, &l, 4);
    const uint64_t u = uint64_t(hb) | (uint64_t(lb) << 32);
    double d;
    memcpy(&d, &u, 8);
    return d;
  };
  std::vector<char> words(hp.mats.size(), 0);  // CZ code words: not numbers
  for (const TilePass& P : hp.passes)
    for (int i = 0; i < P.nops; ++i) {
      const TileOp& op = hp.ops[size_t(P.op0) + i];
      if (op.type == TOP_CZSET)
        for (int e = 0; e < op.s0; ++e) words[size_t(P.mat0) + size_t(op.mat) + e] = 1;
    }
  for (size_t i = 0; i < hp.mats.size(); ++i)
    if (!words[i]) hp.mats[i] = enc(hp.mats[i]);
  for (double& x : hp.pool) x = enc(x);
}

thread_local int g_last_pass_count = 0;  // also set by the fused adjoint sweep
thread_local int g_last_fused_path = 0;
thread_local int g_last_stage_count = 0;

// Register stage width SB (a thread holds 2^SB amplitudes) and block size of the tile
// pass per precision: blockDim = 2^(m - SB) <= NT with m = 13 (complex64) / 12.
template <typename R>
struct TileShape;
template <>
struct TileShape<float> {
  // 2^4 amplitudes per thread with 512 threads (108 registers, 16 warps per SM): the
  // QFT-32 passes 259 -> 240 ms against 2^5 with 256 threads (230 registers, 8 warps),
  // the Haar brickwork and the adjoint's forward passes unchanged
  static constexpr int SB = 4, NT = 512;
};
template <>
struct TileShape<double> {
  static constexpr int SB = 4, NT = 256;
};

template <typename R>
static qc_status run_tiles(qc_state* s, const std::vector<ResolvedOp>& rops, int m, bool drop_global_phase) {
  const int n = s->n;
  const int L = sizeof(R) == 4 ? 4 : 3;
  // complex128 states of 2^kDfMinQubits amplitudes or more: double-float passes
  const bool df = sizeof(R) == 8 && n >= kDfMinQubits;
  const int SB = df ? kDfTileSB : TileShape<R>::SB;
  std::vector<PlanOp> pops;
  to_plan_ops(rops, pops);
  if (drop_global_phase) drop_global_phases(pops);
  std::vector<BuiltPass> bps = build_passes(pops, n, m, L);
  HostPlan<R> hp;
  // complex128 applies an exact SWAP as a register permutation; in the complex64
  // kernel that dispatch costs more (register allocation of every gate body) than the
  // dense 4x4 it replaces
  for (const BuiltPass& bp : bps)
    emit_pass<R>(bp, pops, n, m, L, SB, hp, /*swap_ops=*/sizeof(R) == 8, /*phase1_ops=*/true, /*relabel_swaps=*/true,
                 /*bfly_ops=*/sizeof(R) == 8, /*real1_ops=*/sizeof(R) == 8);
  g_last_pass_count = int(hp.passes.size());
  g_last_fused_path = 1;
  g_last_stage_count = int(hp.stages.size());
  if constexpr (sizeof(R) == 8) {
    if (df) encode_df_slots(hp);
  }
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
  const size_t fixed_smem = 2 * sizeof(Cplx<R>) * (size_t(1) << m) +
                            (sizeof(uint64_t) + sizeof(uint32_t)) * (size_t(1) << (m - L)) +
                            sizeof(uint64_t) * kTileNumberTab;
  // a pass's phase tables go to shared memory where they fit beside the tiles (the
  // tiles' copies stream through L1 and would evict them there)
  size_t plan_max = 0;
  for (TilePass& P : hp.passes) {
    const size_t plan = P.nstages * sizeof(TileStage) + P.nops * sizeof(TileOp) + ((P.nmat + 3) & ~3) * sizeof(R);
    const size_t with_pool = plan + size_t(P.npool) * sizeof(R);
    P.spool = P.npool > 0 && fixed_smem + with_pool <= kTileSmemBudget ? 1 : 0;
    plan_max = std::max(plan_max, P.spool ? with_pool : plan);
  }
  const size_t smem = fixed_smem + plan_max;
  constexpr int NT = TileShape<R>::NT;
  bool extops = false;
  for (const TileOp& op : hp.ops)
    extops |= op.type == TOP_CZSET || op.type == TOP_PHASE1 || op.type == TOP_BFLY || op.type == TOP_REAL1;
  for (const TilePass& P : hp.passes) extops |= P.permuted != 0;
  constexpr int SBK = TileShape<R>::SB;
  auto kern = extops ? k_tile_pass<R, NT, SBK, true> : k_tile_pass<R, NT, SBK, false>;
  if constexpr (sizeof(R) == 8) {
    if (df) kern = tile_pass_df_kernel(extops);
  }
  if (qc_status st = check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)),
                                "tile pass shared memory"))
    return st;
  const uint64_t ntiles = uint64_t(1) << (n - m);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (per_sm < 1) per_sm = 1;
  const uint64_t cap = uint64_t(device_sm_count()) * per_sm;
  const unsigned grid = unsigned(ntiles < cap ? ntiles : cap);
  R* a = reinterpret_cast<R*>(s->amps);
  for (const TilePass& P : hp.passes) {
    QC_COUNT(), kern<<<grid, threads, smem, s->stream>>>(a, P, dst, dop, dpool, dmats);
  }
  return check_launch("tile pass");
}

qc_status launch_copy_pass(qc_state* s, const TilePass& P0) {
  TilePass P = P0;  // no stages, ops or tables: the tiles are copied through the relabeling
  P.stage0 = P.nstages = P.op0 = P.nops = P.mat0 = P.nmat = P.pool0 = P.npool = P.spool = 0;
  const int m = P.m, L = P.L;
  const size_t smem = 2 * sizeof(Cplx<float>) * (size_t(1) << m) +
                      (sizeof(uint64_t) + sizeof(uint32_t)) * (size_t(1) << (m - L)) +
                      sizeof(uint64_t) * kTileNumberTab;
  constexpr int NT = TileShape<float>::NT, SBK = TileShape<float>::SB;
  auto kern = k_tile_pass<float, NT, SBK, true>;
  if (qc_status st = check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)),
                                "copy pass shared memory"))
    return st;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
  if (per_sm < 1) per_sm = 1;
  const uint64_t cap = uint64_t(device_sm_count()) * per_sm;
  const unsigned grid = unsigned(P.ntiles < cap ? P.ntiles : cap);
  QC_COUNT(), kern<<<grid, NT, smem, s->stream>>>(reinterpret_cast<float*>(s->amps), P, nullptr, nullptr, nullptr,
                                                  nullptr);
  return check_launch("copy pass");
}

int tile_bits_for(const qc_state* s) {
  const int want = s->dtype == QC_C64 ? 13 : 12;
  return std::min(want, s->n);
}

void drop_global_phases(std::vector<PlanOp>& pops) {
  for (PlanOp& p : pops)
    if (p.phase && p.cmask == 0) p.c = 0.0;
}

// QC_PREC_AUTO: the choice between the CUDA-core tile passes (0) and the tensor-core
// stage passes (2) per (device name, n, circuit structure), made by timing both once on
// a scratch state; optionally appended to / read from the file QC_AUTOTUNE_CACHE.
static std::mutex g_auto_mu;
static std::map<std::string, int> g_auto_choice;

static std::string auto_key(const qc_state* s, const std::vector<ResolvedOp>& rops) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
  for (const ResolvedOp& r : rops) {
    mix(uint64_t(r.form));
    mix(uint64_t(r.nq));
    for (int k = 0; k < r.nq; ++k) mix(uint64_t(r.bits[k]));
    mix(uint64_t(r.cstate));
  }
  cudaDeviceProp prop;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  std::string key = std::string("fused|") + prop.name + "|" + std::to_string(s->n) + "|" + std::to_string(rops.size()) +
                    "|" + std::to_string(h);
  for (char& ch : key)
    if (ch == ' ') ch = '_';
  return key;
}

static qc_status time_path(qc_state* t, const std::vector<ResolvedOp>& rops, int path, bool drop_global_phase,
                           float* ms) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  qc_status st = QC_OK;
  bool ran = true;
  for (int rep = 0; rep < 2 && st == QC_OK && ran; ++rep) {  // the first run plans and uploads
    cudaEventRecord(e0, t->stream);
    if (path == 2) {
      st = run_tiles_tc(t, rops, &ran);  // ran = false: the circuit does not fit the stages
    } else {
      st = run_tiles<float>(t, rops, tile_bits_for(t), drop_global_phase);
    }
    cudaEventRecord(e1, t->stream);
    cudaEventSynchronize(e1);
    if (st == QC_OK && ran) cudaEventElapsedTime(ms, e0, e1);
  }
  if (!ran) *ms = 1e30f;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

static qc_status auto_choice(qc_state* s, const std::vector<ResolvedOp>& rops, bool drop_global_phase, int* choice) {
  const std::string key = auto_key(s, rops) + (drop_global_phase ? "|nophase" : "");
  std::lock_guard<std::mutex> lock(g_auto_mu);
  auto it = g_auto_choice.find(key);
  if (it != g_auto_choice.end()) {
    *choice = it->second;
    return QC_OK;
  }
  const char* path = getenv("QC_AUTOTUNE_CACHE");
  if (path) {
    if (FILE* f = fopen(path, "r")) {
      char k[512];
      int v;
      while (fscanf(f, "%511s %d", k, &v) == 2)
        if (key == k && (v == 0 || v == 2)) {
          fclose(f);
          g_auto_choice[key] = v;
          *choice = v;
          return QC_OK;
        }
      fclose(f);
    }
  }
  // a scratch state of the same size (timing does not depend on the amplitudes)
  qc_state t = *s;
  t.amps = nullptr;
  t.owned = false;
  t.scratch = nullptr;
  t.scratch_bytes = 0;
  t.host_buf = nullptr;
  if (cudaMalloc(&t.amps, state_len(s) * amp_bytes(s->dtype)) != cudaSuccess) {
    cudaGetLastError();
    *choice = 2;  // no room to time: the tensor-core passes
    return QC_OK;
  }
  qc_status st = qc_state_init_basis(&t, 0);
  float ms_cuda = 1e30f, ms_tc = 1e30f;
  if (st == QC_OK) st = time_path(&t, rops, 0, drop_global_phase, &ms_cuda);
  if (st == QC_OK) st = time_path(&t, rops, 2, drop_global_phase, &ms_tc);
  cudaStreamSynchronize(t.stream);
  cudaFree(t.amps);
  if (t.scratch) cudaFree(t.scratch);
  if (st != QC_OK) return st;
  *choice = ms_tc < ms_cuda ? 2 : 0;
  g_auto_choice[key] = *choice;
  if (path) {
    if (FILE* f = fopen(path, "a")) {
      fprintf(f, "%s %d\n", key.c_str(), *choice);
      fclose(f);
    }
  }
  return QC_OK;
}

qc_status run_fused(qc_state* s, const qc_circuit* c, const double* params, qc_prec prec, bool drop_global_phase) {
  std::vector<ResolvedOp> rops(c->nops);
  for (int i = 0; i < c->nops; ++i)
    if (qc_status st = resolve_op(c, c->ops[i], params, &rops[i])) return st;
  if (prec == QC_PREC_AUTO) {
    prec = QC_PREC_NATIVE;
    // (the tensor-core passes keep a global phase the CUDA-core passes may drop; the
    // callers that drop it accept either)
    if (s->dtype == QC_C64 && s->n >= 12) {
      int choice = 0;
      if (qc_status st = auto_choice(s, rops, drop_global_phase, &choice)) return st;
      if (choice == 2) prec = QC_PREC_TF32X3;
    }
  }
  if (prec == QC_PREC_TF32X3 && s->dtype == QC_C64) {
    bool handled = false;
    if (qc_status st = run_tiles_tc(s, rops, &handled)) return st;
    if (handled) return QC_OK;
  }
  const int m = tile_bits_for(s);
  if (s->n < 10 || m < kMaxStageBits + 4) {
    g_last_fused_path = 0;
    g_last_stage_count = 0;
    return run_per_gate(s, c, params);
  }
  return s->dtype == QC_C64 ? run_tiles<float>(s, rops, m, drop_global_phase)
                            : run_tiles<double>(s, rops, m, drop_global_phase);
}

template <typename R>
static void plan_stats(int n, const std::vector<ResolvedOp>& rops, int m, int* passes, int* stages, int* ops) {
  const int L = sizeof(R) == 4 ? 4 : 3;
  const int SB = sizeof(R) == 8 && n >= kDfMinQubits ? kDfTileSB : TileShape<R>::SB;
  std::vector<PlanOp> pops;
  to_plan_ops(rops, pops);
  std::vector<BuiltPass> bps = build_passes(pops, n, m, L);
  HostPlan<R> hp;
  for (const BuiltPass& bp : bps)
    emit_pass<R>(bp, pops, n, m, L, SB, hp, /*swap_ops=*/sizeof(R) == 8, /*phase1_ops=*/true, /*relabel_swaps=*/true,
                 /*bfly_ops=*/sizeof(R) == 8, /*real1_ops=*/sizeof(R) == 8);
  *passes = int(hp.passes.size());
  *stages = int(hp.stages.size());
  *ops = int(hp.ops.size());
}

}  // namespace qcgb

using namespace qcgb;

extern "C" int qc_last_pass_count(void) { return qcgb::g_last_pass_count; }
extern "C" int qc_last_fused_path(void) { return qcgb::g_last_fused_path; }
extern "C" int qc_last_stage_count(void) { return qcgb::g_last_stage_count; }

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

// ---------------------------------------------------------------------------
// host emulation of the CUDA-core tile passes (a check of the plan's logic)
// ---------------------------------------------------------------------------
namespace qcgb {

// One tile op of a CUDA-core plan on a thread's 2^SB amplitudes v (slot combination j at
// v[j]), interpreted in FP64 (conditions checked by the caller)
void emulate_tile_op(const TileOp& op, const double* mats, const TilePass& P, const std::complex<double>* cpool,
                     int m, uint64_t t, uint64_t base, uint32_t r0, std::vector<std::complex<double>>& v) {
  const uint32_t NA = uint32_t(v.size());
  const double* mm = mats + op.mat;
  auto pairs = [&](int s0, auto f) {
    for (uint32_t j = 0; j < NA; ++j)
      if (!((j >> s0) & 1) && ((op.jmask >> j) & 1u)) f(j, j | (1u << s0));
  };
  if (op.type == TOP_DENSE1) {
    const cd u00(mm[0], mm[1]), u01(mm[2], mm[3]), u10(mm[4], mm[5]), u11(mm[6], mm[7]);
    pairs(op.s0, [&](uint32_t j, uint32_t j1) {
      const cd x = v[j], y = v[j1];
      v[j] = u00 * x + u01 * y;
      v[j1] = u10 * x + u11 * y;
    });
  } else if (op.type == TOP_DENSE2) {
    const uint32_t b0 = 1u << op.s0, b1 = 1u << op.s1;
    for (uint32_t j = 0; j < NA; ++j) {
      if (j & (b0 | b1)) continue;
      const uint32_t ix[4] = {j, j | b1, j | b0, j | b0 | b1};
      cd x[4], o[4];
      for (int c = 0; c < 4; ++c) x[c] = v[ix[c]];
      for (int r = 0; r < 4; ++r) {
        o[r] = 0.0;
        for (int c = 0; c < 4; ++c) o[r] += cd(mm[8 * r + 2 * c], mm[8 * r + 2 * c + 1]) * x[c];
      }
      for (int r = 0; r < 4; ++r) v[ix[r]] = o[r];
    }
  } else if (op.type == TOP_SWAP) {
    const uint32_t b0 = 1u << op.s0, b1 = 1u << op.s1;
    for (uint32_t j = 0; j < NA; ++j)
      if (!(j & (b0 | b1))) std::swap(v[j | b0], v[j | b1]);
  } else if (op.type == TOP_CZSET) {
    // code words: per pair, bytes 0 and 1 = 0x80 | slot, a lane bit, or 0x40 | global bit
    for (uint32_t j = 0; j < NA; ++j) {
      int parity = 0;
      for (int e = 0; e < op.s0; ++e) {
        uint32_t code;
        memcpy(&code, mm + e, sizeof(code));
        int bit[2];
        for (int h = 0; h < 2; ++h) {
          const uint32_t c = (code >> (8 * h)) & 0xFFu;
          bit[h] = (c & 0x80u) ? int((j >> (c & 7u)) & 1u)
                               : (c & 0x40u) ? int((base >> (c & 63u)) & 1u) : int((r0 >> c) & 1u);
        }
        parity ^= bit[0] & bit[1];
      }
      if (parity) v[j] = -v[j];
    }
  } else if (op.type == TOP_BFLY) {
    const double sp = mm[0];
    pairs(op.s0, [&](uint32_t j, uint32_t j1) {
      const cd x0 = v[j], x1 = v[j1];
      v[j] = sp * x0 + sp * x1;
      v[j1] = sp * x0 - sp * x1;
    });
  } else if (op.type == TOP_REAL1) {
    const double ra = mm[0], rb = mm[1], rc = mm[2], rd = mm[3];
    pairs(op.s0, [&](uint32_t j, uint32_t j1) {
      const cd x0 = v[j], x1 = v[j1];
      v[j] = ra * x0 + rb * x1;
      v[j1] = rc * x0 + rd * x1;
    });
  } else if (op.type == TOP_PHASE1) {
    const cd z0(mm[0], mm[1]), z1(mm[2], mm[3]);
    const uint32_t fixed =
        op.s0 >= 0 ? 0u : op.zloc >= 0 ? (r0 >> op.zloc) & 1u : uint32_t((base >> op.zglob) & 1u);
    for (uint32_t j = 0; j < NA; ++j) {
      if (!((op.jmask >> j) & 1u)) continue;
      const uint32_t b = op.s0 >= 0 ? (j >> op.s0) & 1u : fixed;
      v[j] *= b ? z1 : z0;
    }
  } else {  // TOP_PHASE: tile-number chunks, the thread's two local chunks, slot table
    const cd* l0 = cpool + op.tab;
    const cd* l1 = l0 + (1 << P.c0);
    const cd* g0 = l1 + (1 << (m - P.c0));
    const uint64_t gn = uint64_t(1) << P.cg, gm = gn - 1;
    const cd w = g0[t & gm] * g0[gn + ((t >> P.cg) & gm)] * g0[2 * gn + ((t >> (2 * P.cg)) & gm)] *
                 l0[r0 & ((1u << P.c0) - 1)] * l1[r0 >> P.c0];
    for (uint32_t j = 0; j < NA; ++j)
      if ((op.jmask >> j) & 1u) v[j] *= w * cd(mm[2 * j], mm[2 * j + 1]);
  }
}

// `state` (2^n complex128) through the plan QC_RUN_FUSED builds for a state of `dtype` --
// its passes, register stages, tile ops with their conditions, matrices, phase tables,
// CZ code words and relabeled SWAPs -- in FP64 and in the kernel's order (the complex64
// plan's structure with the complex128 plan's value format)
static void emulate_tile_plan(int n, const std::vector<ResolvedOp>& rops, qc_dtype dtype, cd* a) {
  const bool c64 = dtype == QC_C64;
  const int m = std::min(c64 ? 13 : 12, n);
  const int L = c64 ? 4 : 3;
  const int SB = c64 ? TileShape<float>::SB : (n >= kDfMinQubits ? kDfTileSB : TileShape<double>::SB);
  std::vector<PlanOp> pops;
  to_plan_ops(rops, pops);
  const std::vector<BuiltPass> bps = build_passes(pops, n, m, L);
  HostPlan<double> hp;
  for (const BuiltPass& bp : bps)
    emit_pass<double>(bp, pops, n, m, L, SB, hp, /*swap_ops=*/!c64, /*phase1_ops=*/true, /*relabel_swaps=*/true,
                      /*bfly_ops=*/!c64, /*real1_ops=*/!c64);
  const uint32_t T = 1u << m, NA = 1u << SB;
  const uint64_t ntiles = uint64_t(1) << (n - m);
  std::vector<cd> tile(T), out(T);
  const cd* cpool = reinterpret_cast<const cd*>(hp.pool.data());
  for (const TilePass& P : hp.passes) {
    bool in[64] = {false};
    for (int k = 0; k < m; ++k) in[P.bits[k]] = true;
    std::vector<int> tnb;  // bit i of a tile number sits at global bit tnb[i]
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
      for (uint32_t u = 0; u < T; ++u) tile[u] = a[addr(u)];
      for (int s = 0; s < P.nstages; ++s) {
        const TileStage& st = hp.stages[size_t(P.stage0 + s)];
        for (uint32_t th = 0; th < (1u << (m - SB)); ++th) {
          uint32_t r0 = 0;
          for (int k = 0; k < m - SB; ++k) r0 |= ((th >> k) & 1u) << st.lane_bit[k];
          std::vector<uint32_t> pos(NA);
          std::vector<cd> v(NA);
          for (uint32_t j = 0; j < NA; ++j) {
            uint32_t u = r0;
            for (int k = 0; k < SB; ++k)
              if ((j >> k) & 1) u |= 1u << st.slot_bit[k];
            pos[j] = u;
            v[j] = tile[u];
          }
          for (int q = 0; q < st.nops; ++q) {
            const TileOp& op = hp.ops[size_t(P.op0 + st.op0 + q)];
            if ((base & op.gmask) != op.gval) continue;
            if ((r0 & op.lmask) != op.lval) continue;
            emulate_tile_op(op, mats, P, cpool, m, t, base, r0, v);
          }
          for (uint32_t j = 0; j < NA; ++j) tile[pos[j]] = v[j];
        }
      }
      // write-out through the relabeling: output u from the position whose bit rbit[k]
      // is bit k of u
      for (uint32_t u = 0; u < T; ++u) {
        uint32_t src = 0;
        for (int k = 0; k < m; ++k) src |= ((u >> k) & 1u) << P.rbit[k];
        out[u] = tile[src];
      }
      for (uint32_t u = 0; u < T; ++u) a[addr(u)] = out[u];
    }
  }
}

}  // namespace qcgb

extern "C" qc_status qc_tile_emulate(const qc_circuit* c, const double* params, qc_dtype dtype, double* state) {
  clear_error();
  if (!c || !state || c->n < 10 || c->n > 24 || (c->nops > 0 && !c->ops) || (dtype != QC_C64 && dtype != QC_C128)) {
    set_error("qc_tile_emulate: invalid arguments (10 <= n <= 24)");
    return QC_ERR_INVALID_ARG;
  }
  std::vector<ResolvedOp> rops(size_t(c->nops));
  for (int i = 0; i < c->nops; ++i)
    if (qc_status st = resolve_op(c, c->ops[i], params, &rops[size_t(i)])) return st;
  emulate_tile_plan(c->n, rops, dtype, reinterpret_cast<std::complex<double>*>(state));
  return QC_OK;
}
