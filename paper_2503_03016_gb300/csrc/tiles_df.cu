// Complex128 tile passes in double-float arithmetic (the circuit passes of planner.cu
// for complex128 states of at least 2^kDfMinQubits amplitudes).
//
// The same passes, stages and ops as k_tile_pass<double>; what changes is the
// arithmetic.  A tile arrives from HBM as binary64 (the same cp.async copies), is split
// in place in shared memory into double-float amplitudes -- 16 bytes each, laid out
// (re_hi, im_hi, re_lo, im_lo) -- and every stage computes on those with the packed
// FP32 operations and error-free transformations of dfloat.cuh; the write-out joins
// them back to binary64.  The plan's matrices and phase tables arrive as double-float
// slots as well: 8 bytes per value, binary32 hi in the low half and lo in the high half
// (the host splits them; CZ code words stay as they are).
//
// A complex product u x is the two packed terms (u.re, u.re) * (x.re, x.im) and
// (-u.im, u.im) * (x.im, x.re) of an output pair, as in the double-float sweeps.
#include "common.cuh"
#include "dfloat.cuh"
#include "kernels.cuh"
#include "tiles.cuh"
#include "tiles_df.cuh"

namespace qcgb {

// ---------------------------------------------------------------------------
// the pass (shared-memory layout, tiles, stages and ops as in k_tile_pass)
// ---------------------------------------------------------------------------
template <int NT, int SB, bool EXTOPS>
__global__ void __launch_bounds__(NT, 1) k_tile_pass_df(double* __restrict__ amps, const TilePass P,
                                                        const TileStage* __restrict__ stages,
                                                        const TileOp* __restrict__ ops, const double* __restrict__ pool,
                                                        const double* __restrict__ mats) {
  constexpr int NA = 1 << SB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = P.m, L = P.L;
  const uint32_t T = 1u << m;
  Cplx<double>* bufs = reinterpret_cast<Cplx<double>*>(smem_raw);  // 2 x T, binary64 then double-float
  uint64_t* hioff = reinterpret_cast<uint64_t*>(smem_raw + 2 * sizeof(Cplx<double>) * T);
  const int nhi = m - L;
  uint32_t* rhi = reinterpret_cast<uint32_t*>(hioff + (1u << nhi));
  uint64_t* tnt = reinterpret_cast<uint64_t*>(rhi + (1u << nhi));
  TileStage* sst = reinterpret_cast<TileStage*>(tnt + kTileNumberTab);
  TileOp* sop = reinterpret_cast<TileOp*>(sst + P.nstages);
  double* smat = reinterpret_cast<double*>(sop + P.nops);
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
  __syncthreads();
  const uint32_t lowmask = (1u << L) - 1;
  const double* dpool = pool;
  uint64_t t = blockIdx.x;
  if (t < P.ntiles) prefetch_tile<double>(bufs, amps, tile_base(t, tnt), hioff, L, T);
  cp_async_commit();
  for (int it = 0; t < P.ntiles; t += gridDim.x, ++it) {
    Cplx<double>* dtile = bufs + (it & 1) * T;
    float4* tile = reinterpret_cast<float4*>(dtile);
    const uint64_t base = tile_base(t, tnt);
    const uint64_t tn = t + gridDim.x;
    if (tn < P.ntiles) prefetch_tile<double>(bufs + ((it + 1) & 1) * T, amps, tile_base(tn, tnt), hioff, L, T);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    // binary64 -> double-float, in place (each thread its own positions)
    for (uint32_t p = threadIdx.x; p < T; p += blockDim.x) {
      const Cplx<double> d = dtile[p];
      float rh, rl, ih, il;
      df_split(d.re, rh, rl);
      df_split(d.im, ih, il);
      tile[p] = make_float4(rh, ih, rl, il);
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
      DFC v[NA];
#pragma unroll
      for (int j = 0; j < NA; ++j) v[j] = dfc_ld(tile, p0 ^ slot_xor<SB>(j, sw));
      for (int q = 0; q < st.nops; ++q) {
        const TileOp op = sop[st.op0 + q];
        if ((base & op.gmask) != op.gval) continue;
        if ((r0 & op.lmask) != op.lval) continue;
        const double* mm = smat + op.mat;
        if (op.type == TOP_DENSE1) {
          df_apply_dense1<SB>(op.s0, v, mm, op.jmask);
        } else if (op.type == TOP_DENSE2) {
          df_apply_dense2<SB>(op.s0, op.s1, v, mm);
        } else if (op.type == TOP_SWAP) {
          df_apply_swap<SB>(op.s0, op.s1, v);
        } else if (EXTOPS && op.type == TOP_CZSET) {
          const uint32_t flip = czset_flips<double, SB>(mm, op.s0, r0, base);
#pragma unroll
          for (int j = 0; j < NA; ++j)
            if ((flip >> j) & 1u) {
              v[j].hi = make_float2(-v[j].hi.x, -v[j].hi.y);
              v[j].lo = make_float2(-v[j].lo.x, -v[j].lo.y);
            }
        } else if (EXTOPS && op.type == TOP_BFLY) {
          df_apply_bfly<SB>(op.s0, v, mm, op.jmask);
        } else if (EXTOPS && op.type == TOP_REAL1) {
          df_apply_real1<SB>(op.s0, v, mm, op.jmask);
        } else if (EXTOPS && op.type == TOP_PHASE1) {
          const uint32_t fixed =
              op.s0 >= 0 ? 0u : op.zloc >= 0 ? (r0 >> op.zloc) & 1u : uint32_t((base >> op.zglob) & 1u);
          df_apply_phase1<SB>(v, mm, op.s0, fixed, op.jmask);
        } else {
          // exp(i (c + sum beta_p b_p)) from the tables (complex slots): tile-index
          // chunks (3), the thread's inactive local bits (2 chunks), slot combinations
          const double* l0 = dpool + 2 * op.tab;
          const double* l1 = l0 + 2 * (1 << P.c0);
          const double* g0 = l1 + 2 * (1 << (m - P.c0));
          const uint32_t gn = 1u << P.cg, gm = gn - 1;
          DFC w = dfc_mul(dfc_slots(g0 + 2 * (t & gm)), dfc_slots(g0 + 2 * (gn + ((t >> P.cg) & gm))));
          w = dfc_mul(dfc_slots(g0 + 2 * (2 * gn + ((t >> (2 * P.cg)) & gm))), w);
          w = dfc_mul(dfc_slots(l0 + 2 * (r0 & ((1u << P.c0) - 1))), w);
          w = dfc_mul(dfc_slots(l1 + 2 * (r0 >> P.c0)), w);
          const DFPair pw = df_pairs(w);
#pragma unroll
          for (int j = 0; j < NA; ++j) {
            if (!((op.jmask >> j) & 1u)) continue;
            DF2Acc a;
            dfc_first(a, pw, dfc_slots(mm + 2 * j));
            const DFC z = dfc_res(a);
            v[j] = dfc_mul(z, v[j]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < NA; ++j) dfc_st(tile, p0 ^ slot_xor<SB>(j, sw), v[j]);
      if (st.warp_local)
        __syncwarp();
      else
        __syncthreads();
    }
    // double-float -> binary64 on the way out
    for (uint32_t e = threadIdx.x; e < T / 2; e += blockDim.x) {
      const uint32_t u = 2 * e;
      const uint64_t gi = base | hioff[u >> L] | (u & lowmask);
      uint32_t pa, pb;
      if constexpr (EXTOPS) {
        const uint32_t hi = rhi[u >> L];
        pa = tile_swz(hi | rlo[u & lowmask]);
        pb = tile_swz(hi | rlo[(u | 1u) & lowmask]);
      } else {
        pa = tile_swz(u);
        pb = pa ^ 1u;
      }
      const float4 a = tile[pa], b = tile[pb];
      st_amp2<double>(amps, gi, Cplx<double>{df_join(a.x, a.z), df_join(a.y, a.w)},
                      Cplx<double>{df_join(b.x, b.z), df_join(b.y, b.w)});
    }
    __syncthreads();
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

TilePassFn tile_pass_df_kernel(bool extops) {
  constexpr int NT = kDfTileNT, SB = kDfTileSB;
  return extops ? k_tile_pass_df<NT, SB, true> : k_tile_pass_df<NT, SB, false>;
}

}  // namespace qcgb
