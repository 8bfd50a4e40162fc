// Double-float gate bodies on register stages of complex128 amplitudes (the tile passes
// of tiles_df.cu and the adjoint reverse passes of adjoint_tiles.cu).
//
// A stage amplitude is a complex double-float value: hi = (re_hi, im_hi), lo = (re_lo,
// im_lo).  A complex product u x is the two packed terms (u.re, u.re) * (x.re, x.im) and
// (-u.im, u.im) * (x.im, x.re) of an output pair, as in the double-float sweeps; matrix
// entries and phase factors come from double-float slots (8 bytes per value: binary32
// hi in the low half, lo in the high half).
#pragma once

#include "common.cuh"
#include "dfloat.cuh"
#include "tiles.cuh"

namespace qcgb {

// a complex double-float value: hi = (re_hi, im_hi), lo = (re_lo, im_lo)
struct DFC {
  float2 hi, lo;
};

// a complex value from two double-float slots (re, im)
__device__ __forceinline__ DFC dfc_slots(const double* s) {
  const float4 t = *reinterpret_cast<const float4*>(s);  // re_hi, re_lo, im_hi, im_lo
  return DFC{make_float2(t.x, t.z), make_float2(t.y, t.w)};
}
// a binary64 complex value split into a double-float one
__device__ __forceinline__ DFC dfc_of(const Cplx<double>& z) {
  float rh, rl, ih, il;
  df_split(z.re, rh, rl);
  df_split(z.im, ih, il);
  return DFC{make_float2(rh, ih), make_float2(rl, il)};
}
// a real value from one slot: (hi, lo)
__device__ __forceinline__ float2 dfr_slot(const double* s) { return *reinterpret_cast<const float2*>(s); }

__device__ __forceinline__ DFC dfc_ld(const float4* tile, uint32_t p) {
  const float4 t = tile[p];
  return DFC{make_float2(t.x, t.y), make_float2(t.z, t.w)};
}
__device__ __forceinline__ void dfc_st(float4* tile, uint32_t p, const DFC& v) {
  tile[p] = make_float4(v.hi.x, v.hi.y, v.lo.x, v.lo.y);
}

// the lane pairs of a complex coefficient u: (u.re, u.re) and (-u.im, u.im), each as
// hi, -hi, lo
struct DFPair {
  float2 h1, n1, l1, h2, n2, l2;
};
__device__ __forceinline__ DFPair df_pairs(const DFC& u) {
  DFPair p;
  p.h1 = make_float2(u.hi.x, u.hi.x);
  p.n1 = make_float2(-u.hi.x, -u.hi.x);
  p.l1 = make_float2(u.lo.x, u.lo.x);
  p.h2 = make_float2(-u.hi.y, u.hi.y);
  p.n2 = make_float2(u.hi.y, -u.hi.y);
  p.l2 = make_float2(-u.lo.y, u.lo.y);
  return p;
}
__device__ __forceinline__ DF2 dfc_x(const DFC& x) { return DF2{x.hi, x.lo}; }
__device__ __forceinline__ DF2 dfc_sw(const DFC& x) {
  return DF2{make_float2(x.hi.y, x.hi.x), make_float2(x.lo.y, x.lo.x)};
}

__device__ __forceinline__ void dfc_first(DF2Acc& a, const DFPair& u, const DFC& x) {
  df2_first(a, u.h1, u.n1, u.l1, dfc_x(x));
  df2_mac(a, u.h2, u.n2, u.l2, dfc_sw(x));
}
__device__ __forceinline__ void dfc_mac(DF2Acc& a, const DFPair& u, const DFC& x) {
  df2_mac(a, u.h1, u.n1, u.l1, dfc_x(x));
  df2_mac(a, u.h2, u.n2, u.l2, dfc_sw(x));
}
// a real coefficient r = (hi, lo) on both lanes
__device__ __forceinline__ void dfr_first(DF2Acc& a, float2 r, const DFC& x) {
  df2_first(a, make_float2(r.x, r.x), make_float2(-r.x, -r.x), make_float2(r.y, r.y), dfc_x(x));
}
__device__ __forceinline__ void dfr_mac(DF2Acc& a, float2 r, const DFC& x) {
  df2_mac(a, make_float2(r.x, r.x), make_float2(-r.x, -r.x), make_float2(r.y, r.y), dfc_x(x));
}
__device__ __forceinline__ DFC dfc_res(const DF2Acc& a) {
  const DF2 r = df2_result(a);
  return DFC{r.hi, r.lo};
}
__device__ __forceinline__ DFC dfc_mul(const DFC& u, const DFC& x) {
  DF2Acc a;
  dfc_first(a, df_pairs(u), x);
  return dfc_res(a);
}

// ---------------------------------------------------------------------------
// gate bodies on a register stage of 2^SB double-float amplitudes
// ---------------------------------------------------------------------------
template <int SB, int S0>
__device__ __forceinline__ void dfdense1(DFC (&v)[1 << SB], const double* u, uint32_t jmask) {
  const DFPair p00 = df_pairs(dfc_slots(u)), p01 = df_pairs(dfc_slots(u + 2));
  const DFPair p10 = df_pairs(dfc_slots(u + 4)), p11 = df_pairs(dfc_slots(u + 6));
#pragma unroll
  for (int j = 0; j < (1 << SB); ++j) {
    if (j & (1 << S0)) continue;
    if (!((jmask >> j) & 1u)) continue;
    const int j1 = j | (1 << S0);
    const DFC x = v[j], y = v[j1];
    DF2Acc a0, a1;
    dfc_first(a0, p00, x);
    dfc_first(a1, p10, x);
    dfc_mac(a0, p01, y);
    dfc_mac(a1, p11, y);
    v[j] = dfc_res(a0);
    v[j1] = dfc_res(a1);
  }
}

template <int SB, int S0, int S1>
__device__ __forceinline__ void dfdense2(DFC (&v)[1 << SB], const double* u) {
#pragma unroll
  for (int j = 0; j < (1 << SB); ++j) {
    if (j & ((1 << S0) | (1 << S1))) continue;
    const int i[4] = {j, j | (1 << S1), j | (1 << S0), j | (1 << S0) | (1 << S1)};
    const DFC x[4] = {v[i[0]], v[i[1]], v[i[2]], v[i[3]]};
#pragma unroll
    for (int r = 0; r < 4; r += 2) {
      // two output rows side by side (independent chains)
      DF2Acc a0, a1;
      dfc_first(a0, df_pairs(dfc_slots(u + 8 * r)), x[0]);
      dfc_first(a1, df_pairs(dfc_slots(u + 8 * r + 8)), x[0]);
#pragma unroll
      for (int c = 1; c < 4; ++c) {
        dfc_mac(a0, df_pairs(dfc_slots(u + 8 * r + 2 * c)), x[c]);
        dfc_mac(a1, df_pairs(dfc_slots(u + 8 * r + 8 + 2 * c)), x[c]);
      }
      v[i[r]] = dfc_res(a0);
      v[i[r + 1]] = dfc_res(a1);
    }
  }
}

// s [[1, 1], [1, -1]]: ss = (s, s, -s, -s) as slots
template <int SB, int S0>
__device__ __forceinline__ void dfbfly(DFC (&v)[1 << SB], const double* ss, uint32_t jmask) {
  const float2 s = dfr_slot(ss), ns = dfr_slot(ss + 2);
#pragma unroll
  for (int j = 0; j < (1 << SB); ++j) {
    if (j & (1 << S0)) continue;
    if (!((jmask >> j) & 1u)) continue;
    const int j1 = j | (1 << S0);
    const DFC x0 = v[j], x1 = v[j1];
    DF2Acc a0, a1;
    dfr_first(a0, s, x0);
    dfr_first(a1, s, x0);
    dfr_mac(a0, s, x1);
    dfr_mac(a1, ns, x1);
    v[j] = dfc_res(a0);
    v[j1] = dfc_res(a1);
  }
}

// a real 2x2 [[a, b], [c, d]] as slots (a, b, c, d)
template <int SB, int S0>
__device__ __forceinline__ void dfreal1(DFC (&v)[1 << SB], const double* rm, uint32_t jmask) {
  const float2 a = dfr_slot(rm), b = dfr_slot(rm + 1), c = dfr_slot(rm + 2), d = dfr_slot(rm + 3);
#pragma unroll
  for (int j = 0; j < (1 << SB); ++j) {
    if (j & (1 << S0)) continue;
    if (!((jmask >> j) & 1u)) continue;
    const int j1 = j | (1 << S0);
    const DFC x0 = v[j], x1 = v[j1];
    DF2Acc a0, a1;
    dfr_first(a0, a, x0);
    dfr_first(a1, c, x0);
    dfr_mac(a0, b, x1);
    dfr_mac(a1, d, x1);
    v[j] = dfc_res(a0);
    v[j1] = dfc_res(a1);
  }
}

// factor z1 where slot KS reads 1 and z0 elsewhere (KS = -1: z0 everywhere)
template <int SB, int KS>
__device__ __forceinline__ void dfphase1_k(DFC (&v)[1 << SB], const DFC& z0, const DFC& z1, uint32_t jmask) {
  const DFPair p0 = df_pairs(z0);
  DFPair p1;
  if (KS >= 0) p1 = df_pairs(z1);
#pragma unroll
  for (int j = 0; j < (1 << SB); ++j) {
    if (!((jmask >> j) & 1u)) continue;
    DF2Acc a;
    dfc_first(a, (KS >= 0 && ((j >> KS) & 1)) ? p1 : p0, v[j]);
    v[j] = dfc_res(a);
  }
}

// SWAP of slots S0 < S1: a permutation of the registers
template <int SB, int S0, int S1>
__device__ __forceinline__ void dfswap2(DFC (&v)[1 << SB]) {
#pragma unroll
  for (int j = 0; j < (1 << SB); ++j) {
    if (j & ((1 << S0) | (1 << S1))) continue;
    const DFC t = v[j | (1 << S0)];
    v[j | (1 << S0)] = v[j | (1 << S1)];
    v[j | (1 << S1)] = t;
  }
}

// dispatch on the slots (the planner emits only the slots a stage has)
#define QC_DF_SLOT_FN(NAME, FN)                                                                   \
  template <int SB>                                                                             \
  __device__ __forceinline__ void NAME(int s0, DFC (&v)[1 << SB], const double* u, uint32_t jmask) { \
    switch (s0) {                                                                               \
      case 0: FN<SB, 0>(v, u, jmask); return;                                                   \
      case 1: FN<SB, 1>(v, u, jmask); return;                                                   \
      case 2: FN<SB, 2>(v, u, jmask); return;                                                   \
      default:                                                                                  \
        if constexpr (SB > 3) FN<SB, 3>(v, u, jmask);                                           \
        return;                                                                                 \
    }                                                                                           \
  }
QC_DF_SLOT_FN(df_apply_dense1, dfdense1)
QC_DF_SLOT_FN(df_apply_bfly, dfbfly)
QC_DF_SLOT_FN(df_apply_real1, dfreal1)
#undef QC_DF_SLOT_FN

template <int SB>
__device__ __forceinline__ void df_apply_dense2(int s0, int s1, DFC (&v)[1 << SB], const double* u) {
  switch (s0 * 8 + s1) {
    case 0 * 8 + 1: dfdense2<SB, 0, 1>(v, u); return;
    case 0 * 8 + 2: dfdense2<SB, 0, 2>(v, u); return;
    case 1 * 8 + 2: dfdense2<SB, 1, 2>(v, u); return;
    default: break;
  }
  if constexpr (SB > 3) {
    switch (s0 * 8 + s1) {
      case 0 * 8 + 3: dfdense2<SB, 0, 3>(v, u); return;
      case 1 * 8 + 3: dfdense2<SB, 1, 3>(v, u); return;
      case 2 * 8 + 3: dfdense2<SB, 2, 3>(v, u); return;
      default: break;
    }
  }
}

template <int SB>
__device__ __forceinline__ void df_apply_swap(int s0, int s1, DFC (&v)[1 << SB]) {
  switch (s0 * 8 + s1) {
    case 0 * 8 + 1: dfswap2<SB, 0, 1>(v); return;
    case 0 * 8 + 2: dfswap2<SB, 0, 2>(v); return;
    case 1 * 8 + 2: dfswap2<SB, 1, 2>(v); return;
    default: break;
  }
  if constexpr (SB > 3) {
    switch (s0 * 8 + s1) {
      case 0 * 8 + 3: dfswap2<SB, 0, 3>(v); return;
      case 1 * 8 + 3: dfswap2<SB, 1, 3>(v); return;
      case 2 * 8 + 3: dfswap2<SB, 2, 3>(v); return;
      default: break;
    }
  }
}

template <int SB>
__device__ __forceinline__ void df_apply_phase1(DFC (&v)[1 << SB], const double* zs, int ks, uint32_t fixed,
                                                uint32_t jmask) {
  const DFC z0 = dfc_slots(zs), z1 = dfc_slots(zs + 2);
  switch (ks) {
    case 0: dfphase1_k<SB, 0>(v, z0, z1, jmask); return;
    case 1: dfphase1_k<SB, 1>(v, z0, z1, jmask); return;
    case 2: dfphase1_k<SB, 2>(v, z0, z1, jmask); return;
    case 3:
      if constexpr (SB > 3) dfphase1_k<SB, 3>(v, z0, z1, jmask);
      return;
    default: dfphase1_k<SB, -1>(v, fixed ? z1 : z0, z1, jmask); return;
  }
}

}  // namespace qcgb
