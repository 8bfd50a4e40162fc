// Shared-memory tile passes: the device plan records, the device helpers that apply a
// pass's gates to a register stage, and the host planner's interface.  Used by the
// circuit passes (planner.cu) and the fused adjoint sweep (adjoint_tiles.cu).
#pragma once

#include <complex>
#include <utility>
#include <vector>

#include "circuit.cuh"
#include "common.cuh"

namespace qcgb {

constexpr int kMaxStageBits = 5;  // amplitudes a thread holds per stage: 2^SB, SB <= 5

enum TileOpType : int32_t {
  TOP_DENSE1 = 0, TOP_DENSE2 = 1, TOP_PHASE = 2, TOP_SWAP = 3, TOP_CZSET = 4, TOP_PHASE1 = 5,
  TOP_BFLY = 6,  // s [[1, 1], [1, -1]] (a Hadamard): a butterfly, no general 2x2 product
  TOP_REAL1 = 7  // a real 2x2 matrix (a Y rotation, X): real coefficients on complex amplitudes
};

struct TileOp {
  int8_t type;
  int8_t gen;            // adjoint sweep: generator of the recorded rotation (0 X, 1 Y, 2 Z)
  int8_t zloc, zglob;    // Z rotation: local bit of its qubit (-1: outside the tile), global bit
  int32_t s0, s1;        // stage slots of the targets (DENSE2: s0 = first qubit = row MSB)
  uint32_t lmask, lval;  // condition on the thread's non-slot local (in-tile) index bits
  uint32_t jmask;        // bit j: slot combination j meets the condition on the slot bits
  uint64_t gmask, gval;  // condition on the index bits outside the tile
  int64_t mat;           // DENSE: matrix / PHASE: 2^SB-entry slot table, offset (R values)
                         // in the pass's matrix block
  int64_t tab;           // PHASE: offset (complex entries) of its other tables in the pool
  int32_t grad;          // adjoint sweep: rotation whose gradient is recorded before the op, or -1
  int32_t gslot;         // ... its slot among the pass's recorded rotations
};
static_assert(sizeof(TileOp) == 64, "TileOp must be 64 bytes");

struct TileStage {
  int32_t op0, nops;
  int8_t slot_bit[7];   // local bit of each slot (SB used)
  int8_t warp_local;    // 1: the next stage gives every warp the same amplitudes (the same
                        // local bits receive thread-index bits 5 and up), so a warp
                        // barrier ends this stage; 0: a block barrier
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
  int32_t pool0, npool; // the pass's other phase tables (R values in the pool; pool0 even);
                        // tensor-core passes: the pass's deferred phase factors (global
                        // indices [pool0, pool0 + npool))
  int32_t spool;        // 1: the kernel stages those tables in shared memory
  int8_t bits[16];   // B ascending (global bit positions); bits[0..L) = 0..L-1
  int32_t c0, c1;    // local phase-table chunks: local bits [0,c0) and [c0,m)
  int32_t cg;        // tile-index phase-table chunk width (3 chunks)
  uint64_t ntiles;
  int32_t ngrad;     // adjoint sweep: rotations recorded in this pass
  int32_t permuted;  // exact SWAPs taken as relabelings: the data of global bit bits[k]
  int8_t rbit[16];   // sits at local bit rbit[k] when the pass writes the tile back
};

// ---------------------------------------------------------------------------
// device side
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t tile_swz(uint32_t r) {
  uint32_t x = r >> 4;
  return r ^ ((x ^ (x >> 4) ^ (x >> 8)) & 15u);
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

// jmask bit j: the pair (j, j | 2^S0) meets the gate's condition (controls in the slots)
template <typename R, int SB, int S0>
__device__ __forceinline__ void dense1(Cplx<R> (&v)[1 << SB], const R* __restrict__ u, uint32_t jmask) {
  if constexpr (sizeof(R) == 4) {
    float2 a[4], b[4];
    load_packed<4>(a, b, u);
#pragma unroll
    for (int j = 0; j < (1 << SB); ++j) {
      if (j & (1 << S0)) continue;
      const int j1 = j | (1 << S0);
      if (!((jmask >> j) & 1u)) continue;
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
      if (!((jmask >> j) & 1u)) continue;
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
__device__ __forceinline__ void apply_dense1(int s0, Cplx<R> (&v)[1 << SB], const R* u, uint32_t jmask) {
  // slots s0 >= SB do not exist for this stage width (the planner never emits them)
  switch (s0) {
    case 0: dense1<R, SB, 0>(v, u, jmask); break;
    case 1: dense1<R, SB, 1>(v, u, jmask); break;
    case 2: dense1<R, SB, 2>(v, u, jmask); break;
    case 3:
      if constexpr (SB > 3) dense1<R, SB, 3>(v, u, jmask);
      break;
    default:
      if constexpr (SB > 4) dense1<R, SB, 4>(v, u, jmask);
      break;
  }
}

#define QC_D2(A, B) \
  case (A) * 8 + (B): dense2<R, SB, A, B>(v, u); return;
template <typename R, int SB>
__device__ __forceinline__ void apply_dense2(int s0, int s1, Cplx<R> (&v)[1 << SB], const R* u) {
  switch (s0 * 8 + s1) {
    // the planner orders every two-qubit gate so that s0 < s1
    QC_D2(0, 1) QC_D2(0, 2) QC_D2(1, 2)
    default: break;
  }
  if constexpr (SB > 3) {
    switch (s0 * 8 + s1) {
      QC_D2(0, 3) QC_D2(1, 3) QC_D2(2, 3)
      default: break;
    }
  }
  if constexpr (SB > 4) {
    switch (s0 * 8 + s1) {
      QC_D2(0, 4) QC_D2(1, 4) QC_D2(2, 4) QC_D2(3, 4)
      default: break;
    }
  }
}
#undef QC_D2

// SWAP of slots S0 < S1: a permutation of the thread's registers, no arithmetic
template <typename R, int SB, int S0, int S1>
__device__ __forceinline__ void swap2(Cplx<R> (&v)[1 << SB]) {
#pragma unroll
  for (int j = 0; j < (1 << SB); ++j) {
    if (j & ((1 << S0) | (1 << S1))) continue;
    const Cplx<R> t = v[j | (1 << S0)];
    v[j | (1 << S0)] = v[j | (1 << S1)];
    v[j | (1 << S1)] = t;
  }
}

#define QC_SW(A, B) \
  case (A) * 8 + (B): swap2<R, SB, A, B>(v); return;
template <typename R, int SB>
__device__ __forceinline__ void apply_swap(int s0, int s1, Cplx<R> (&v)[1 << SB]) {
  switch (s0 * 8 + s1) {
    QC_SW(0, 1) QC_SW(0, 2) QC_SW(1, 2)
    default: break;
  }
  if constexpr (SB > 3) {
    switch (s0 * 8 + s1) {
      QC_SW(0, 3) QC_SW(1, 3) QC_SW(2, 3)
      default: break;
    }
  }
  if constexpr (SB > 4) {
    switch (s0 * 8 + s1) {
      QC_SW(0, 4) QC_SW(1, 4) QC_SW(2, 4) QC_SW(3, 4)
      default: break;
    }
  }
}
#undef QC_SW

// TOP_PHASE1: multiply by z0 or z1 as the op's bit reads 0 or 1 -- the bit is register
// slot ks (>= 0), or fixed for the thread (`fixed`)
// complex64: the slot is a template argument (KS; -1: the bit is fixed), so that each
// slot combination's factor is known at compile time instead of being selected per
// amplitude; complex128 keeps the selecting form (its FP64 passes are bound elsewhere,
// and the switch costs them registers)
template <typename R, int SB, int KS>
__device__ __forceinline__ void phase1_k(Cplx<R> (&v)[1 << SB], Cplx<R> z0, Cplx<R> z1, uint32_t jmask) {
#pragma unroll
  for (int j = 0; j < (1 << SB); ++j) {
    if (!((jmask >> j) & 1u)) continue;
    v[j] = cmul(v[j], (KS >= 0 && ((j >> KS) & 1)) ? z1 : z0);
  }
}

template <typename R, int SB>
__device__ __forceinline__ void apply_phase1(Cplx<R> (&v)[1 << SB], const R* zs, int ks, uint32_t fixed,
                                             uint32_t jmask) {
  const Cplx<R> z0{zs[0], zs[1]}, z1{zs[2], zs[3]};
  if constexpr (sizeof(R) == 4) {
    switch (ks) {
      case 0: phase1_k<R, SB, 0>(v, z0, z1, jmask); return;
      case 1: phase1_k<R, SB, 1>(v, z0, z1, jmask); return;
      case 2:
        if constexpr (SB > 2) phase1_k<R, SB, 2>(v, z0, z1, jmask);
        return;
      case 3:
        if constexpr (SB > 3) phase1_k<R, SB, 3>(v, z0, z1, jmask);
        return;
      case 4:
        if constexpr (SB > 4) phase1_k<R, SB, 4>(v, z0, z1, jmask);
        return;
      default:
        phase1_k<R, SB, -1>(v, fixed ? z1 : z0, z1, jmask);
        return;
    }
  } else {
    const Cplx<R> zf = fixed ? z1 : z0;
#pragma unroll
    for (int j = 0; j < (1 << SB); ++j) {
      if (!((jmask >> j) & 1u)) continue;
      const Cplx<R> z = ks >= 0 ? (((j >> ks) & 1) ? z1 : z0) : zf;
      v[j] = cmul(v[j], z);
    }
  }
}

// TOP_BFLY on slot S0: (x0, x1) -> (s x0 + s x1, s x0 - s x1), t = s x0 formed once;
// three FMA-pipe operations per pair (complex64: on packed pairs) instead of the eight
// products and sums of a general 2x2.  ss = (s, s, -s, -s) in the matrix block.
template <typename R, int SB, int S0>
__device__ __forceinline__ void bfly(Cplx<R> (&v)[1 << SB], const R* __restrict__ ss, uint32_t jmask) {
#pragma unroll
  for (int j = 0; j < (1 << SB); ++j) {
    if (j & (1 << S0)) continue;
    if (!((jmask >> j) & 1u)) continue;
    const int j1 = j | (1 << S0);
    if constexpr (sizeof(R) == 4) {
      const float2 sp = make_float2(ss[0], ss[1]), sn = make_float2(ss[2], ss[3]);
      const float2 t = __fmul2_rn(f2(v[j]), sp), x1 = f2(v[j1]);
      v[j] = c2(__ffma2_rn(x1, sp, t));
      v[j1] = c2(__ffma2_rn(x1, sn, t));
    } else {
      const R sp = ss[0];
      const R tr = v[j].re * sp, ti = v[j].im * sp;
      const Cplx<R> x1 = v[j1];
      v[j] = Cplx<R>{fma(x1.re, sp, tr), fma(x1.im, sp, ti)};
      v[j1] = Cplx<R>{fma(x1.re, -sp, tr), fma(x1.im, -sp, ti)};
    }
  }
}

template <typename R, int SB>
__device__ __forceinline__ void apply_bfly(int s0, Cplx<R> (&v)[1 << SB], const R* ss, uint32_t jmask) {
  switch (s0) {
    case 0: bfly<R, SB, 0>(v, ss, jmask); return;
    case 1: bfly<R, SB, 1>(v, ss, jmask); return;
    case 2: bfly<R, SB, 2>(v, ss, jmask); return;
    default: break;
  }
  if constexpr (SB > 3)
    if (s0 == 3) bfly<R, SB, 3>(v, ss, jmask);
  if constexpr (SB > 4)
    if (s0 == 4) bfly<R, SB, 4>(v, ss, jmask);
}

// TOP_REAL1 on slot S0: a real 2x2 matrix [[a, b], [c, d]]: each output is two real
// multiply-adds per component (complex64: two packed operations, no swapped copies)
// instead of two complex products.  rm = (a, a, b, b, c, c, d, d) for complex64,
// (a, b, c, d) for complex128, in the matrix block.
template <typename R, int SB, int S0>
__device__ __forceinline__ void real1(Cplx<R> (&v)[1 << SB], const R* __restrict__ rm, uint32_t jmask) {
  if constexpr (sizeof(R) == 4) {
    const float4 ab = *reinterpret_cast<const float4*>(rm), cd = *reinterpret_cast<const float4*>(rm + 4);
    const float2 a = make_float2(ab.x, ab.y), b = make_float2(ab.z, ab.w);
    const float2 c = make_float2(cd.x, cd.y), d = make_float2(cd.z, cd.w);
#pragma unroll
    for (int j = 0; j < (1 << SB); ++j) {
      if (j & (1 << S0)) continue;
      if (!((jmask >> j) & 1u)) continue;
      const int j1 = j | (1 << S0);
      const float2 x0 = f2(v[j]), x1 = f2(v[j1]);
      v[j] = c2(__ffma2_rn(x1, b, __fmul2_rn(x0, a)));
      v[j1] = c2(__ffma2_rn(x1, d, __fmul2_rn(x0, c)));
    }
  } else {
    const R a = rm[0], b = rm[1], c = rm[2], d = rm[3];
#pragma unroll
    for (int j = 0; j < (1 << SB); ++j) {
      if (j & (1 << S0)) continue;
      if (!((jmask >> j) & 1u)) continue;
      const int j1 = j | (1 << S0);
      const Cplx<R> x0 = v[j], x1 = v[j1];
      v[j] = Cplx<R>{fma(x1.re, b, x0.re * a), fma(x1.im, b, x0.im * a)};
      v[j1] = Cplx<R>{fma(x1.re, d, x0.re * c), fma(x1.im, d, x0.im * c)};
    }
  }
}

template <typename R, int SB>
__device__ __forceinline__ void apply_real1(int s0, Cplx<R> (&v)[1 << SB], const R* rm, uint32_t jmask) {
  switch (s0) {
    case 0: real1<R, SB, 0>(v, rm, jmask); return;
    case 1: real1<R, SB, 1>(v, rm, jmask); return;
    case 2: real1<R, SB, 2>(v, rm, jmask); return;
    default: break;
  }
  if constexpr (SB > 3)
    if (s0 == 3) real1<R, SB, 3>(v, rm, jmask);
  if constexpr (SB > 4)
    if (s0 == 4) real1<R, SB, 4>(v, rm, jmask);
}

// Slot combinations j (of 2^SB) whose bit k is set, as a 32-bit mask.
__device__ __forceinline__ uint32_t slot_set_mask(uint32_t k) {
  switch (k) {
    case 0: return 0xAAAAAAAAu;
    case 1: return 0xCCCCCCCCu;
    case 2: return 0xF0F0F0F0u;
    case 3: return 0xFF00FF00u;
    default: return 0xFFFF0000u;
  }
}

// A set of CZ gates as one sign op: bit j of the result is the parity of
// sum over pairs (a, b) of b_a b_b for slot combination j of this thread.  Each pair is a
// 32-bit code word (stored in the matrix block, one R slot per pair): byte 0 end a,
// byte 1 end b, each 0x80 | slot, a lane bit (< 16) or 0x40 | global bit.
// (kept out of line: inlined, it changes the register allocation of the gate bodies)
template <typename R, int SB>
__device__ __noinline__ uint32_t czset_flips(const R* words, int npairs, uint32_t r0, uint64_t base) {
  uint32_t flip = 0, fixed = 0;
  for (int e = 0; e < npairs; ++e) {
    uint32_t code;
    memcpy(&code, words + e, sizeof(code));
    uint32_t m[2], f[2];
    bool slot[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t c = (code >> (8 * h)) & 0xFFu;
      slot[h] = (c & 0x80u) != 0;
      m[h] = slot[h] ? slot_set_mask(c & 7u) : 0u;
      f[h] = slot[h] ? 0u : (c & 0x40u) ? uint32_t(base >> (c & 63u)) & 1u : (r0 >> c) & 1u;
    }
    if (slot[0] && slot[1])
      flip ^= m[0] & m[1];
    else if (slot[0])
      flip ^= f[1] ? m[0] : 0u;
    else if (slot[1])
      flip ^= f[0] ? m[1] : 0u;
    else
      fixed ^= f[0] & f[1];
  }
  return fixed ? ~flip : flip;
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
  const R* src = amps + 2 * base;  // the tile's bits and base's bits are disjoint
  for (uint32_t r = threadIdx.x; r < T; r += blockDim.x)
    cp_async_amp<R>(buf + tile_swz(r), src + 2 * (hioff[r >> L] | (r & lowmask)));
}

// Tile number t -> its index bits outside the tile (t's bits deposited, in order, on
// the global bits not in the tile), by three lookups in tables of 256 entries that
// cover the tile number 8 bits at a time (at most 24 tile-number bits).
constexpr int kTileNumberTab = 3 * 256;
__device__ __forceinline__ void build_tile_number_tables(uint64_t* tab, const int8_t* sbits, int m, int nt_bits) {
  for (int e = threadIdx.x; e < kTileNumberTab; e += blockDim.x) {
    const int c = e >> 8, v = e & 255;
    uint64_t o = 0;
    int idx = 0, j = 0;  // tile-number bit counter; next tile bit (sbits ascending)
    for (int b = 0; b < 64 && idx < nt_bits && idx < 8 * c + 8; ++b) {
      if (j < m && sbits[j] == b) {
        ++j;
        continue;
      }
      if (idx >= 8 * c && ((v >> (idx - 8 * c)) & 1)) o |= uint64_t(1) << b;
      ++idx;
    }
    tab[e] = o;
  }
}
__device__ __forceinline__ uint64_t tile_base(uint64_t t, const uint64_t* tab) {
  return tab[t & 255] | tab[256 + ((t >> 8) & 255)] | tab[512 + ((t >> 16) & 255)];
}

// ---------------------------------------------------------------------------
// host planner interface (planner.cu)
// ---------------------------------------------------------------------------
struct PlanOp {
  // dense: 1 or 2 target bits, matrix, control mask/values (global bits)
  // phase: condition mask/values (global), constant angle and per-bit coefficients
  // grad/gen: adjoint sweep only -- the rotation (and its generator) whose gradient
  // Im <lambda|G|psi> is recorded just before this op is applied
  bool phase;
  int nt;
  int tb[2];
  double m[32];
  uint64_t cmask, cval;
  double c;
  std::vector<std::pair<int, double>> beta;  // (bit, coefficient)
  uint64_t touched;                          // every bit the op reads or writes
  int grad = -1, gen = -1;
};

constexpr int kMaxPassOps = 128;  // bounds the plan staged in shared memory per pass
// shared memory a tile pass may use (tiles, tables and the staged plan) on sm_103a
constexpr size_t kTileSmemBudget = 220 * 1024;

struct BuiltPass {
  std::vector<int> B;       // ascending
  std::vector<int> ops;     // indices into plan ops, in order
};

// Device plan assembled on the host.
template <typename R>
struct HostPlan {
  std::vector<TilePass> passes;
  std::vector<TileStage> stages;
  std::vector<TileOp> ops;
  std::vector<R> pool;  // phase tables read per thread (global memory)
  std::vector<R> mats;  // per-pass matrices and slot tables (staged in shared memory)
};

// the complex128 circuit pass in double-float arithmetic (tiles_df.cu): the same
// launch signature as k_tile_pass<double>; its matrices and tables are double-float
// slots (encode_df_slots)
using TilePassFn = void (*)(double*, const TilePass, const TileStage*, const TileOp*, const double*, const double*);
TilePassFn tile_pass_df_kernel(bool extops);
// its register stages: 2^3 amplitudes per thread, 512 threads (16 warps per SM: the
// double-float gate bodies are latency-bound at 8)
constexpr int kDfTileSB = 3, kDfTileNT = 512;
// a plan's numeric matrix entries and phase tables -> double-float slots in place (8 bytes
// per value: binary32 hi in the low half, lo = the rest rounded, in the high half); the
// CZ code words are left as they are
void encode_df_slots(HostPlan<double>& hp);

// tile passes of the most recent fused circuit run or fused adjoint reverse sweep
extern thread_local int g_last_pass_count;
// how the most recent QC_RUN_FUSED circuit ran: 0 per gate, 1 CUDA-core tile passes,
// 2 tile passes with tensor-core stages
extern thread_local int g_last_fused_path;
// register stages (or tensor-core stage blocks) of the most recent fused circuit run
extern thread_local int g_last_stage_count;

// resolved gates -> plan ops (diagonal gates become phase ops); with `grad`/`gen`, op i
// carries the tag grad[i] (>= 0: a rotation exp(-i t G/2) with generator gen[i]; X and Y
// rotations stay dense, Z rotations become phase ops)
void to_plan_ops(const std::vector<ResolvedOp>& in, std::vector<PlanOp>& out, const std::vector<int>* grad = nullptr,
                 const std::vector<int>* gen = nullptr);
// a complex64 pass with no stages whose SWAPs are a relabeling (P.permuted, P.rbit; P.bits
// ascending): each tile copied through the permutation by the CUDA-core tile pass
qc_status launch_copy_pass(qc_state* s, const TilePass& P);
// host emulation: one tile op of a CUDA-core plan (complex128 value format) on a thread's
// 2^SB amplitudes v, in FP64 (the op's conditions checked by the caller); mats: the
// pass's matrix block, cpool: the plan's phase tables as complex values
void emulate_tile_op(const TileOp& op, const double* mats, const TilePass& P, const std::complex<double>* cpool,
                     int m, uint64_t t, uint64_t base, uint32_t r0, std::vector<std::complex<double>>& v);
// exactly the SWAP permutation of its two target bits, with no condition
bool is_exact_swap(const PlanOp& p);
// an op with its global bits renamed: bit b -> ren[b]
PlanOp renamed(const PlanOp& p, const int* ren);
// sets the constant of every unconditioned phase op to 0 (a global phase)
void drop_global_phases(std::vector<PlanOp>& pops);
// plan ops -> passes of tile bit sets B (m bits, the L lowest always included); with
// cond_in_tile every condition bit of an op (a control, a phase op's condition) is a
// tile bit of the pass that takes it, as the tensor-core stages need
std::vector<BuiltPass> build_passes(const std::vector<PlanOp>& ops, int n, int m, int L, bool cond_in_tile = false);
// one pass -> its register stages, tile ops and matrices (sb: stage width); with
// swap_ops, an exact SWAP becomes a register permutation (TOP_SWAP) instead of a dense
// 4x4 (kernels that hold two states per thread keep the dense form: fewer registers);
// with phase1_ops, a phase op on at most one bit becomes TOP_PHASE1 (two factors, no
// per-thread table lookups)
// with relabel_swaps, an exact SWAP of two tile bits applies no arithmetic: the pass's
// later ops name the exchanged bits and the write-out reads the tile accordingly; with
// bfly_ops, a 1-qubit matrix s [[1, 1], [1, -1]] becomes TOP_BFLY (kernels that know it;
// the circuit passes use it for complex128, where FP64 arithmetic bounds the pass)
// with real1_ops, a real 1-qubit matrix becomes TOP_REAL1 (kernels that know it)
template <typename R>
void emit_pass(const BuiltPass& bp, const std::vector<PlanOp>& pops, int n, int m, int L, int sb,
               HostPlan<R>& hp, bool swap_ops = true, bool phase1_ops = true, bool relabel_swaps = false,
               bool bfly_ops = false, bool real1_ops = false);
// a pass's ops -> register stages (local_of: local bit of each global bit, -1 outside
// the tile); takes[s] = the ops of stage s, acts[s] = the local bits their targets use
// (whole_ops 1: control and phase bits in the tile count as active bits too; 2: as 1,
// except the phase bits of a phase op conditioned on at most one bit)
void split_stages(const BuiltPass& bp, const std::vector<PlanOp>& pops, const int* local_of, int sb,
                  std::vector<std::vector<int>>& takes, std::vector<std::vector<int>>& acts, int whole_ops = 0);
// as split_stages, each stage chosen among the same candidates by the fewest stages for
// the pass when the next `depth` stages are searched and the rest cut greedily; cuts are
// kept by the pass's structure and reused (matrices and angles do not enter them)
void split_stages_lookahead(const BuiltPass& bp, const std::vector<PlanOp>& pops, const int* local_of, int sb,
                            std::vector<std::vector<int>>& takes, std::vector<std::vector<int>>& acts, int whole_ops,
                            int depth);
// slot bits (acts[s] padded to sb) and thread-index bits of each stage (m - sb of them,
// the first ones one per residue mod nres); warp bits kept over runs of stages
std::vector<TileStage> stage_layouts(const std::vector<std::vector<int>>& acts, int m, int sb, int nres);

}  // namespace qcgb
