// Complex128 per-gate sweeps in double-float arithmetic (Sec. 3.2's sparse product
// (I_l (x) U' (x) I_r) psi, the same index groups as the FP64 sweeps of runtime.cu).
//
// Every amplitude is read as binary64, split into FP32 pairs, multiplied by the gate's
// entries (each held as hi + lo pairs) with error-free products and sums, and joined
// back to binary64 (dfloat.cuh).  The packed FP32 lanes hold the real and imaginary
// parts of one output: for an entry u and an input x,
//     (out.re, out.im) += (u.re, u.re) * (x.re, x.im) + (-u.im, u.im) * (x.im, x.re),
// so each entry is stored as the two lane pairs (u.re, u.re) and (-u.im, u.im), and
// each input in both orders.  Relative error per gate: a few units of 2^-48.
#include <cstring>

#include "common.cuh"
#include "dfloat.cuh"
#include "kernels.cuh"

namespace qcgb {

// one complex entry: lane pairs (u.re, u.re) and (-u.im, u.im), each as hi, -hi, lo
struct DFCoef {
  float2 h1, n1, l1;
  float2 h2, n2, l2;
};
struct DFMat2 {
  DFCoef e[4];
};
struct DFMat4 {
  DFCoef e[16];
};

// an input amplitude in both lane orders
struct DFAmp {
  DF2 x, s;
};

__device__ __forceinline__ DFAmp df_amp(Cplx<double> z) {
  float rh, rl, ih, il;
  df_split(z.re, rh, rl);
  df_split(z.im, ih, il);
  return DFAmp{DF2{make_float2(rh, ih), make_float2(rl, il)}, DF2{make_float2(ih, rh), make_float2(il, rl)}};
}

__device__ __forceinline__ Cplx<double> df_out(const DF2& r) {
  return Cplx<double>{df_join(r.hi.x, r.lo.x), df_join(r.hi.y, r.lo.y)};
}

__device__ __forceinline__ void df_cfirst(DF2Acc& a, const DFCoef& u, const DFAmp& x) {
  df2_first(a, u.h1, u.n1, u.l1, x.x);
  df2_mac(a, u.h2, u.n2, u.l2, x.s);
}
__device__ __forceinline__ void df_cmac(DF2Acc& a, const DFCoef& u, const DFAmp& x) {
  df2_mac(a, u.h1, u.n1, u.l1, x.x);
  df2_mac(a, u.h2, u.n2, u.l2, x.s);
}

// u x
__device__ __forceinline__ Cplx<double> df_mul1(const DFCoef& u, const DFAmp& x) {
  DF2Acc a;
  df_cfirst(a, u, x);
  return df_out(df2_result(a));
}
// u0 x0 + u1 x1
__device__ __forceinline__ Cplx<double> df_row2(const DFCoef& u0, const DFAmp& x0, const DFCoef& u1,
                                                const DFAmp& x1) {
  DF2Acc a;
  df_cfirst(a, u0, x0);
  df_cmac(a, u1, x1);
  return df_out(df2_result(a));
}
// sum_c u[c] x[c], c = 0..3
__device__ __forceinline__ Cplx<double> df_row4(const DFCoef* u, const DFAmp* x) {
  DF2Acc a;
  df_cfirst(a, u[0], x[0]);
#pragma unroll
  for (int c = 1; c < 4; ++c) df_cmac(a, u[c], x[c]);
  return df_out(df2_result(a));
}

// ---------------------------------------------------------------------------
// kernels (index groups as in the FP64 sweeps)
// ---------------------------------------------------------------------------
template <bool VEC>
__global__ void __launch_bounds__(256) k_1q_dense_df(double* __restrict__ a, SweepSpec sp, DFMat2 u) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t it = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; it < sp.items; it += stride) {
    uint64_t i0 = insert_zero_bits(it, sp.pos, sp.cnt);
    if (VEC) i0 <<= 1;
    i0 |= sp.set_mask;
    const uint64_t i1 = i0 | sp.t0;
    if (VEC) {
      Cplx<double> x0, x1, y0, y1;
      ld_amp2<double>(a, i0, x0, x1);
      ld_amp2<double>(a, i1, y0, y1);
      const DFAmp X0 = df_amp(x0), X1 = df_amp(x1), Y0 = df_amp(y0), Y1 = df_amp(y1);
      st_amp2<double>(a, i0, df_row2(u.e[0], X0, u.e[1], Y0), df_row2(u.e[0], X1, u.e[1], Y1));
      st_amp2<double>(a, i1, df_row2(u.e[2], X0, u.e[3], Y0), df_row2(u.e[2], X1, u.e[3], Y1));
    } else {
      const DFAmp X = df_amp(ld_amp<double>(a, i0)), Y = df_amp(ld_amp<double>(a, i1));
      st_amp<double>(a, i0, df_row2(u.e[0], X, u.e[1], Y));
      st_amp<double>(a, i1, df_row2(u.e[2], X, u.e[3], Y));
    }
  }
}

// target bit 0: each pair is the neighbour pair (i, i + 1)
__global__ void __launch_bounds__(256) k_1q_dense_low_df(double* __restrict__ a, SweepSpec sp, DFMat2 u) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t it = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; it < sp.items; it += stride) {
    const uint64_t i0 = insert_zero_bits(it, sp.pos, sp.cnt) | sp.set_mask;
    Cplx<double> x, y;
    ld_amp2<double>(a, i0, x, y);
    const DFAmp X = df_amp(x), Y = df_amp(y);
    st_amp2<double>(a, i0, df_row2(u.e[0], X, u.e[1], Y), df_row2(u.e[2], X, u.e[3], Y));
  }
}

// diag(d0, d1); ONLY1: d0 = 1 and only the members with the target bit set are touched
template <bool VEC, bool ONLY1>
__global__ void __launch_bounds__(256) k_1q_diag_df(double* __restrict__ a, SweepSpec sp, DFCoef d0, DFCoef d1) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t it = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; it < sp.items; it += stride) {
    uint64_t i0 = insert_zero_bits(it, sp.pos, sp.cnt);
    if (VEC) i0 <<= 1;
    i0 |= sp.set_mask;
    if (ONLY1) {
      if (VEC) {
        Cplx<double> x0, x1;
        ld_amp2<double>(a, i0, x0, x1);
        st_amp2<double>(a, i0, df_mul1(d1, df_amp(x0)), df_mul1(d1, df_amp(x1)));
      } else {
        st_amp<double>(a, i0, df_mul1(d1, df_amp(ld_amp<double>(a, i0))));
      }
    } else {
      const uint64_t i1 = i0 | sp.t0;
      if (VEC) {
        Cplx<double> x0, x1, y0, y1;
        ld_amp2<double>(a, i0, x0, x1);
        ld_amp2<double>(a, i1, y0, y1);
        st_amp2<double>(a, i0, df_mul1(d0, df_amp(x0)), df_mul1(d0, df_amp(x1)));
        st_amp2<double>(a, i1, df_mul1(d1, df_amp(y0)), df_mul1(d1, df_amp(y1)));
      } else {
        st_amp<double>(a, i0, df_mul1(d0, df_amp(ld_amp<double>(a, i0))));
        st_amp<double>(a, i1, df_mul1(d1, df_amp(ld_amp<double>(a, i1))));
      }
    }
  }
}

// [[0, b], [c, 0]]: out0 = b in1, out1 = c in0
template <bool VEC>
__global__ void __launch_bounds__(256) k_1q_anti_df(double* __restrict__ a, SweepSpec sp, DFCoef b, DFCoef c) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t it = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; it < sp.items; it += stride) {
    uint64_t i0 = insert_zero_bits(it, sp.pos, sp.cnt);
    if (VEC) i0 <<= 1;
    i0 |= sp.set_mask;
    const uint64_t i1 = i0 | sp.t0;
    if (VEC) {
      Cplx<double> x0, x1, y0, y1;
      ld_amp2<double>(a, i0, x0, x1);
      ld_amp2<double>(a, i1, y0, y1);
      st_amp2<double>(a, i0, df_mul1(b, df_amp(y0)), df_mul1(b, df_amp(y1)));
      st_amp2<double>(a, i1, df_mul1(c, df_amp(x0)), df_mul1(c, df_amp(x1)));
    } else {
      const DFAmp X = df_amp(ld_amp<double>(a, i0)), Y = df_amp(ld_amp<double>(a, i1));
      st_amp<double>(a, i0, df_mul1(b, Y));
      st_amp<double>(a, i1, df_mul1(c, X));
    }
  }
}

// dense 4x4 on quads; member r = 2 b_qa + b_qb; t0 = mask of qa, t1 = mask of qb.
// Four blocks per SM (at most 64 registers): the kernel is bound by the FP32 pipe and
// instruction issue, and the extra warps raise both utilisations (2.24 -> 2.12 ms at 28
// qubits).
template <bool VEC>
__global__ void __launch_bounds__(256, 4) k_2q_dense_df(double* __restrict__ a, SweepSpec sp, DFMat4 u) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t it = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; it < sp.items; it += stride) {
    uint64_t b = insert_zero_bits(it, sp.pos, sp.cnt);
    if (VEC) b <<= 1;
    b |= sp.set_mask;
    const uint64_t idx[4] = {b, b | sp.t1, b | sp.t0, b | sp.t0 | sp.t1};
    if (VEC) {
      Cplx<double> x[4], y[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) ld_amp2<double>(a, idx[r], x[r], y[r]);
      DFAmp X[4], Y[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        X[r] = df_amp(x[r]);
        Y[r] = df_amp(y[r]);
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) st_amp2<double>(a, idx[r], df_row4(&u.e[4 * r], X), df_row4(&u.e[4 * r], Y));
    } else {
      DFAmp X[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) X[r] = df_amp(ld_amp<double>(a, idx[r]));
#pragma unroll
      for (int r = 0; r < 4; ++r) st_amp<double>(a, idx[r], df_row4(&u.e[4 * r], X));
    }
  }
}

// dense 4x4 with bit 0 among the targets: neighbour pairs (b, b|1) and (b|m, b|m|1)
__global__ void __launch_bounds__(256, 4) k_2q_dense_low_df(double* __restrict__ a, SweepSpec sp, DFMat4 u,
                                                         bool qa_low) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  const uint64_t mo = qa_low ? sp.t1 : sp.t0;
  for (uint64_t it = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; it < sp.items; it += stride) {
    const uint64_t b = insert_zero_bits(it, sp.pos, sp.cnt);
    Cplx<double> p0, p1, q0, q1;
    ld_amp2<double>(a, b, p0, p1);
    ld_amp2<double>(a, b | mo, q0, q1);
    DFAmp X[4];
    if (qa_low) {
      X[0] = df_amp(p0); X[2] = df_amp(p1); X[1] = df_amp(q0); X[3] = df_amp(q1);
    } else {
      X[0] = df_amp(p0); X[1] = df_amp(p1); X[2] = df_amp(q0); X[3] = df_amp(q1);
    }
    Cplx<double> y[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) y[r] = df_row4(&u.e[4 * r], X);
    if (qa_low) {
      st_amp2<double>(a, b, y[0], y[2]);
      st_amp2<double>(a, b | mo, y[1], y[3]);
    } else {
      st_amp2<double>(a, b, y[0], y[1]);
      st_amp2<double>(a, b | mo, y[2], y[3]);
    }
  }
}

// ---------------------------------------------------------------------------
// host side: entries split into FP32 pairs, launches
// ---------------------------------------------------------------------------
static void split_host(double x, float& hi, float& lo) {
  hi = float(x);
  lo = float(x - double(hi));  // x - hi is exact in binary64
}

static DFCoef df_coef(double re, double im) {
  float rh, rl, ih, il;
  split_host(re, rh, rl);
  split_host(im, ih, il);
  DFCoef c;
  c.h1 = make_float2(rh, rh);
  c.n1 = make_float2(-rh, -rh);
  c.l1 = make_float2(rl, rl);
  c.h2 = make_float2(-ih, ih);
  c.n2 = make_float2(ih, -ih);
  c.l2 = make_float2(-il, il);
  return c;
}

qc_status df_1q_dense(double* a, const SweepSpec& sp, bool vec, bool low, const double* U, unsigned g,
                      cudaStream_t st) {
  DFMat2 m;
  for (int i = 0; i < 4; ++i) m.e[i] = df_coef(U[2 * i], U[2 * i + 1]);
  if (vec)
    QC_COUNT(), k_1q_dense_df<true><<<g, 256, 0, st>>>(a, sp, m);
  else if (low)
    QC_COUNT(), k_1q_dense_low_df<<<g, 256, 0, st>>>(a, sp, m);
  else
    QC_COUNT(), k_1q_dense_df<false><<<g, 256, 0, st>>>(a, sp, m);
  return check_launch("single-qubit gate (complex128)");
}

qc_status df_1q_diag(double* a, const SweepSpec& sp, bool vec, bool only1, const double* d0, const double* d1,
                     unsigned g, cudaStream_t st) {
  const DFCoef c0 = df_coef(d0[0], d0[1]), c1 = df_coef(d1[0], d1[1]);
  if (only1) {
    if (vec)
      QC_COUNT(), k_1q_diag_df<true, true><<<g, 256, 0, st>>>(a, sp, c1, c1);
    else
      QC_COUNT(), k_1q_diag_df<false, true><<<g, 256, 0, st>>>(a, sp, c1, c1);
  } else {
    if (vec)
      QC_COUNT(), k_1q_diag_df<true, false><<<g, 256, 0, st>>>(a, sp, c0, c1);
    else
      QC_COUNT(), k_1q_diag_df<false, false><<<g, 256, 0, st>>>(a, sp, c0, c1);
  }
  return check_launch("diagonal gate (complex128)");
}

qc_status df_1q_anti(double* a, const SweepSpec& sp, bool vec, const double* b, const double* c, unsigned g,
                     cudaStream_t st) {
  const DFCoef cb = df_coef(b[0], b[1]), cc = df_coef(c[0], c[1]);
  if (vec)
    QC_COUNT(), k_1q_anti_df<true><<<g, 256, 0, st>>>(a, sp, cb, cc);
  else
    QC_COUNT(), k_1q_anti_df<false><<<g, 256, 0, st>>>(a, sp, cb, cc);
  return check_launch("anti-diagonal gate (complex128)");
}

qc_status df_2q_dense(double* a, const SweepSpec& sp, bool vec, int low, const double* U, unsigned g,
                      cudaStream_t st) {
  DFMat4 m;
  for (int i = 0; i < 16; ++i) m.e[i] = df_coef(U[2 * i], U[2 * i + 1]);
  if (vec)
    QC_COUNT(), k_2q_dense_df<true><<<g, 256, 0, st>>>(a, sp, m);
  else if (low >= 0)
    QC_COUNT(), k_2q_dense_low_df<<<g, 256, 0, st>>>(a, sp, m, low == 1);
  else
    QC_COUNT(), k_2q_dense_df<false><<<g, 256, 0, st>>>(a, sp, m);
  return check_launch("two-qubit gate (complex128)");
}

}  // namespace qcgb
