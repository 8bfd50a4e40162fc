// State handles, initialisation and the plain per-gate sweeps.
//
// QCLAB Sec. 3.2 applies a gate as the sparse product (I_l (x) U' (x) I_r) psi.  On
// the GPU that product is a sweep over the index groups the gate couples: for a
// single-qubit gate on bit p, the pairs (i, i | 2^p) with bit p clear; for a
// two-qubit gate, quads.  A work item's base index is obtained by inserting zero
// bits at the gate's (and controls') bit positions into a compressed counter, so
// consecutive threads touch consecutive addresses whenever bit 0 is not one of
// those positions; then each thread moves two neighbouring amplitudes per group
// member (one 16-byte access for complex64).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace qcgb {

static thread_local char g_err[512] = "";
static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
void clear_error() { g_err[0] = 0; }

qc_status check_cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return QC_OK;
  set_error("%s: %s", what, cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return QC_ERR_OOM;
  }
  return QC_ERR_CUDA;
}

qc_status check_launch(const char* what) { return check_cuda(cudaGetLastError(), what); }

int device_sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return kNumSMs;
  if (!cached[dev]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = kNumSMs;
    cached[dev] = v;
  }
  return cached[dev];
}

qc_status device_status(int word, const char* what) {
  if (word == 0) return QC_OK;
  if (word == 1) {
    set_error("%s: a bounded wait for a copy or the products ran out; the state's amplitudes are undefined", what);
    return QC_ERR_TIMEOUT;
  }
  set_error("%s: unexpected device status word %d; the state's amplitudes are undefined", what, word);
  return QC_ERR_CUDA;
}

qc_status state_scratch(qc_state* s, size_t bytes, void** out) {
  bytes = (bytes + 255) & ~size_t(255);
  if (s->scratch_bytes < bytes) {
    if (s->scratch) {
      cudaStreamSynchronize(s->stream);
      cudaFree(s->scratch);
      s->scratch = nullptr;
      s->scratch_bytes = 0;
    }
    void* p = nullptr;
    qc_status st = check_cuda(cudaMalloc(&p, bytes), "scratch allocation");
    if (st != QC_OK) return st;
    s->scratch = p;
    s->scratch_bytes = bytes;
  }
  *out = s->scratch;
  return QC_OK;
}

// ---------------------------------------------------------------------------
// initialisation kernels
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_set_basis(R* a, uint64_t index) {
  reinterpret_cast<R*>(a)[2 * index] = R(1);
}

template <typename RS, typename RD>
__global__ void k_convert(const RS* __restrict__ src, RD* __restrict__ dst, uint64_t len2) {
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < len2; i += uint64_t(gridDim.x) * blockDim.x)
    dst[i] = RD(src[i]);
}

// SplitMix64 (Steele, Lea, Flood 2014) as a counter-based stream
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t c) {
  uint64_t z = seed + (c + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double sm_uniform(uint64_t seed, uint64_t c) {
  return double(splitmix64(seed, c) >> 11) * 0x1.0p-53;
}
// Box-Muller (Box and Muller 1958) on uniforms 2j and 2j+1
__device__ __forceinline__ void gauss_amp(uint64_t seed, uint64_t j, double& re, double& im) {
  const double u1 = sm_uniform(seed, 2 * j), u2 = sm_uniform(seed, 2 * j + 1);
  const double r = sqrt(-2.0 * log1p(-u1));
  double sn, cs;
  sincos(2.0 * 3.141592653589793 * u2, &sn, &cs);
  re = r * cs;
  im = r * sn;
}

// Complex64 states: the same transform in FP32 (relative error ~1e-7 per amplitude,
// the size of complex64 rounding), with 1 - u1 = (2^53 - k1) 2^-53 formed exactly from
// the integer draw so that the logarithm stays accurate for u1 near 1.
__device__ __forceinline__ void gauss_amp(uint64_t seed, uint64_t j, float& re, float& im) {
  const uint64_t k1 = splitmix64(seed, 2 * j) >> 11, k2 = splitmix64(seed, 2 * j + 1) >> 11;
  const float v = float((uint64_t(1) << 53) - k1) * 0x1.0p-53f;  // 1 - u1 in (0, 1]
  const float r = sqrtf(-2.0f * logf(v));
  float sn, cs;
  sincospif(float(k2) * 0x1.0p-52f, &sn, &cs);  // angle 2 pi u2
  re = r * cs;
  im = r * sn;
}

template <typename R>
__global__ void k_gauss_norm_partials(uint64_t seed, uint64_t N, double* partials) {
  double acc = 0.0;
  for (uint64_t j = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; j < N; j += uint64_t(gridDim.x) * blockDim.x) {
    R re, im;
    gauss_amp(seed, j, re, im);
    if constexpr (sizeof(R) == 4)
      acc += widen_exact(fmaf(re, re, im * im));
    else
      acc += prob_fp64(re, im);
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

template <typename R>
__global__ void k_gauss_fill(uint64_t seed, uint64_t N, const double* norm2, R* a) {
  const double s = sqrt(*norm2);
  const float inv = float(1.0 / s);
  for (uint64_t j = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; j < N; j += uint64_t(gridDim.x) * blockDim.x) {
    R re, im;
    gauss_amp(seed, j, re, im);
    if constexpr (sizeof(R) == 4)
      st_amp<R>(a, j, {re * inv, im * inv});
    else
      st_amp<R>(a, j, {re / s, im / s});
  }
}

// Sum of `count` partials in a fixed order (deterministic), one block.
__global__ void k_sum_partials(const double* partials, int count, int stride, double* out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) acc += partials[size_t(i) * stride];
  acc = block_sum(acc);
  if (threadIdx.x == 0) *out = acc;
}

// ---------------------------------------------------------------------------
// per-gate sweeps
// ---------------------------------------------------------------------------
// Dense 2x2 on pairs.  VEC: each member is two neighbouring amplitudes.
template <typename R, bool VEC>
__global__ void __launch_bounds__(256) k_1q_dense(R* __restrict__ a, SweepSpec sp, Mat2<R> u) {
  const Cplx<R> u00{u.m[0], u.m[1]}, u01{u.m[2], u.m[3]}, u10{u.m[4], u.m[5]}, u11{u.m[6], u.m[7]};
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t it = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; it < sp.items; it += stride) {
    uint64_t i0 = insert_zero_bits(it, sp.pos, sp.cnt);
    if (VEC) i0 <<= 1;
    i0 |= sp.set_mask;
    const uint64_t i1 = i0 | sp.t0;
    if (VEC) {
      Cplx<R> x0, x1, y0, y1;
      ld_amp2<R>(a, i0, x0, x1);
      ld_amp2<R>(a, i1, y0, y1);
      st_amp2<R>(a, i0, cmul2(u00, x0, u01, y0), cmul2(u00, x1, u01, y1));
      st_amp2<R>(a, i1, cmul2(u10, x0, u11, y0), cmul2(u10, x1, u11, y1));
    } else {
      const Cplx<R> x = ld_amp<R>(a, i0), y = ld_amp<R>(a, i1);
      st_amp<R>(a, i0, cmul2(u00, x, u01, y));
      st_amp<R>(a, i1, cmul2(u10, x, u11, y));
    }
  }
}

// Dense 2x2 on bit 0: each pair is one 16-byte-aligned neighbour pair (i, i+1).
template <typename R>
__global__ void __launch_bounds__(256) k_1q_dense_low(R* __restrict__ a, SweepSpec sp, Mat2<R> u) {
  const Cplx<R> u00{u.m[0], u.m[1]}, u01{u.m[2], u.m[3]}, u10{u.m[4], u.m[5]}, u11{u.m[6], u.m[7]};
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t it = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; it < sp.items; it += stride) {
    const uint64_t i0 = insert_zero_bits(it, sp.pos, sp.cnt) | sp.set_mask;
    Cplx<R> x, y;
    ld_amp2<R>(a, i0, x, y);
    st_amp2<R>(a, i0, cmul2(u00, x, u01, y), cmul2(u10, x, u11, y));
  }
}

// Diagonal diag(d0, d1).  ONLY1: d0 == 1, only the bit-set member is touched
// (the target bit is part of sp.set_mask then).
template <typename R, bool VEC, bool ONLY1>
__global__ void __launch_bounds__(256) k_1q_diag(R* __restrict__ a, SweepSpec sp, Cplx<R> d0, Cplx<R> d1) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t it = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; it < sp.items; it += stride) {
    uint64_t i0 = insert_zero_bits(it, sp.pos, sp.cnt);
    if (VEC) i0 <<= 1;
    i0 |= sp.set_mask;
    if (ONLY1) {
      if (VEC) {
        Cplx<R> x0, x1;
        ld_amp2<R>(a, i0, x0, x1);
        st_amp2<R>(a, i0, cmul(d1, x0), cmul(d1, x1));
      } else {
        st_amp<R>(a, i0, cmul(d1, ld_amp<R>(a, i0)));
      }
    } else {
      const uint64_t i1 = i0 | sp.t0;
      if (VEC) {
        Cplx<R> x0, x1, y0, y1;
        ld_amp2<R>(a, i0, x0, x1);
        ld_amp2<R>(a, i1, y0, y1);
        st_amp2<R>(a, i0, cmul(d0, x0), cmul(d0, x1));
        st_amp2<R>(a, i1, cmul(d1, y0), cmul(d1, y1));
      } else {
        st_amp<R>(a, i0, cmul(d0, ld_amp<R>(a, i0)));
        st_amp<R>(a, i1, cmul(d1, ld_amp<R>(a, i1)));
      }
    }
  }
}

// Anti-diagonal [[0, b], [c, 0]]: out0 = b*in1, out1 = c*in0.  PURE: b = c = 1 (a swap).
template <typename R, bool VEC, bool PURE>
__global__ void __launch_bounds__(256) k_1q_anti(R* __restrict__ a, SweepSpec sp, Cplx<R> b, Cplx<R> c) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t it = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; it < sp.items; it += stride) {
    uint64_t i0 = insert_zero_bits(it, sp.pos, sp.cnt);
    if (VEC) i0 <<= 1;
    i0 |= sp.set_mask;
    const uint64_t i1 = i0 | sp.t0;
    if (VEC) {
      Cplx<R> x0, x1, y0, y1;
      ld_amp2<R>(a, i0, x0, x1);
      ld_amp2<R>(a, i1, y0, y1);
      if (PURE) {
        st_amp2<R>(a, i0, y0, y1);
        st_amp2<R>(a, i1, x0, x1);
      } else {
        st_amp2<R>(a, i0, cmul(b, y0), cmul(b, y1));
        st_amp2<R>(a, i1, cmul(c, x0), cmul(c, x1));
      }
    } else {
      const Cplx<R> x = ld_amp<R>(a, i0), y = ld_amp<R>(a, i1);
      st_amp<R>(a, i0, PURE ? y : cmul(b, y));
      st_amp<R>(a, i1, PURE ? x : cmul(c, x));
    }
  }
}

// Dense 4x4 on quads; member r = 2*b_qa + b_qb; t0 = mask of qa, t1 = mask of qb.
template <typename R, bool VEC>
__global__ void __launch_bounds__(256) k_2q_dense(R* __restrict__ a, SweepSpec sp, Mat4<R> u) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t it = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; it < sp.items; it += stride) {
    uint64_t b = insert_zero_bits(it, sp.pos, sp.cnt);
    if (VEC) b <<= 1;
    b |= sp.set_mask;
    const uint64_t idx[4] = {b, b | sp.t1, b | sp.t0, b | sp.t0 | sp.t1};
    if (VEC) {
      Cplx<R> x[4], y[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) ld_amp2<R>(a, idx[r], x[r], y[r]);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const Cplx<R> u0{u.m[8 * r + 0], u.m[8 * r + 1]}, u1{u.m[8 * r + 2], u.m[8 * r + 3]};
        const Cplx<R> u2{u.m[8 * r + 4], u.m[8 * r + 5]}, u3{u.m[8 * r + 6], u.m[8 * r + 7]};
        Cplx<R> o0 = cmul2(u0, x[0], u1, x[1]), o0b = cmul2(u2, x[2], u3, x[3]);
        Cplx<R> o1 = cmul2(u0, y[0], u1, y[1]), o1b = cmul2(u2, y[2], u3, y[3]);
        st_amp2<R>(a, idx[r], Cplx<R>{o0.re + o0b.re, o0.im + o0b.im}, Cplx<R>{o1.re + o1b.re, o1.im + o1b.im});
      }
    } else {
      Cplx<R> x[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) x[r] = ld_amp<R>(a, idx[r]);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const Cplx<R> u0{u.m[8 * r + 0], u.m[8 * r + 1]}, u1{u.m[8 * r + 2], u.m[8 * r + 3]};
        const Cplx<R> u2{u.m[8 * r + 4], u.m[8 * r + 5]}, u3{u.m[8 * r + 6], u.m[8 * r + 7]};
        Cplx<R> o0 = cmul2(u0, x[0], u1, x[1]), o0b = cmul2(u2, x[2], u3, x[3]);
        st_amp<R>(a, idx[r], Cplx<R>{o0.re + o0b.re, o0.im + o0b.im});
      }
    }
  }
}

// Dense 4x4 when bit 0 is one of the two targets: the quad is two 16-byte-aligned
// neighbour pairs, (b, b|1) and (b|m, b|m|1), m the other target's mask.  qa_low: bit 0
// belongs to the first qubit (row index 2*b_qa + b_qb).
template <typename R>
__global__ void __launch_bounds__(256) k_2q_dense_low(R* __restrict__ a, SweepSpec sp, Mat4<R> u, bool qa_low) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  const uint64_t mo = qa_low ? sp.t1 : sp.t0;  // mask of the other target
  for (uint64_t it = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; it < sp.items; it += stride) {
    const uint64_t b = insert_zero_bits(it, sp.pos, sp.cnt);
    Cplx<R> p0, p1, q0, q1;  // p = (b, b|1), q = (b|mo, b|mo|1)
    ld_amp2<R>(a, b, p0, p1);
    ld_amp2<R>(a, b | mo, q0, q1);
    // x[r], r = 2*b_qa + b_qb
    Cplx<R> x[4];
    if (qa_low) {
      x[0] = p0; x[2] = p1; x[1] = q0; x[3] = q1;
    } else {
      x[0] = p0; x[1] = p1; x[2] = q0; x[3] = q1;
    }
    Cplx<R> y[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const Cplx<R> u0{u.m[8 * r + 0], u.m[8 * r + 1]}, u1{u.m[8 * r + 2], u.m[8 * r + 3]};
      const Cplx<R> u2{u.m[8 * r + 4], u.m[8 * r + 5]}, u3{u.m[8 * r + 6], u.m[8 * r + 7]};
      const Cplx<R> o0 = cmul2(u0, x[0], u1, x[1]), o1 = cmul2(u2, x[2], u3, x[3]);
      y[r] = Cplx<R>{o0.re + o1.re, o0.im + o1.im};
    }
    if (qa_low) {
      st_amp2<R>(a, b, y[0], y[2]);
      st_amp2<R>(a, b | mo, y[1], y[3]);
    } else {
      st_amp2<R>(a, b, y[0], y[1]);
      st_amp2<R>(a, b | mo, y[2], y[3]);
    }
  }
}

// SWAP of two qubits: exchanges members 01 and 10 of every quad.
template <typename R, bool VEC>
__global__ void __launch_bounds__(256) k_2q_swap(R* __restrict__ a, SweepSpec sp) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t it = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; it < sp.items; it += stride) {
    uint64_t b = insert_zero_bits(it, sp.pos, sp.cnt);
    if (VEC) b <<= 1;
    b |= sp.set_mask;
    const uint64_t i01 = b | sp.t1, i10 = b | sp.t0;
    if (VEC) {
      Cplx<R> x0, x1, y0, y1;
      ld_amp2<R>(a, i01, x0, x1);
      ld_amp2<R>(a, i10, y0, y1);
      st_amp2<R>(a, i01, y0, y1);
      st_amp2<R>(a, i10, x0, x1);
    } else {
      const Cplx<R> x = ld_amp<R>(a, i01), y = ld_amp<R>(a, i10);
      st_amp<R>(a, i01, y);
      st_amp<R>(a, i10, x);
    }
  }
}

// ---------------------------------------------------------------------------
// host dispatch
// ---------------------------------------------------------------------------
static bool is_zero(double re, double im) { return re == 0.0 && im == 0.0; }
static bool is_one(double re, double im) { return re == 1.0 && im == 0.0; }

// Builds the sweep spec for `special` bit positions (targets and controls); the
// items count covers one group per combination of the other bits.
static SweepSpec make_spec(int n, std::vector<int> special, uint64_t set_mask, uint64_t t0, uint64_t t1,
                           bool& vec) {
  std::sort(special.begin(), special.end());
  SweepSpec sp{};
  vec = special.empty() || special[0] >= 1;
  if (n - int(special.size()) < 1) vec = false;  // too few free bits to pair neighbours
  sp.cnt = int(special.size());
  for (int j = 0; j < sp.cnt; ++j) sp.pos[j] = int8_t(vec ? special[j] - 1 : special[j]);
  const int free_bits = n - sp.cnt - (vec ? 1 : 0);
  sp.items = uint64_t(1) << free_bits;
  sp.set_mask = set_mask;
  sp.t0 = t0;
  sp.t1 = t1;
  return sp;
}

template <typename R>
static qc_status launch_1q(qc_state* s, int tbit, const std::vector<int>& cbits, uint64_t cset, const double* U) {
  R* a = reinterpret_cast<R*>(s->amps);
  const uint64_t tm = uint64_t(1) << tbit;
  const bool diag = is_zero(U[2], U[3]) && is_zero(U[4], U[5]);
  const bool anti = is_zero(U[0], U[1]) && is_zero(U[6], U[7]);
  std::vector<int> special = cbits;
  special.push_back(tbit);
  bool vec = false;
  const int B = 256;
  if (diag && is_one(U[0], U[1])) {
    if (is_one(U[6], U[7])) return QC_OK;  // identity
    SweepSpec sp = make_spec(s->n, special, cset | tm, tm, 0, vec);
    const Cplx<R> d1{R(U[6]), R(U[7])};
    const unsigned g = stream_grid(sp.items, B);
    if (sizeof(R) == 8 && s->n >= kDfMinQubits)
      return df_1q_diag(reinterpret_cast<double*>(a), sp, vec, true, U, U + 6, g, s->stream);
    if (vec)
      QC_COUNT(), k_1q_diag<R, true, true><<<g, B, 0, s->stream>>>(a, sp, d1, d1);
    else
      QC_COUNT(), k_1q_diag<R, false, true><<<g, B, 0, s->stream>>>(a, sp, d1, d1);
    return check_launch("diagonal gate");
  }
  SweepSpec sp = make_spec(s->n, special, cset, tm, 0, vec);
  const unsigned g = stream_grid(sp.items, B);
  const bool pure_anti = anti && is_one(U[2], U[3]) && is_one(U[4], U[5]);
  if (sizeof(R) == 8 && s->n >= kDfMinQubits && !pure_anti) {
    double* ad = reinterpret_cast<double*>(a);
    if (diag) return df_1q_diag(ad, sp, vec, false, U, U + 6, g, s->stream);
    if (anti) return df_1q_anti(ad, sp, vec, U + 2, U + 4, g, s->stream);
    return df_1q_dense(ad, sp, vec, tbit == 0, U, g, s->stream);
  }
  if (diag) {
    const Cplx<R> d0{R(U[0]), R(U[1])}, d1{R(U[6]), R(U[7])};
    if (vec)
      QC_COUNT(), k_1q_diag<R, true, false><<<g, B, 0, s->stream>>>(a, sp, d0, d1);
    else
      QC_COUNT(), k_1q_diag<R, false, false><<<g, B, 0, s->stream>>>(a, sp, d0, d1);
  } else if (anti) {
    const Cplx<R> b{R(U[2]), R(U[3])}, c{R(U[4]), R(U[5])};
    if (pure_anti) {
      if (vec)
        QC_COUNT(), k_1q_anti<R, true, true><<<g, B, 0, s->stream>>>(a, sp, b, c);
      else
        QC_COUNT(), k_1q_anti<R, false, true><<<g, B, 0, s->stream>>>(a, sp, b, c);
    } else {
      if (vec)
        QC_COUNT(), k_1q_anti<R, true, false><<<g, B, 0, s->stream>>>(a, sp, b, c);
      else
        QC_COUNT(), k_1q_anti<R, false, false><<<g, B, 0, s->stream>>>(a, sp, b, c);
    }
  } else {
    Mat2<R> m;
    for (int i = 0; i < 8; ++i) m.m[i] = R(U[i]);
    if (vec)
      QC_COUNT(), k_1q_dense<R, true><<<g, B, 0, s->stream>>>(a, sp, m);
    else
      QC_COUNT(), (tbit == 0 ? k_1q_dense_low<R> : k_1q_dense<R, false>)<<<g, B, 0, s->stream>>>(a, sp, m);
  }
  return check_launch("single-qubit gate");
}

qc_status apply_1q_bits(qc_state* s, int tbit, const int* cbits, const int* cvals, int nctrl, const double* U) {
  std::vector<int> cb(cbits, cbits + nctrl);
  uint64_t cset = 0;
  for (int j = 0; j < nctrl; ++j)
    if (cvals[j]) cset |= uint64_t(1) << cbits[j];
  return s->dtype == QC_C64 ? launch_1q<float>(s, tbit, cb, cset, U) : launch_1q<double>(s, tbit, cb, cset, U);
}

template <typename R>
static qc_status launch_2q(qc_state* s, int pa, int pb, const double* U) {
  R* a = reinterpret_cast<R*>(s->amps);
  bool vec = false;
  SweepSpec sp = make_spec(s->n, {pa, pb}, 0, uint64_t(1) << pa, uint64_t(1) << pb, vec);
  const int B = 256;
  const unsigned g = stream_grid(sp.items, B);
  if (sizeof(R) == 8 && s->n >= kDfMinQubits)
    return df_2q_dense(reinterpret_cast<double*>(a), sp, vec, vec ? -1 : pa == 0 ? 1 : pb == 0 ? 0 : -1, U, g,
                       s->stream);
  Mat4<R> m;
  for (int i = 0; i < 32; ++i) m.m[i] = R(U[i]);
  if (vec)
    QC_COUNT(), k_2q_dense<R, true><<<g, B, 0, s->stream>>>(a, sp, m);
  else if (pa == 0 || pb == 0)
    QC_COUNT(), k_2q_dense_low<R><<<g, B, 0, s->stream>>>(a, sp, m, pa == 0);
  else
    QC_COUNT(), k_2q_dense<R, false><<<g, B, 0, s->stream>>>(a, sp, m);
  return check_launch("two-qubit gate");
}

template <typename R>
static qc_status launch_swap(qc_state* s, int pa, int pb) {
  R* a = reinterpret_cast<R*>(s->amps);
  bool vec = false;
  SweepSpec sp = make_spec(s->n, {pa, pb}, 0, uint64_t(1) << pa, uint64_t(1) << pb, vec);
  const int B = 256;
  const unsigned g = stream_grid(sp.items, B);
  if (vec)
    QC_COUNT(), k_2q_swap<R, true><<<g, B, 0, s->stream>>>(a, sp);
  else
    QC_COUNT(), k_2q_swap<R, false><<<g, B, 0, s->stream>>>(a, sp);
  return check_launch("swap gate");
}

// Two-qubit dense gate with a structure check: diagonal and SWAP-like matrices
// go to the cheaper sweeps.
qc_status apply_2q_bits(qc_state* s, int pa, int pb, const double* U) {
  // SWAP: permutation 0->0, 1->2, 2->1, 3->3 with unit entries
  bool swap = true, diag = true;
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      const double re = U[8 * r + 2 * c], im = U[8 * r + 2 * c + 1];
      const int sc = (r == 1) ? 2 : (r == 2) ? 1 : r;
      if (c == sc) {
        if (!is_one(re, im)) swap = false;
      } else if (!is_zero(re, im)) {
        swap = false;
      }
      if (r != c && !is_zero(re, im)) diag = false;
    }
  if (swap) return s->dtype == QC_C64 ? launch_swap<float>(s, pa, pb) : launch_swap<double>(s, pa, pb);
  if (diag && is_one(U[0], U[1]) && is_one(U[10], U[11]) && is_one(U[20], U[21])) {
    // diag(1,1,1,d): controlled phase, touches a quarter of the state
    const double d[8] = {1, 0, 0, 0, 0, 0, U[30], U[31]};
    const int c = 1;
    return apply_1q_bits(s, pb, &pa, &c, 1, d);
  }
  return s->dtype == QC_C64 ? launch_2q<float>(s, pa, pb, U) : launch_2q<double>(s, pa, pb, U);
}

}  // namespace qcgb

using namespace qcgb;

// ---------------------------------------------------------------------------
// C ABI: handles and initialisation
// ---------------------------------------------------------------------------
extern "C" {

const char* qc_last_error(void) { return g_err; }
int qc_abi_version(void) { return 2; }

qc_status qc_status_of_device_word(int word) {
  clear_error();
  return device_status(word, "tensor-core kernel");
}
uint64_t qc_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

static qc_status valid_state(const qc_state* s) {
  if (!s || !s->amps || s->n < 1) {
    set_error("invalid state handle");
    return QC_ERR_INVALID_ARG;
  }
  return QC_OK;
}

static qc_status bind_device(const qc_state* s) {
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != s->device) return check_cuda(cudaSetDevice(s->device), "cudaSetDevice");
  return QC_OK;
}

qc_status qc_state_alloc(int n, qc_dtype dtype, void* stream, qc_state** out) {
  clear_error();
  if (!out || n < 1 || n > 34 || (dtype != QC_C64 && dtype != QC_C128)) {
    set_error("qc_state_alloc: invalid arguments (n=%d, dtype=%d)", n, int(dtype));
    return QC_ERR_INVALID_ARG;
  }
  const size_t bytes = (size_t(1) << n) * amp_bytes(dtype);
  void* p = nullptr;
  qc_status st = check_cuda(cudaMalloc(&p, bytes), "state allocation");
  if (st != QC_OK) return st;
  qc_state* s = new qc_state();
  s->n = n;
  s->dtype = dtype;
  s->amps = p;
  s->owned = true;
  s->stream = reinterpret_cast<cudaStream_t>(stream);
  cudaGetDevice(&s->device);
  *out = s;
  return QC_OK;
}

qc_status qc_state_wrap(int n, qc_dtype dtype, void* dev_amps, void* stream, qc_state** out) {
  clear_error();
  if (!out || !dev_amps || n < 1 || n > 34 || (dtype != QC_C64 && dtype != QC_C128) ||
      (reinterpret_cast<uintptr_t>(dev_amps) & 15)) {
    set_error("qc_state_wrap: invalid arguments (n=%d, dtype=%d, ptr=%p; 16-byte alignment required)", n,
              int(dtype), dev_amps);
    return QC_ERR_INVALID_ARG;
  }
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, dev_amps) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    set_error("qc_state_wrap: pointer is not device memory");
    return QC_ERR_INVALID_ARG;
  }
  qc_state* s = new qc_state();
  s->n = n;
  s->dtype = dtype;
  s->amps = dev_amps;
  s->owned = false;
  s->stream = reinterpret_cast<cudaStream_t>(stream);
  s->device = attr.device;
  *out = s;
  return QC_OK;
}

qc_status qc_state_free(qc_state* s) {
  clear_error();
  if (!s) return QC_OK;
  int cur = -1;
  cudaGetDevice(&cur);
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->stream);
  if (s->owned && s->amps) cudaFree(s->amps);
  if (s->scratch) cudaFree(s->scratch);
  if (s->host_buf) cudaFreeHost(s->host_buf);
  if (cur >= 0) cudaSetDevice(cur);
  delete s;
  return check_launch("qc_state_free");
}

qc_status qc_state_info(const qc_state* s, int* n, qc_dtype* dtype, void** dev_amps) {
  clear_error();
  if (qc_status st = valid_state(s)) return st;
  if (n) *n = s->n;
  if (dtype) *dtype = s->dtype;
  if (dev_amps) *dev_amps = s->amps;
  return QC_OK;
}

qc_status qc_state_set_stream(qc_state* s, void* stream) {
  clear_error();
  if (qc_status st = valid_state(s)) return st;
  s->stream = reinterpret_cast<cudaStream_t>(stream);
  return QC_OK;
}

qc_status qc_state_init_basis(qc_state* s, uint64_t index) {
  clear_error();
  if (qc_status st = valid_state(s)) return st;
  if (index >= state_len(s)) {
    set_error("qc_state_init_basis: index %llu out of range", (unsigned long long)index);
    return QC_ERR_INVALID_ARG;
  }
  if (qc_status st = bind_device(s)) return st;
  qc_status st = check_cuda(cudaMemsetAsync(s->amps, 0, state_len(s) * amp_bytes(s->dtype), s->stream), "memset");
  if (st != QC_OK) return st;
  if (s->dtype == QC_C64)
    QC_COUNT(), k_set_basis<float><<<1, 1, 0, s->stream>>>(reinterpret_cast<float*>(s->amps), index);
  else
    QC_COUNT(), k_set_basis<double><<<1, 1, 0, s->stream>>>(reinterpret_cast<double*>(s->amps), index);
  return check_launch("qc_state_init_basis");
}

qc_status qc_state_init_vector(qc_state* s, const void* amps, qc_dtype src, int src_on_host) {
  clear_error();
  if (qc_status st = valid_state(s)) return st;
  if (!amps || (src != QC_C64 && src != QC_C128)) {
    set_error("qc_state_init_vector: invalid arguments");
    return QC_ERR_INVALID_ARG;
  }
  if (qc_status st = bind_device(s)) return st;
  const uint64_t N = state_len(s);
  const size_t src_bytes = N * amp_bytes(src);
  const void* dsrc = amps;
  if (src_on_host) {
    if (src == s->dtype)
      return check_cuda(cudaMemcpyAsync(s->amps, amps, src_bytes, cudaMemcpyHostToDevice, s->stream), "H2D copy");
    void* tmp = nullptr;
    if (qc_status st = state_scratch(s, src_bytes, &tmp)) return st;
    if (qc_status st = check_cuda(cudaMemcpyAsync(tmp, amps, src_bytes, cudaMemcpyHostToDevice, s->stream), "H2D"))
      return st;
    dsrc = tmp;
  } else if (src == s->dtype) {
    return check_cuda(cudaMemcpyAsync(s->amps, amps, src_bytes, cudaMemcpyDeviceToDevice, s->stream), "D2D copy");
  }
  const unsigned g = stream_grid(2 * N, 256);
  if (src == QC_C64)
    QC_COUNT(), k_convert<float, double><<<g, 256, 0, s->stream>>>(reinterpret_cast<const float*>(dsrc),
                                                       reinterpret_cast<double*>(s->amps), 2 * N);
  else
    QC_COUNT(), k_convert<double, float><<<g, 256, 0, s->stream>>>(reinterpret_cast<const double*>(dsrc),
                                                       reinterpret_cast<float*>(s->amps), 2 * N);
  return check_launch("qc_state_init_vector");
}

qc_status qc_state_init_gaussian(qc_state* s, uint64_t seed) {
  clear_error();
  if (qc_status st = valid_state(s)) return st;
  if (qc_status st = bind_device(s)) return st;
  const uint64_t N = state_len(s);
  const int B = 256;
  const unsigned g = stream_grid(N, B, 8);
  void* scr = nullptr;
  if (qc_status st = state_scratch(s, sizeof(double) * (g + 1), &scr)) return st;
  double* partials = reinterpret_cast<double*>(scr);
  if (s->dtype == QC_C64)
    QC_COUNT(), k_gauss_norm_partials<float><<<g, B, 0, s->stream>>>(seed, N, partials);
  else
    QC_COUNT(), k_gauss_norm_partials<double><<<g, B, 0, s->stream>>>(seed, N, partials);
  QC_COUNT(), k_sum_partials<<<1, 1024, 0, s->stream>>>(partials, int(g), 1, partials + g);
  if (s->dtype == QC_C64)
    QC_COUNT(), k_gauss_fill<float><<<g, B, 0, s->stream>>>(seed, N, partials + g, reinterpret_cast<float*>(s->amps));
  else
    QC_COUNT(), k_gauss_fill<double><<<g, B, 0, s->stream>>>(seed, N, partials + g, reinterpret_cast<double*>(s->amps));
  if (qc_status st = check_launch("qc_state_init_gaussian")) return st;
  return check_cuda(cudaStreamSynchronize(s->stream), "qc_state_init_gaussian");
}

qc_status qc_state_copy(qc_state* dst, const qc_state* src) {
  clear_error();
  if (qc_status st = valid_state(dst)) return st;
  if (qc_status st = valid_state(src)) return st;
  if (dst->n != src->n || dst->dtype != src->dtype) {
    set_error("qc_state_copy: shape mismatch");
    return QC_ERR_INVALID_ARG;
  }
  if (qc_status st = bind_device(dst)) return st;
  return check_cuda(cudaMemcpyAsync(dst->amps, src->amps, state_len(src) * amp_bytes(src->dtype),
                                    cudaMemcpyDeviceToDevice, dst->stream),
                    "qc_state_copy");
}

qc_status qc_state_download(const qc_state* s, void* host_dst) {
  clear_error();
  if (qc_status st = valid_state(s)) return st;
  if (!host_dst) {
    set_error("qc_state_download: null destination");
    return QC_ERR_INVALID_ARG;
  }
  if (qc_status st = bind_device(s)) return st;
  qc_status st = check_cuda(
      cudaMemcpyAsync(host_dst, s->amps, state_len(s) * amp_bytes(s->dtype), cudaMemcpyDeviceToHost, s->stream),
      "D2H copy");
  if (st != QC_OK) return st;
  return check_cuda(cudaStreamSynchronize(s->stream), "qc_state_download");
}

// ---------------------------------------------------------------------------
// C ABI: gates
// ---------------------------------------------------------------------------
static bool valid_qubits(const qc_state* s, const int* q, int k) {
  for (int i = 0; i < k; ++i) {
    if (q[i] < 0 || q[i] >= s->n) return false;
    for (int j = 0; j < i; ++j)
      if (q[i] == q[j]) return false;
  }
  return true;
}

qc_status qc_apply_1q(qc_state* s, int q, const double U[8]) {
  clear_error();
  if (qc_status st = valid_state(s)) return st;
  if (!U || !valid_qubits(s, &q, 1)) {
    set_error("qc_apply_1q: invalid qubit %d or matrix", q);
    return QC_ERR_INVALID_ARG;
  }
  if (qc_status st = bind_device(s)) return st;
  return apply_1q_bits(s, s->n - 1 - q, nullptr, nullptr, 0, U);
}

qc_status qc_apply_2q(qc_state* s, int qa, int qb, const double U[32]) {
  clear_error();
  if (qc_status st = valid_state(s)) return st;
  int qs[2] = {qa, qb};
  if (!U || s->n < 2 || !valid_qubits(s, qs, 2)) {
    set_error("qc_apply_2q: invalid qubits (%d, %d) or matrix", qa, qb);
    return QC_ERR_INVALID_ARG;
  }
  if (qc_status st = bind_device(s)) return st;
  return apply_2q_bits(s, s->n - 1 - qa, s->n - 1 - qb, U);
}

qc_status qc_apply_ctrl(qc_state* s, const int* ctrls, const int* ctrl_states, int nctrl, int target,
                        const double U[8]) {
  clear_error();
  if (qc_status st = valid_state(s)) return st;
  if (!U || nctrl < 0 || nctrl > 6 || (nctrl > 0 && !ctrls) || nctrl + 1 > s->n) {
    set_error("qc_apply_ctrl: invalid arguments");
    return QC_ERR_INVALID_ARG;
  }
  int qs[8];
  for (int j = 0; j < nctrl; ++j) qs[j] = ctrls[j];
  qs[nctrl] = target;
  if (!valid_qubits(s, qs, nctrl + 1)) {
    set_error("qc_apply_ctrl: qubits must be distinct and in [0, n)");
    return QC_ERR_INVALID_ARG;
  }
  int cb[8], cv[8];
  for (int j = 0; j < nctrl; ++j) {
    cb[j] = s->n - 1 - ctrls[j];
    cv[j] = ctrl_states ? ctrl_states[j] : 1;
    if (cv[j] != 0 && cv[j] != 1) {
      set_error("qc_apply_ctrl: control states must be 0 or 1");
      return QC_ERR_INVALID_ARG;
    }
  }
  if (qc_status st = bind_device(s)) return st;
  return apply_1q_bits(s, s->n - 1 - target, cb, cv, nctrl, U);
}

}  // extern "C"
