// Shared definitions of the GB300 state-vector library (sm_103a).
//
// Index convention (QCLAB Sec. 3.2 / Sec. 5.1): qubit q is bit n-1-q of the
// amplitude index; "bit position" below always means the index bit, p = n-1-q.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "qc.h"

// ---------------------------------------------------------------------------
// state handle
// ---------------------------------------------------------------------------
struct qc_state {
  int n = 0;
  qc_dtype dtype = QC_C64;
  void* amps = nullptr;
  bool owned = false;
  cudaStream_t stream = nullptr;
  int device = 0;
  // lazily grown scratch owned by the handle (reductions, sampling tables)
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  // pinned host word for synchronising scalar reads
  double* host_buf = nullptr;
};

namespace qcgb {

constexpr int kNumSMs = 152;  // GB300: 2 dies x 76 SMs (queried at run time too)

// ---------------------------------------------------------------------------
// error reporting (thread-local message, status codes)
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();
qc_status check_cuda(cudaError_t e, const char* what);
qc_status check_launch(const char* what);
// Every kernel launch of the library is counted (qc_launch_count).
void count_launch();
#define QC_COUNT() ::qcgb::count_launch()

// Per-state scratch of at least `bytes`, aligned to 256 bytes.
qc_status state_scratch(qc_state* s, size_t bytes, void** out);
int device_sm_count();
// The status of a tensor-core kernel's device status word (0: completed; 1: a bounded
// wait ran out, the state's amplitudes are undefined), with the message set.
qc_status device_status(int word, const char* what);

inline uint64_t state_len(const qc_state* s) { return uint64_t(1) << s->n; }
inline size_t amp_bytes(qc_dtype d) { return d == QC_C64 ? 8 : 16; }

// grid for a grid-stride streaming kernel over `items` work items
inline unsigned stream_grid(uint64_t items, int block, int waves_per_sm = 16) {
  uint64_t need = (items + block - 1) / block;
  uint64_t cap = uint64_t(device_sm_count()) * waves_per_sm;
  if (need < 1) need = 1;
  return unsigned(need < cap ? need : cap);
}

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
// Inserts a zero bit at each of the `cnt` ascending positions in `pos`.
__device__ __forceinline__ uint64_t insert_zero_bits(uint64_t k, const int8_t* pos, int cnt) {
#pragma unroll 1
  for (int j = 0; j < cnt; ++j) {
    const int p = pos[j];
    const uint64_t lo = k & ((uint64_t(1) << p) - 1);
    k = ((k >> p) << (p + 1)) | lo;
  }
  return k;
}

template <typename R>
struct Cplx {
  R re, im;
};

template <typename R>
__device__ __forceinline__ Cplx<R> cmul(Cplx<R> a, Cplx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// a*x + b*y
template <typename R>
__device__ __forceinline__ Cplx<R> cmul2(Cplx<R> a, Cplx<R> x, Cplx<R> b, Cplx<R> y) {
  Cplx<R> r;
  r.re = fma(a.re, x.re, fma(-a.im, x.im, fma(b.re, y.re, -b.im * y.im)));
  r.im = fma(a.re, x.im, fma(a.im, x.re, fma(b.re, y.im, b.im * y.re)));
  return r;
}

// amplitude load/store (interleaved re, im)
template <typename R>
__device__ __forceinline__ Cplx<R> ld_amp(const R* a, uint64_t i);
template <>
__device__ __forceinline__ Cplx<float> ld_amp<float>(const float* a, uint64_t i) {
  float2 v = reinterpret_cast<const float2*>(a)[i];
  return {v.x, v.y};
}
template <>
__device__ __forceinline__ Cplx<double> ld_amp<double>(const double* a, uint64_t i) {
  double2 v = reinterpret_cast<const double2*>(a)[i];
  return {v.x, v.y};
}
template <typename R>
__device__ __forceinline__ void st_amp(R* a, uint64_t i, Cplx<R> v);
template <>
__device__ __forceinline__ void st_amp<float>(float* a, uint64_t i, Cplx<float> v) {
  reinterpret_cast<float2*>(a)[i] = make_float2(v.re, v.im);
}
template <>
__device__ __forceinline__ void st_amp<double>(double* a, uint64_t i, Cplx<double> v) {
  reinterpret_cast<double2*>(a)[i] = make_double2(v.re, v.im);
}

// two consecutive amplitudes i, i+1 (i even): one 16-byte access for complex64
template <typename R>
__device__ __forceinline__ void ld_amp2(const R* a, uint64_t i, Cplx<R>& x0, Cplx<R>& x1);
template <>
__device__ __forceinline__ void ld_amp2<float>(const float* a, uint64_t i, Cplx<float>& x0, Cplx<float>& x1) {
  float4 v = reinterpret_cast<const float4*>(a)[i >> 1];
  x0 = {v.x, v.y};
  x1 = {v.z, v.w};
}
template <>
__device__ __forceinline__ void ld_amp2<double>(const double* a, uint64_t i, Cplx<double>& x0,
                                                Cplx<double>& x1) {
  const double2* p = reinterpret_cast<const double2*>(a) + i;
  double2 v0 = p[0], v1 = p[1];
  x0 = {v0.x, v0.y};
  x1 = {v1.x, v1.y};
}
template <typename R>
__device__ __forceinline__ void st_amp2(R* a, uint64_t i, Cplx<R> x0, Cplx<R> x1);
template <>
__device__ __forceinline__ void st_amp2<float>(float* a, uint64_t i, Cplx<float> x0, Cplx<float> x1) {
  reinterpret_cast<float4*>(a)[i >> 1] = make_float4(x0.re, x0.im, x1.re, x1.im);
}
template <>
__device__ __forceinline__ void st_amp2<double>(double* a, uint64_t i, Cplx<double> x0, Cplx<double> x1) {
  double2* p = reinterpret_cast<double2*>(a) + i;
  p[0] = make_double2(x0.re, x0.im);
  p[1] = make_double2(x1.re, x1.im);
}

// complex64 amplitude as a packed FP32 pair (re, im), its swap (im, re), and back
__device__ __forceinline__ float2 f2(Cplx<float> z) { return make_float2(z.re, z.im); }
__device__ __forceinline__ float2 f2swap(Cplx<float> z) { return make_float2(z.im, z.re); }
__device__ __forceinline__ Cplx<float> c2(float2 z) { return Cplx<float>{z.x, z.y}; }

// |a|^2 in FP64 as two rounded products and one rounded sum (never fused)
__device__ __forceinline__ double prob_fp64(double re, double im) {
  return __dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im));
}

// Exact binary32 -> binary64 widening with integer operations only (IEEE 754 formats:
// sign bit, 8/11 exponent bits with bias 127/1023, 23/52 fraction bits), so that no
// conversion occupies the FP64 pipe.  A normal float keeps its sign and fraction
// (shifted up 29 bits) and has its exponent re-biased by 1023 - 127 = 896; zero keeps
// its sign; a subnormal m * 2^-149 with leading fraction bit p becomes a normal double
// with exponent p - 149 (biased: p + 874) and the bits below p as its fraction;
// infinities and NaNs keep their fraction under the all-ones exponent.
__device__ __forceinline__ double widen_exact(float x) {
  const uint32_t b = __float_as_uint(x);
  const uint32_t e = (b >> 23) & 0xFFu;
  const uint32_t m = b & 0x7FFFFFu;
  const uint64_t sign = uint64_t(b >> 31) << 63;
  uint64_t ed, md;
  if (e == 255u) {
    ed = 2047u;
    md = uint64_t(m) << 29;
  } else if (e != 0u) {
    ed = e + 896u;
    md = uint64_t(m) << 29;
  } else if (m == 0u) {
    ed = 0u;
    md = 0u;
  } else {
    const int p = 31 - __clz(int(m));
    ed = uint64_t(p + 874);
    md = (uint64_t(m) << (52 - p)) & ((uint64_t(1) << 52) - 1);
  }
  return __longlong_as_double((long long)(sign | (ed << 52) | md));
}

// x^2 as an exact double with integer operations only.  For a float with biased
// exponent e, |x| = M * 2^(max(e,1) - 150) with M = fraction | 2^23 for a normal float
// (M = fraction for a subnormal one), so x^2 = M^2 * 2^(2 max(e,1) - 300).  M^2 is
// an exact 48-bit integer product; with t its leading bit, x^2 is the normal double
// with exponent t + 2 max(e,1) - 300 and the bits of M^2 below t as its fraction.
// Infinities and NaNs keep their fraction under the all-ones exponent.
__device__ __forceinline__ double square_exact(float x) {
  const uint32_t b = __float_as_uint(x) & 0x7FFFFFFFu;
  const uint32_t e = b >> 23, m = b & 0x7FFFFFu;
  if (e == 255u) return __longlong_as_double((long long)((uint64_t(2047) << 52) | (uint64_t(m) << 29)));
  if (b == 0u) return 0.0;
  const uint32_t M = e ? (m | 0x800000u) : m;
  const int off = 2 * int(e ? e : 1u) - 300;
  const uint64_t P = uint64_t(M) * M;
  const int t = 63 - __clzll((long long)P);
  return __longlong_as_double(
      (long long)((uint64_t(t + off + 1023) << 52) | ((P << (52 - t)) & ((uint64_t(1) << 52) - 1))));
}

// The same |a|^2 for complex64 amplitudes: the squares of widened floats are exact in
// FP64 (24-bit significands), so one fused multiply-add of im * im onto the exact re^2
// rounds re^2 + im^2 once -- bit for bit the value of the two-product form above, with
// a single FP64 operation (re^2 is built with integer operations).
__device__ __forceinline__ double prob_fp64(float re, float im) {
  const double dim = widen_exact(im);
  return __fma_rn(dim, dim, square_exact(re));
}

// ---------------------------------------------------------------------------
// host-side gate matrices (FP64) -- the CUDA path's own definitions
// ---------------------------------------------------------------------------
struct HostMat2 {
  double m[8];  // row-major 2x2, (re, im)
};
struct HostMat4 {
  double m[32];
};

}  // namespace qcgb
