// Measurement, probabilities and sampling (QCLAB Sec. 3.3).
//
//  * P(o) = sum_{i : bit_q(i) = o} |psi_i|^2, reduced per block in FP64 and summed in a
//    fixed order (deterministic).
//  * Collapse keeps the outcome's half and divides it by sqrt(P(o)) in FP64.
//  * Sampling draws min{k : u*T < cdf_k}.  The prefix sums are exact: every FP64
//    p_i is converted to a 128-bit fixed-point integer (unit 2^-118), integer sums are
//    associative, so any blocking gives the same cdf_k = round-to-nearest(exact
//    prefix), which is what the sequential double-double oracle approximates to
//    ~2^-100 relative.  The table kept between kernels is one 128-bit sum per leaf
//    of 64 amplitudes; each shot re-derives its leaf's 64 prefix values with half a warp.
#include <cmath>

#include "common.cuh"
#include "kernels.cuh"

namespace qcgb {

// ---------------------------------------------------------------------------
// P(0), P(1) partials
// ---------------------------------------------------------------------------
// Two neighbouring amplitudes i, i+1 into the outcome sums: complex128 adds the four
// squares into the FP64 sums with fused multiply-adds; complex64 forms the squared
// magnitudes in FP32 (relative error 2^-24 each) and adds them to the FP32 group sums
// g0, g1, which the caller widens into the FP64 sums every four steps (eight
// amplitudes: relative error below 7 * 2^-24 per group), so that the FP64 pipe sees
// one add per group and outcome instead of one per step.
template <typename R>
__device__ __forceinline__ void outcome_add(uint64_t i, uint64_t m, const Cplx<R>& x0, const Cplx<R>& x1, R& g0,
                                            R& g1) {
  if constexpr (sizeof(R) == 4) {
    const float f0 = fmaf(x0.re, x0.re, x0.im * x0.im), f1 = fmaf(x1.re, x1.re, x1.im * x1.im);
    if (m == 1) {
      g0 += f0;
      g1 += f1;
    } else if (i & m) {
      g1 += f0 + f1;
    } else {
      g0 += f0 + f1;
    }
  } else {
    if (m == 1) {
      g0 = fma(x0.im, x0.im, fma(x0.re, x0.re, g0));
      g1 = fma(x1.im, x1.im, fma(x1.re, x1.re, g1));
    } else {
      R& g = (i & m) ? g1 : g0;
      g = fma(x1.im, x1.im, fma(x1.re, x1.re, fma(x0.im, x0.im, fma(x0.re, x0.re, g))));
    }
  }
}

template <typename R>
__device__ __forceinline__ void outcome_flush(float& g0, float& g1, double& s0, double& s1) {
  s0 += widen_exact(g0);
  s1 += widen_exact(g1);
  g0 = g1 = 0.f;
}

// Two neighbouring amplitudes per step; each thread issues the loads of four steps
// before it uses them, so enough bytes are in flight to cover the memory latency.
template <typename R>
__global__ void __launch_bounds__(256) k_outcome_partials(const R* __restrict__ a, uint64_t N, uint64_t m,
                                                          double* partials) {
  // complex64: FP32 group sums g, FP64 sums s; complex128: the FP64 sums directly
  R g0 = R(0), g1 = R(0);
  double s0 = 0.0, s1 = 0.0;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  const uint64_t half = N / 2;
  uint64_t it = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x;
  for (; it + 3 * stride < half; it += 4 * stride) {
    Cplx<R> x[8];
#pragma unroll
    for (int u = 0; u < 4; ++u) ld_amp2<R>(a, 2 * (it + u * stride), x[2 * u], x[2 * u + 1]);
#pragma unroll
    for (int u = 0; u < 4; ++u) outcome_add<R>(2 * (it + u * stride), m, x[2 * u], x[2 * u + 1], g0, g1);
    if constexpr (sizeof(R) == 4) outcome_flush<R>(g0, g1, s0, s1);
  }
  for (; it < half; it += stride) {
    Cplx<R> x0, x1;
    ld_amp2<R>(a, 2 * it, x0, x1);
    outcome_add<R>(2 * it, m, x0, x1, g0, g1);
    if constexpr (sizeof(R) == 4) outcome_flush<R>(g0, g1, s0, s1);
  }
  if constexpr (sizeof(R) == 8) {
    s0 = g0;
    s1 = g1;
  }
  s0 = block_sum(s0);
  s1 = block_sum(s1);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = s0;
    partials[2 * blockIdx.x + 1] = s1;
  }
}

__global__ void k_sum2(const double* partials, int count, double* out) {
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    a += partials[2 * i];
    b += partials[2 * i + 1];
  }
  a = block_sum(a);
  b = block_sum(b);
  if (threadIdx.x == 0) {
    out[0] = a;
    out[1] = b;
  }
}

// Keeps the amplitudes whose bit m reads `outcome`, scaled by inv = 1/sqrt(P) (formed
// once in FP64 by the host; complex64 applies it rounded to FP32), and zeroes the rest
// without reading them.  Two neighbouring amplitudes per step (N >= 2); each thread
// issues the loads of four steps before their stores.
template <typename R>
__device__ __forceinline__ bool collapse_reads(uint64_t i, uint64_t m, int outcome) {
  return m == 1 || ((i & m) ? 1 : 0) == outcome;
}

template <typename R>
__device__ __forceinline__ void collapse_store(R* a, uint64_t i, uint64_t m, int outcome, R f, const Cplx<R>& x0,
                                               const Cplx<R>& x1) {
  const Cplx<R> zero{R(0), R(0)};
  if (m == 1) {
    if (outcome == 0)
      st_amp2<R>(a, i, Cplx<R>{x0.re * f, x0.im * f}, zero);
    else
      st_amp2<R>(a, i, zero, Cplx<R>{x1.re * f, x1.im * f});
  } else if (((i & m) ? 1 : 0) != outcome) {
    st_amp2<R>(a, i, zero, zero);
  } else {
    st_amp2<R>(a, i, Cplx<R>{x0.re * f, x0.im * f}, Cplx<R>{x1.re * f, x1.im * f});
  }
}

template <typename R>
__global__ void __launch_bounds__(256) k_collapse(R* __restrict__ a, uint64_t N, uint64_t m, int outcome,
                                                  double inv) {
  const R f = R(inv);
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  const uint64_t half = N / 2;
  uint64_t it = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x;
  for (; it + 3 * stride < half; it += 4 * stride) {
    Cplx<R> x[8];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint64_t i = 2 * (it + u * stride);
      if (collapse_reads<R>(i, m, outcome))
        ld_amp2<R>(a, i, x[2 * u], x[2 * u + 1]);
      else
        x[2 * u] = x[2 * u + 1] = Cplx<R>{R(0), R(0)};
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) collapse_store<R>(a, 2 * (it + u * stride), m, outcome, f, x[2 * u], x[2 * u + 1]);
  }
  for (; it < half; it += stride) {
    const uint64_t i = 2 * it;
    Cplx<R> x0{R(0), R(0)}, x1{R(0), R(0)};
    if (collapse_reads<R>(i, m, outcome)) ld_amp2<R>(a, i, x0, x1);
    collapse_store<R>(a, i, m, outcome, f, x0, x1);
  }
}

// ---------------------------------------------------------------------------
// probabilities
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_probs(const R* __restrict__ a, uint64_t N, double* __restrict__ p) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  if (N == 1) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      Cplx<R> v = ld_amp<R>(a, 0);
      p[0] = prob_fp64(v.re, v.im);
    }
    return;
  }
  for (uint64_t it = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; it < N / 2; it += stride) {
    Cplx<R> x0, x1;
    ld_amp2<R>(a, 2 * it, x0, x1);
    reinterpret_cast<double2*>(p)[it] =
        make_double2(prob_fp64(x0.re, x0.im), prob_fp64(x1.re, x1.im));
  }
}

// ---------------------------------------------------------------------------
// exact prefix sums in 128-bit fixed point (unit 2^-118, sums below 2^10)
// ---------------------------------------------------------------------------
struct U128 {
  uint64_t lo, hi;
};
__device__ __forceinline__ U128 add128(U128 a, U128 b) {
  U128 r;
  r.lo = a.lo + b.lo;
  r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ull : 0ull);
  return r;
}
__device__ __forceinline__ U128 shfl_up128(U128 v, int d) {
  U128 r;
  r.lo = __shfl_up_sync(0xffffffffu, v.lo, d);
  r.hi = __shfl_up_sync(0xffffffffu, v.hi, d);
  return r;
}
__device__ __forceinline__ U128 shfl128(U128 v, int src) {
  U128 r;
  r.lo = __shfl_sync(0xffffffffu, v.lo, src);
  r.hi = __shfl_sync(0xffffffffu, v.hi, src);
  return r;
}

// p (finite, >= 0) in units of 2^-118, bits below the unit truncated.
__device__ __forceinline__ U128 to_fixed(double p) {
  const uint64_t b = uint64_t(__double_as_longlong(p));
  const int e = int((b >> 52) & 0x7FF);
  U128 r{0, 0};
  if (e == 0) return r;  // zero or subnormal (< 2^-1022): below the unit
  const uint64_t m = (b & ((1ull << 52) - 1)) | (1ull << 52);
  const int sh = e - 957;  // p = m * 2^(e-1075) = m * 2^(e-957) units
  if (sh >= 0) {
    if (sh >= 64) {
      r.hi = m << (sh - 64);
    } else {
      r.lo = m << sh;
      r.hi = sh == 0 ? 0 : (m >> (64 - sh));
    }
  } else if (sh > -64) {
    r.lo = m >> (-sh);
  }
  return r;
}

// Round-to-nearest-even conversion back to FP64, built as the double's bit pattern with
// integer operations (IEEE 754 binary64: 11-bit exponent biased by 1023, 52 fraction
// bits).  Values lie in [0, 2^10): every nonzero one is a normal double.
__device__ __forceinline__ uint64_t fixed_to_bits(U128 x) {
  constexpr uint64_t kFrac = (1ull << 52) - 1;
  if (x.hi == 0 && x.lo < (1ull << 53)) {  // exact: at most 53 significant bits
    if (x.lo == 0) return 0;
    const int h = 63 - __clzll(x.lo);  // value = 1.f x 2^(h - 118)
    return (uint64_t(h - 118 + 1023) << 52) | ((x.lo << (52 - h)) & kFrac);
  }
  const int h = x.hi ? 127 - __clzll(x.hi) : 63 - __clzll(x.lo);  // top bit
  int sh = h - 52;                                                 // >= 1
  uint64_t mant, rem_hi_bit, rem_rest;
  // mant = x >> sh (53 bits)
  if (sh >= 64) {
    mant = x.hi >> (sh - 64);
  } else {
    mant = (x.lo >> sh) | (x.hi << (64 - sh));
  }
  // the bit just below the kept bits, and whether anything below it is set
  const int hb = sh - 1;
  if (hb >= 64) {
    rem_hi_bit = (x.hi >> (hb - 64)) & 1;
    rem_rest = (x.lo != 0) || ((hb - 64) > 0 && (x.hi & ((1ull << (hb - 64)) - 1)) != 0);
  } else {
    rem_hi_bit = (x.lo >> hb) & 1;
    rem_rest = hb > 0 && (x.lo & ((1ull << hb) - 1)) != 0;
  }
  if (rem_hi_bit && (rem_rest || (mant & 1))) mant += 1;
  if (mant >> 53) {  // rounded up into the next binade
    mant >>= 1;
    sh += 1;
  }
  // value = mant x 2^(sh - 118) = 1.f x 2^(52 + sh - 118)
  return (uint64_t(52 + sh - 118 + 1023) << 52) | (mant & kFrac);
}
__device__ __forceinline__ double from_fixed(U128 x) { return __longlong_as_double((long long)fixed_to_bits(x)); }

// Non-negative doubles compare like their bit patterns as unsigned integers.
__device__ __forceinline__ uint64_t dbits(double x) { return uint64_t(__double_as_longlong(x)); }

// Sources of p_i: amplitudes (p = re*re + im*im in FP64) or a probability vector.
template <typename R>
struct AmpSource {
  const R* a;
  __device__ __forceinline__ void load2(uint64_t i, double& p0, double& p1) const {
    Cplx<R> x0, x1;
    ld_amp2<R>(a, i, x0, x1);
    p0 = prob_fp64(x0.re, x0.im);
    p1 = prob_fp64(x1.re, x1.im);
  }
  __device__ __forceinline__ double load1(uint64_t i) const {
    Cplx<R> x = ld_amp<R>(a, i);
    return prob_fp64(x.re, x.im);
  }
};
struct ProbSource {
  const double* p;
  __device__ __forceinline__ void load2(uint64_t i, double& p0, double& p1) const {
    double2 v = reinterpret_cast<const double2*>(p)[i >> 1];
    p0 = v.x;
    p1 = v.y;
  }
  __device__ __forceinline__ double load1(uint64_t i) const { return p[i]; }
};

constexpr int kLeaf = 64;  // amplitudes per leaf: two per lane of one warp

// lane's two fixed-point values of leaf `leaf` (leaf size `ls` = min(64, N))
template <typename Src>
__device__ __forceinline__ void leaf_values(const Src& src, uint64_t leaf, int ls, int lane, U128& v0, U128& v1) {
  const uint64_t i = leaf * uint64_t(ls) + 2 * lane;
  v0 = U128{0, 0};
  v1 = U128{0, 0};
  if (2 * lane + 1 < ls) {
    double p0, p1;
    src.load2(i, p0, p1);
    v0 = to_fixed(p0);
    v1 = to_fixed(p1);
  } else if (2 * lane < ls) {
    v0 = to_fixed(src.load1(i));
  }
}

__device__ __forceinline__ U128 warp_sum128(U128 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    U128 t;
    t.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    t.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    v = add128(v, t);
  }
  return v;
}

// K1: leaf sums.  Full leaves (ls = 64): eight lanes per leaf, each converting and adding
// eight consecutive values, then three shuffle levels combine the eight lanes; a warp
// takes four neighbouring leaves at a time.  The integer sums are exact, so the leaf
// sum does not depend on this grouping.  A single short leaf (N < 64): the whole warp,
// two values per lane.
template <typename Src>
__global__ void __launch_bounds__(256) k_leaf_sums(Src src, uint64_t nleaf, int ls, U128* __restrict__ sums) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  if (ls < kLeaf) {
    for (uint64_t leaf = warp; leaf < nleaf; leaf += nwarps) {
      U128 v0, v1;
      leaf_values(src, leaf, ls, lane, v0, v1);
      U128 t = warp_sum128(add128(v0, v1));
      if (lane == 0) sums[leaf] = t;
    }
    return;
  }
  const int sub = lane >> 3, part = lane & 7;  // leaf within the warp's four, eighth of it
  for (uint64_t l0 = 4 * warp; l0 < nleaf; l0 += 4 * nwarps) {
    const uint64_t leaf = l0 + sub;
    U128 acc{0, 0};
    if (leaf < nleaf) {
      const uint64_t i = leaf * kLeaf + 8 * part;
      double p[8];
#pragma unroll
      for (int q = 0; q < 4; ++q) src.load2(i + 2 * q, p[2 * q], p[2 * q + 1]);
#pragma unroll
      for (int q = 0; q < 8; ++q) acc = add128(acc, to_fixed(p[q]));
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      U128 t;
      t.lo = __shfl_xor_sync(0xffffffffu, acc.lo, o);
      t.hi = __shfl_xor_sync(0xffffffffu, acc.hi, o);
      acc = add128(acc, t);
    }
    if (part == 0 && leaf < nleaf) sums[leaf] = acc;
  }
}

// K2a: per chunk of leaves, the chunk total
constexpr int kScanBlock = 256;
constexpr int kChunk = 2048;  // leaves per chunk

__device__ __forceinline__ U128 block_exclusive_scan128(U128 v, U128* total) {
  __shared__ U128 wsum[kScanBlock / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  U128 inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    U128 t = shfl_up128(inc, d);
    if (lane >= d) inc = add128(inc, t);
  }
  __syncthreads();
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  U128 off{0, 0}, tot{0, 0};
  for (int j = 0; j < kScanBlock / 32; ++j) {
    if (j < w) off = add128(off, wsum[j]);
    tot = add128(tot, wsum[j]);
  }
  *total = tot;
  U128 exc = shfl_up128(inc, 1);
  if (lane == 0) exc = U128{0, 0};
  return add128(off, exc);
}

__global__ void __launch_bounds__(kScanBlock) k_chunk_sums(const U128* __restrict__ sums, uint64_t nleaf,
                                                           U128* __restrict__ chunk) {
  const uint64_t base = uint64_t(blockIdx.x) * kChunk;
  U128 acc{0, 0};
  for (int j = threadIdx.x; j < kChunk; j += kScanBlock) {
    const uint64_t b = base + j;
    if (b < nleaf) acc = add128(acc, sums[b]);
  }
  U128 tot;
  block_exclusive_scan128(acc, &tot);
  if (threadIdx.x == 0) chunk[blockIdx.x] = tot;
}

// K2b: exclusive scan of the chunk totals (one block); chunk[nchunk] = grand total
__global__ void __launch_bounds__(kScanBlock) k_scan_chunks(U128* chunk, int nchunk) {
  const int per = (nchunk + kScanBlock - 1) / kScanBlock;
  const int beg = threadIdx.x * per;
  U128 acc{0, 0};
  for (int j = 0; j < per; ++j)
    if (beg + j < nchunk) acc = add128(acc, chunk[beg + j]);
  U128 tot;
  U128 off = block_exclusive_scan128(acc, &tot);
  __syncthreads();
  for (int j = 0; j < per; ++j)
    if (beg + j < nchunk) {
      U128 v = chunk[beg + j];
      chunk[beg + j] = off;
      off = add128(off, v);
    }
  if (threadIdx.x == 0) chunk[nchunk] = tot;
}

// K2c: leaf exclusive offsets (in place) and the rounded cdf at each leaf's end.  A block
// takes its chunk of kChunk leaves through shared memory: coalesced loads, each thread
// scans kChunk / kScanBlock consecutive leaves, coalesced stores.  One padding slot per
// thread run keeps both access patterns free of bank conflicts.
__global__ void __launch_bounds__(kScanBlock) k_leaf_offsets(U128* __restrict__ sums, uint64_t nleaf,
                                                             const U128* __restrict__ chunk,
                                                             double* __restrict__ leaf_end) {
  constexpr int per = kChunk / kScanBlock;
  __shared__ U128 st[kChunk + kChunk / per];
  auto slot = [](int i) { return i + i / per; };
  const uint64_t base = uint64_t(blockIdx.x) * kChunk;
  const int t = threadIdx.x;
#pragma unroll
  for (int k = 0; k < per; ++k) {
    const int i = t + k * kScanBlock;
    st[slot(i)] = base + i < nleaf ? sums[base + i] : U128{0, 0};
  }
  __syncthreads();
  U128 v[per];
  U128 acc{0, 0};
#pragma unroll
  for (int j = 0; j < per; ++j) {
    v[j] = st[slot(t * per + j)];
    acc = add128(acc, v[j]);
  }
  U128 tot;
  U128 off = add128(block_exclusive_scan128(acc, &tot), chunk[blockIdx.x]);
  double e[per];
#pragma unroll
  for (int j = 0; j < per; ++j) {
    const U128 o = off;
    off = add128(off, v[j]);
    e[j] = from_fixed(off);
    v[j] = o;
  }
  __syncthreads();  // every thread has read its run
#pragma unroll
  for (int j = 0; j < per; ++j) st[slot(t * per + j)] = v[j];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < per; ++k) {
    const int i = t + k * kScanBlock;
    if (base + i < nleaf) sums[base + i] = st[slot(i)];
  }
  __syncthreads();
  double* sd = reinterpret_cast<double*>(st);
#pragma unroll
  for (int j = 0; j < per; ++j) sd[slot(t * per + j)] = e[j];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < per; ++k) {
    const int i = t + k * kScanBlock;
    if (base + i < nleaf) leaf_end[base + i] = sd[slot(i)];
  }
}

// K3: two shots per warp, one per half-warp of 16 lanes, so that every warp instruction
// serves two shots.  Comparisons of non-negative doubles are done on their bit patterns
// (integer pipe).  The search starts in a table of kPivots leaf ends staged in shared
// memory per block, then continues in global memory; then each lane converts four of
// the leaf's values and the half-warp scans their 128-bit sums.
constexpr int kPivots = 4096;

template <typename Src>
__global__ void __launch_bounds__(256) k_draw(Src src, uint64_t nleaf, int ls, const U128* __restrict__ leaf_off,
                                              const double* __restrict__ leaf_end, const double* __restrict__ u,
                                              int64_t shots, uint64_t* __restrict__ out) {
  constexpr unsigned kFull = 0xffffffffu;
  __shared__ uint64_t piv[kPivots];
  const int lane = threadIdx.x & 31, hl = lane & 15, half = lane >> 4;
  const uint64_t warp = (blockIdx.x * uint64_t(blockDim.x) + threadIdx.x) >> 5;
  const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  const uint64_t Tb = dbits(leaf_end[nleaf - 1]);
  const double T = leaf_end[nleaf - 1];
  // pivot k = end of leaf min((k+1) seg - 1, nleaf - 1): the last pivot is the last leaf
  const uint64_t seg = (nleaf + kPivots - 1) / kPivots;
  for (int k = threadIdx.x; k < kPivots; k += blockDim.x) {
    uint64_t e = (uint64_t(k) + 1) * seg - 1;
    if (e > nleaf - 1) e = nleaf - 1;
    piv[k] = dbits(leaf_end[e]);
  }
  __syncthreads();
  for (uint64_t s0 = 2 * warp; s0 < uint64_t(shots); s0 += 2 * nwarps) {
    const uint64_t s = s0 + half;
    const bool active = s < uint64_t(shots);  // an idle half searches for t = 0, writes nothing
    const uint64_t tb = active ? dbits(u[s] * T) & 0x7FFFFFFFFFFFFFFFull : 0;  // -0 reads as +0
    const bool below = tb < Tb;
    // the test on a leaf end (false, then true, along the leaves; true at the last)
    auto pass_test = [&](uint64_t cb) { return below ? (tb < cb) : (cb >= Tb); };
    // 16-ary search: the answer stays in [lo, hi]; each round the 16 lanes of a half
    // probe the ends of 16 equal parts of it and the first part whose end passes is
    // kept.  Both halves step together (every lane takes part in the shuffles); a half
    // whose interval is a single leaf keeps it.
    auto narrow = [&](uint64_t& lo, uint64_t& hi, auto load) {
      while (__any_sync(kFull, lo < hi)) {
        const bool open = lo < hi;
        const uint64_t step = open ? (hi - lo + 16) / 16 : 1;  // ceil((hi - lo + 1) / 16)
        uint64_t pos = lo + (uint64_t(hl) + 1) * step - 1;
        if (pos > hi) pos = hi;
        const unsigned pass = (__ballot_sync(kFull, pass_test(load(pos))) >> (16 * half)) & 0xFFFFu;
        const int k = pass ? __ffs(pass) - 1 : 15;  // lane 15 of a half probes hi, which passes
        const uint64_t new_hi = __shfl_sync(kFull, pos, 16 * half + k);
        const uint64_t prev = __shfl_sync(kFull, pos, 16 * half + (k > 0 ? k - 1 : 0));
        if (open) {
          lo = k > 0 ? prev + 1 : lo;
          hi = new_hi;
        }
      }
    };
    uint64_t plo = 0, phi = kPivots - 1;
    narrow(plo, phi, [&](uint64_t i) { return piv[i]; });
    uint64_t lo = plo * seg, hi = (plo + 1) * seg - 1;
    if (hi > nleaf - 1) hi = nleaf - 1;
    narrow(lo, hi, [&](uint64_t i) { return dbits(leaf_end[i]); });
    const uint64_t leaf = lo;
    // this lane's four values (elements e0 .. e0 + 3 of the leaf) and their prefix sums
    const int e0 = 4 * hl;
    U128 c[4];
    const uint64_t i0 = leaf * uint64_t(ls) + e0;
    if (e0 + 3 < ls) {
      double p0, p1, p2, p3;
      src.load2(i0, p0, p1);
      src.load2(i0 + 2, p2, p3);
      c[0] = to_fixed(p0);
      c[1] = to_fixed(p1);
      c[2] = to_fixed(p2);
      c[3] = to_fixed(p3);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) c[q] = e0 + q < ls ? to_fixed(src.load1(i0 + q)) : U128{0, 0};
    }
    c[1] = add128(c[1], c[0]);
    c[2] = add128(c[2], c[1]);
    c[3] = add128(c[3], c[2]);
    // inclusive scan of the lane totals over the half-warp, then the exclusive offset
    U128 inc = c[3];
#pragma unroll
    for (int d = 1; d < 16; d <<= 1) {
      U128 x;
      x.lo = __shfl_up_sync(kFull, inc.lo, d, 16);
      x.hi = __shfl_up_sync(kFull, inc.hi, d, 16);
      if (hl >= d) inc = add128(inc, x);
    }
    U128 exc;
    exc.lo = __shfl_up_sync(kFull, inc.lo, 1, 16);
    exc.hi = __shfl_up_sync(kFull, inc.hi, 1, 16);
    if (hl == 0) exc = U128{0, 0};
    const U128 off = add128(leaf_off[leaf], exc);
    bool hit[4];
    if (below) {
      // RN64(c) > t  <=>  c lies above the midpoint between t and the next double up,
      // or on it when t's last significand bit is 1 (the tie goes to the even
      // neighbour): one 128-bit comparison with a threshold formed once per shot
      const int E = int((tb >> 52) & 0x7FF);
      const uint64_t mt = (tb & ((1ull << 52) - 1)) | (E ? (1ull << 52) : 0ull);
      const int e = E ? E : 1;                  // t = mt 2^(e-1075); midpoint (2 mt + 1) 2^(e-1076)
      const uint64_t odd2 = 2 * mt + 1;         // < 2^54
      const int sh = e - 958;                   // the midpoint in units of 2^-118: odd2 2^sh
      U128 M;
      bool exact;
      if (sh >= 0) {
        M.lo = sh >= 64 ? 0 : odd2 << sh;
        M.hi = sh == 0 ? 0 : sh >= 64 ? odd2 << (sh - 64) : odd2 >> (64 - sh);
        exact = true;
      } else {
        M.lo = -sh >= 64 ? 0 : odd2 >> (-sh);  // the floor; odd2 is odd, so never exact
        M.hi = 0;
        exact = false;
      }
      const bool tie_up = exact && (mt & 1);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const U128 cq = add128(off, c[q]);  // cdf of element e0 + q
        hit[q] = e0 + q < ls && (cq.hi > M.hi || (cq.hi == M.hi && (cq.lo > M.lo || (tie_up && cq.lo == M.lo))));
      }
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) hit[q] = e0 + q < ls && pass_test(fixed_to_bits(add128(off, c[q])));
    }
    const bool any = hit[0] || hit[1] || hit[2] || hit[3];
    const unsigned bal = (__ballot_sync(kFull, any) >> (16 * half)) & 0xFFFFu;
    const int first = __ffs(bal) - 1;  // leaf_end[leaf] passes, so some lane of an active half hits
    if (active && hl == first)
      out[s] = leaf * uint64_t(ls) + e0 + (hit[0] ? 0 : hit[1] ? 1 : hit[2] ? 2 : 3);
  }
}

template <typename Src>
static qc_status sample_impl(qc_state* s, uint64_t N, const Src& src, const double* u, int64_t shots,
                             uint64_t* out) {
  const int ls = int(N < uint64_t(kLeaf) ? N : uint64_t(kLeaf));
  const uint64_t nleaf = N / ls;
  const uint64_t nchunk = (nleaf + kChunk - 1) / kChunk;
  const size_t sums_b = ((nleaf * sizeof(U128)) + 255) & ~size_t(255);
  const size_t chunk_b = (((nchunk + 1) * sizeof(U128)) + 255) & ~size_t(255);
  const size_t end_b = ((nleaf * sizeof(double)) + 255) & ~size_t(255);
  void* scr = nullptr;
  if (qc_status st = state_scratch(s, sums_b + chunk_b + end_b, &scr)) return st;
  U128* sums = reinterpret_cast<U128*>(scr);
  U128* chunk = reinterpret_cast<U128*>(reinterpret_cast<char*>(scr) + sums_b);
  double* leaf_end = reinterpret_cast<double*>(reinterpret_cast<char*>(scr) + sums_b + chunk_b);
  const unsigned g1 = stream_grid(ls < kLeaf ? nleaf * 32 : nleaf * 8, 256, 8);
  QC_COUNT(), k_leaf_sums<Src><<<g1, 256, 0, s->stream>>>(src, nleaf, ls, sums);
  QC_COUNT(), k_chunk_sums<<<unsigned(nchunk), kScanBlock, 0, s->stream>>>(sums, nleaf, chunk);
  QC_COUNT(), k_scan_chunks<<<1, kScanBlock, 0, s->stream>>>(chunk, int(nchunk));
  QC_COUNT(), k_leaf_offsets<<<unsigned(nchunk), kScanBlock, 0, s->stream>>>(sums, nleaf, chunk, leaf_end);
  if (shots > 0) {
    const unsigned g3 = stream_grid(uint64_t(shots) * 16, 256, 8);
    QC_COUNT(), k_draw<Src><<<g3, 256, 0, s->stream>>>(src, nleaf, ls, sums, leaf_end, u, shots, out);
  }
  return check_launch("sampling");
}

}  // namespace qcgb

using namespace qcgb;

extern "C" {

static qc_status outcome_sums(qc_state* s, int q, double* P0, double* P1) {
  const uint64_t N = state_len(s);
  const uint64_t m = uint64_t(1) << (s->n - 1 - q);
  const unsigned g = stream_grid(N / 2 ? N / 2 : 1, 256, 8);
  void* scr = nullptr;
  if (qc_status st = state_scratch(s, sizeof(double) * (2 * g + 2), &scr)) return st;
  double* part = reinterpret_cast<double*>(scr);
  if (!s->host_buf) {
    if (qc_status st = check_cuda(cudaMallocHost(&s->host_buf, 4 * sizeof(double)), "pinned buffer")) return st;
  }
  if (s->dtype == QC_C64)
    QC_COUNT(), k_outcome_partials<float><<<g, 256, 0, s->stream>>>(reinterpret_cast<const float*>(s->amps), N, m, part);
  else
    QC_COUNT(), k_outcome_partials<double><<<g, 256, 0, s->stream>>>(reinterpret_cast<const double*>(s->amps), N, m, part);
  QC_COUNT(), k_sum2<<<1, 1024, 0, s->stream>>>(part, int(g), part + 2 * g);
  if (qc_status st = check_launch("outcome probabilities")) return st;
  if (qc_status st = check_cuda(cudaMemcpyAsync(s->host_buf, part + 2 * g, 2 * sizeof(double),
                                                cudaMemcpyDeviceToHost, s->stream),
                                "D2H"))
    return st;
  if (qc_status st = check_cuda(cudaStreamSynchronize(s->stream), "outcome probabilities")) return st;
  *P0 = s->host_buf[0];
  *P1 = s->host_buf[1];
  return QC_OK;
}

static qc_status check_q(const qc_state* s, int q) {
  if (!s || !s->amps) {
    set_error("invalid state handle");
    return QC_ERR_INVALID_ARG;
  }
  if (q < 0 || q >= s->n) {
    set_error("qubit %d out of range", q);
    return QC_ERR_INVALID_ARG;
  }
  return QC_OK;
}

static qc_status do_collapse(qc_state* s, int q, int outcome, double P) {
  const uint64_t N = state_len(s);
  const uint64_t m = uint64_t(1) << (s->n - 1 - q);
  const double inv = 1.0 / sqrt(P);
  const unsigned g = stream_grid(N / 2, 256);
  if (s->dtype == QC_C64)
    QC_COUNT(), k_collapse<float><<<g, 256, 0, s->stream>>>(reinterpret_cast<float*>(s->amps), N, m, outcome, inv);
  else
    QC_COUNT(), k_collapse<double><<<g, 256, 0, s->stream>>>(reinterpret_cast<double*>(s->amps), N, m, outcome, inv);
  return check_launch("collapse");
}

qc_status qc_outcome_prob(const qc_state* cs, int q, int outcome, double* prob) {
  clear_error();
  qc_state* s = const_cast<qc_state*>(cs);
  if (qc_status st = check_q(s, q)) return st;
  if (!prob || (outcome != 0 && outcome != 1)) {
    set_error("qc_outcome_prob: invalid arguments");
    return QC_ERR_INVALID_ARG;
  }
  double P0, P1;
  if (qc_status st = outcome_sums(s, q, &P0, &P1)) return st;
  *prob = outcome ? P1 : P0;
  return QC_OK;
}

qc_status qc_measure(qc_state* s, int q, double u, int* outcome, double* prob) {
  clear_error();
  if (qc_status st = check_q(s, q)) return st;
  if (!outcome || !(u >= 0.0 && u < 1.0)) {
    set_error("qc_measure: u must be in [0, 1) and outcome non-null");
    return QC_ERR_INVALID_ARG;
  }
  double P0, P1;
  if (qc_status st = outcome_sums(s, q, &P0, &P1)) return st;
  const double T = P0 + P1;
  if (!(T > 0.0)) {
    set_error("qc_measure: state has zero norm");
    return QC_ERR_ZERO_PROB;
  }
  const int o = (u * T >= P0) ? 1 : 0;
  const double P = o ? P1 : P0;
  if (qc_status st = do_collapse(s, q, o, P)) return st;
  *outcome = o;
  if (prob) *prob = P / T;
  return QC_OK;
}

qc_status qc_collapse(qc_state* s, int q, int outcome, double* prob) {
  clear_error();
  if (qc_status st = check_q(s, q)) return st;
  if (outcome != 0 && outcome != 1) {
    set_error("qc_collapse: outcome must be 0 or 1");
    return QC_ERR_INVALID_ARG;
  }
  double P0, P1;
  if (qc_status st = outcome_sums(s, q, &P0, &P1)) return st;
  const double T = P0 + P1;
  const double P = outcome ? P1 : P0;
  const double thr = s->dtype == QC_C64 ? 1e-6 : 1e-12;
  if (!(T > 0.0) || P / T <= thr) {
    set_error("qc_collapse: outcome %d has probability %.3g", outcome, T > 0 ? P / T : 0.0);
    return QC_ERR_ZERO_PROB;
  }
  if (qc_status st = do_collapse(s, q, outcome, P)) return st;
  if (prob) *prob = P / T;
  return check_cuda(cudaStreamSynchronize(s->stream), "qc_collapse");
}

qc_status qc_collapse_norm(qc_state* s, int q, int outcome, double p) {
  clear_error();
  if (!s || !s->amps || q < -1 || q >= s->n || (outcome != 0 && outcome != 1) || !(p >= 0.0)) {
    set_error("qc_collapse_norm: invalid arguments");
    return QC_ERR_INVALID_ARG;
  }
  const uint64_t N = state_len(s);
  // q = -1: no qubit is measured (mask 0 keeps every amplitude); p = 0 zeroes them
  const uint64_t m = q < 0 ? 0 : uint64_t(1) << (s->n - 1 - q);
  const double inv = p > 0.0 ? 1.0 / sqrt(p) : 0.0;
  const unsigned g = stream_grid(N / 2, 256);
  if (s->dtype == QC_C64)
    QC_COUNT(), k_collapse<float><<<g, 256, 0, s->stream>>>(reinterpret_cast<float*>(s->amps), N, m, q < 0 ? 0 : outcome,
                                                           inv);
  else
    QC_COUNT(), k_collapse<double><<<g, 256, 0, s->stream>>>(reinterpret_cast<double*>(s->amps), N, m,
                                                            q < 0 ? 0 : outcome, inv);
  return check_launch("qc_collapse_norm");
}

qc_status qc_probs(const qc_state* cs, double* dev_out) {
  clear_error();
  qc_state* s = const_cast<qc_state*>(cs);
  if (!s || !s->amps || !dev_out || (reinterpret_cast<uintptr_t>(dev_out) & 15)) {
    set_error("qc_probs: invalid arguments (output must be 16-byte aligned device memory)");
    return QC_ERR_INVALID_ARG;
  }
  const uint64_t N = state_len(s);
  const unsigned g = stream_grid(N / 2 ? N / 2 : 1, 256);
  if (s->dtype == QC_C64)
    QC_COUNT(), k_probs<float><<<g, 256, 0, s->stream>>>(reinterpret_cast<const float*>(s->amps), N, dev_out);
  else
    QC_COUNT(), k_probs<double><<<g, 256, 0, s->stream>>>(reinterpret_cast<const double*>(s->amps), N, dev_out);
  return check_launch("qc_probs");
}

qc_status qc_sample(const qc_state* cs, const double* dev_u, int64_t shots, uint64_t* dev_out) {
  clear_error();
  qc_state* s = const_cast<qc_state*>(cs);
  if (!s || !s->amps || shots < 0 || (shots > 0 && (!dev_u || !dev_out))) {
    set_error("qc_sample: invalid arguments");
    return QC_ERR_INVALID_ARG;
  }
  const uint64_t N = state_len(s);
  if (s->dtype == QC_C64)
    return sample_impl(s, N, AmpSource<float>{reinterpret_cast<const float*>(s->amps)}, dev_u, shots, dev_out);
  return sample_impl(s, N, AmpSource<double>{reinterpret_cast<const double*>(s->amps)}, dev_u, shots, dev_out);
}

// Sampling from a caller-supplied probability vector (device, N = 2^n doubles, 16-byte
// aligned, nonnegative, sum below 2^10), with the same rule as qc_sample.  `s`
// provides the stream and the scratch; its amplitudes are not read.
qc_status qc_sample_probs(qc_state* s, const double* dev_p, int n, const double* dev_u, int64_t shots,
                          uint64_t* dev_out) {
  clear_error();
  if (!s || !dev_p || n < 1 || n > 34 || shots < 0 || (shots > 0 && (!dev_u || !dev_out)) ||
      (reinterpret_cast<uintptr_t>(dev_p) & 15)) {
    set_error("qc_sample_probs: invalid arguments");
    return QC_ERR_INVALID_ARG;
  }
  return sample_impl(s, uint64_t(1) << n, ProbSource{dev_p}, dev_u, shots, dev_out);
}

}  // extern "C"
