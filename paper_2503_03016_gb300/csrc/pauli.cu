// Pauli-string expectations <psi| P |psi> (the expectations behind the density-matrix
// estimate of QCLAB Sec. 5.2, and the Hamiltonians of the gradient workloads).
//
// With Y = i X Z per qubit, a string with X-or-Y bits x, Z-or-Y bits z and nY Y's is
// P = i^nY X^x Z^z, so P|j> = i^nY (-1)^popc(j&z) |j^x> and
//   <psi|P|psi> = sum_j conj(psi_{j^x}) psi_j i^nY (-1)^popc(j&z).
// Terms that share x are evaluated in one pass.  For x = 0 the summand is
// |psi_j|^2 (-1)^popc(j&z).  For x != 0 the pass visits each pair (j, j^x) once (j
// with the lowest bit of x clear); with w = conj(psi_{j^x}) psi_j the pair contributes
// 2 (-1)^popc(j&z) * {Re w, -Im w, -Re w, Im w}[nY mod 4].
// Accumulation: complex64 states accumulate up to 16 terms per thread in FP32 before
// each FP64 add; complex128 accumulates in FP64 throughout; the cross-thread and
// cross-block reductions are FP64 in a fixed order.
#include <string.h>

#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "dfloat.cuh"
#include "kernels.cuh"

namespace qcgb {

constexpr int kMaxTermsPerPass = 16;

struct PauliGroup {
  uint64_t xmask;
  int hbit;  // lowest set bit of xmask (-1 when xmask == 0)
  int nt;
  uint64_t z[kMaxTermsPerPass];
  int mode[kMaxTermsPerPass];  // nY mod 4
  int slot[kMaxTermsPerPass];  // output position of each term
};

template <typename R>
__global__ void __launch_bounds__(256) k_pauli(const R* __restrict__ a, uint64_t N, PauliGroup g,
                                               double* __restrict__ partials) {
  using Acc = R;  // per-thread short-run accumulator
  double acc[kMaxTermsPerPass];
  Acc run[kMaxTermsPerPass];
#pragma unroll
  for (int t = 0; t < kMaxTermsPerPass; ++t) {
    acc[t] = 0.0;
    run[t] = Acc(0);
  }
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  int cnt = 0;
  if (g.hbit < 0) {
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < N; i += stride) {
      const Cplx<R> v = ld_amp<R>(a, i);
      const R p = v.re * v.re + v.im * v.im;
#pragma unroll
      for (int t = 0; t < kMaxTermsPerPass; ++t)
        if (t < g.nt) run[t] += (__popcll(i & g.z[t]) & 1) ? -p : p;
      if (++cnt == 16) {
#pragma unroll
        for (int t = 0; t < kMaxTermsPerPass; ++t) {
          acc[t] += double(run[t]);
          run[t] = Acc(0);
        }
        cnt = 0;
      }
    }
  } else {
    const uint64_t lo = (uint64_t(1) << g.hbit) - 1;
    for (uint64_t it = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; it < N / 2; it += stride) {
      const uint64_t j = ((it & ~lo) << 1) | (it & lo);
      const Cplx<R> x = ld_amp<R>(a, j), y = ld_amp<R>(a, j ^ g.xmask);
      // w = conj(y) * x
      const R wr = y.re * x.re + y.im * x.im;
      const R wi = y.re * x.im - y.im * x.re;
#pragma unroll
      for (int t = 0; t < kMaxTermsPerPass; ++t) {
        if (t < g.nt) {
          const int m = g.mode[t];
          R v = (m & 1) ? wi : wr;
          if (m == 1 || m == 2) v = -v;
          run[t] += (__popcll(j & g.z[t]) & 1) ? -v : v;
        }
      }
      if (++cnt == 16) {
#pragma unroll
        for (int t = 0; t < kMaxTermsPerPass; ++t) {
          acc[t] += 2.0 * double(run[t]);
          run[t] = Acc(0);
        }
        cnt = 0;
      }
    }
  }
  const double scale = g.hbit < 0 ? 1.0 : 2.0;
#pragma unroll
  for (int t = 0; t < kMaxTermsPerPass; ++t) {
    double v = acc[t] + scale * double(run[t]);
    if (t < g.nt) {
      v = block_sum(v);
      if (threadIdx.x == 0) partials[size_t(blockIdx.x) * kMaxTermsPerPass + t] = v;
    }
  }
}

// Z-only strings (x = 0), up to 32 per pass: <Z_z> = sum_i p_i (-1)^popc(i & z).  With
// h = n - 5, index i = (l << h) | c splits into the 5 top bits l (qubits 0..4) and a
// chunk number c.  A thread takes chunk c, the 32 amplitudes (l << h) | c, forms the
// Walsh-Hadamard transform S(w) = sum_l p_l (-1)^popc(l & w) of their probabilities once
// (in registers, then shared memory), and adds (-1)^popc(c & z) * S(z >> h) to every
// term: per-term work is per chunk, not per amplitude.  Neighbouring threads take
// neighbouring chunks, so each of a warp's 32 loads is one contiguous run of amplitudes.
// complex64 states accumulate per thread in FP32 (the per-amplitude values are FP32
// products already), complex128 in FP64; cross-thread and cross-block sums are FP64 in
// a fixed order.
//
// Signs: there are 2^K virtual threads (K = kbits_base; one resident wave of blocks
// loops over them) and virtual thread g takes the chunks g + k 2^K, k = 0 ..
// 2^kbits - 1, so (-1)^popc(c & z) splits into a per-thread sign (from g) and a sign
// from k shared by all threads.  k runs in Gray-code order: the step from the j-th to
// the (j+1)-th k flips bit ctz(j+1) of k, which toggles the signs of the terms whose z
// has the matching index bit (flip[b], from the host).
constexpr int kMaxZTerms = 32;
constexpr int kZBlock = 128;
constexpr int kZMaxThreadBits = 20;  // at most 2^20 virtual threads (8192 virtual blocks)
struct ZGroup {
  int nt;
  int hshift;         // h = n - 5: log2 of the chunk count, shift of the top 5 bits
  int kbits_base;     // K: log2 of the number of virtual threads
  int kbits;          // chunks per virtual thread = 2^kbits
  uint32_t flip[16];  // bit t: term t's z has index bit K + b
  uint64_t z[kMaxZTerms];
  int slot[kMaxZTerms];
};

template <typename R>
__global__ void __launch_bounds__(kZBlock) k_pauli_z(const R* __restrict__ amps, uint64_t N, ZGroup g,
                                                     double* __restrict__ partials) {
  __shared__ R S[32][kZBlock];
  R acc[kMaxZTerms];
#pragma unroll
  for (int t = 0; t < kMaxZTerms; ++t) acc[t] = R(0);
  const int h = g.hshift;
  const uint64_t nchunk = N >> 5;
  // 2^K virtual threads in virtual blocks of kZBlock, spread over the resident grid
  const uint64_t nvb = uint64_t(1) << (g.kbits_base - 7);
  for (uint64_t vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
    const uint64_t gt = vb * kZBlock + threadIdx.x;
    if (gt >= nchunk) continue;
    // this thread's signs (bit t: term t's sign for chunk gt, i.e. k = 0)
    uint32_t sign = 0;
#pragma unroll
    for (int t = 0; t < kMaxZTerms; ++t)
      if (t < g.nt) sign |= uint32_t(__popcll(gt & g.z[t]) & 1) << t;
    const uint64_t nk = uint64_t(1) << g.kbits;
    for (uint64_t j = 0; j < nk; ++j) {
      const uint64_t k = j ^ (j >> 1);  // Gray code
      const uint64_t c = gt + (k << g.kbits_base);
      R w[32];
#pragma unroll
      for (int l = 0; l < 32; ++l) {
        const Cplx<R> x = ld_amp<R>(amps, (uint64_t(l) << h) | c);
        w[l] = x.re * x.re + x.im * x.im;
      }
      // in-place Walsh-Hadamard transform over the 5 top bits
#pragma unroll
      for (int hb = 1; hb < 32; hb <<= 1)
#pragma unroll
        for (int l = 0; l < 32; ++l)
          if (!(l & hb)) {
            const R a = w[l], b = w[l | hb];
            w[l] = a + b;
            w[l | hb] = a - b;
          }
#pragma unroll
      for (int l = 0; l < 32; ++l) S[l][threadIdx.x] = w[l];
      // S is private to this thread's column: no barrier needed
#pragma unroll
      for (int t = 0; t < kMaxZTerms; ++t) {
        if (t >= g.nt) break;
        const R v = S[g.z[t] >> h][threadIdx.x];
        acc[t] += ((sign >> t) & 1u) ? -v : v;
      }
      if (j + 1 < nk) sign ^= g.flip[__ffsll((long long)(j + 1)) - 1];
    }
  }
#pragma unroll
  for (int t = 0; t < kMaxZTerms; ++t) {
    if (t >= g.nt) break;
    const double v = block_sum(double(acc[t]));
    if (threadIdx.x == 0) partials[size_t(blockIdx.x) * kMaxZTerms + t] = v;
  }
}

// The same Z strings for complex128 states of 2^kDfMinQubits amplitudes or more in
// double-float arithmetic: p_l = re^2 + im^2 from the FP32 pairs of the amplitude (the
// squares of the hi parts exact by TwoProduct, the cross terms 2 hi lo rounded, lo^2
// left out), the Walsh-Hadamard transform and the per-thread term sums as (hi, lo) pairs
// with TwoSum; block and cross-block sums in FP64 as for the other kernels.
__global__ void __launch_bounds__(kZBlock) k_pauli_z_df(const double* __restrict__ amps, uint64_t N, ZGroup g,
                                                        double* __restrict__ partials) {
  __shared__ float2 S[32][kZBlock];
  float2 acc[kMaxZTerms];
#pragma unroll
  for (int t = 0; t < kMaxZTerms; ++t) acc[t] = make_float2(0.0f, 0.0f);
  const int h = g.hshift;
  const uint64_t nchunk = N >> 5;
  const uint64_t nvb = uint64_t(1) << (g.kbits_base - 7);
  for (uint64_t vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
    const uint64_t gt = vb * kZBlock + threadIdx.x;
    if (gt >= nchunk) continue;
    uint32_t sign = 0;
#pragma unroll
    for (int t = 0; t < kMaxZTerms; ++t)
      if (t < g.nt) sign |= uint32_t(__popcll(gt & g.z[t]) & 1) << t;
    const uint64_t nk = uint64_t(1) << g.kbits;
    for (uint64_t j = 0; j < nk; ++j) {
      const uint64_t k = j ^ (j >> 1);  // Gray code
      const uint64_t c = gt + (k << g.kbits_base);
      float2 w[32];
#pragma unroll
      for (int l = 0; l < 32; ++l) {
        const Cplx<double> x = ld_amp<double>(amps, (uint64_t(l) << h) | c);
        float rh, rl, ih, il;
        df_split(x.re, rh, rl);
        df_split(x.im, ih, il);
        const float pr = __fmul_rn(rh, rh), pi = __fmul_rn(ih, ih);
        float er = __fmaf_rn(rh, rh, -pr), ei = __fmaf_rn(ih, ih, -pi);
        er = __fmaf_rn(__fadd_rn(rh, rh), rl, er);
        ei = __fmaf_rn(__fadd_rn(ih, ih), il, ei);
        w[l] = dfs_acc(make_float2(pr, er), make_float2(pi, ei));
      }
      // in-place Walsh-Hadamard transform over the 5 top bits
#pragma unroll
      for (int hb = 1; hb < 32; hb <<= 1)
#pragma unroll
        for (int l = 0; l < 32; ++l)
          if (!(l & hb)) {
            const float2 a = w[l], b = w[l | hb];
            w[l] = dfs_acc(a, b);
            w[l | hb] = dfs_acc(a, make_float2(-b.x, -b.y));
          }
#pragma unroll
      for (int l = 0; l < 32; ++l) S[l][threadIdx.x] = dfs_renorm(w[l]);
#pragma unroll
      for (int t = 0; t < kMaxZTerms; ++t) {
        if (t >= g.nt) break;
        const float2 v = S[g.z[t] >> h][threadIdx.x];
        acc[t] = dfs_acc(acc[t], ((sign >> t) & 1u) ? make_float2(-v.x, -v.y) : v);
      }
      if (j + 1 < nk) sign ^= g.flip[__ffsll((long long)(j + 1)) - 1];
    }
  }
#pragma unroll
  for (int t = 0; t < kMaxZTerms; ++t) {
    if (t >= g.nt) break;
    const double v = block_sum(double(acc[t].x) + double(acc[t].y));
    if (threadIdx.x == 0) partials[size_t(blockIdx.x) * kMaxZTerms + t] = v;
  }
}

// Cross-block sums, one block per term (grid = number of terms): each block adds its
// term's block partials in a fixed order.
__global__ void __launch_bounds__(256) k_sum_zterms(const double* partials, int nblocks, ZGroup g, double* out) {
  const int t = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) acc += partials[size_t(i) * kMaxZTerms + t];
  acc = block_sum(acc);
  if (threadIdx.x == 0) out[g.slot[t]] = acc;
}

__global__ void __launch_bounds__(256) k_sum_terms(const double* partials, int nblocks, PauliGroup g, double* out) {
  const int t = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) acc += partials[size_t(i) * kMaxTermsPerPass + t];
  acc = block_sum(acc);
  if (threadIdx.x == 0) out[g.slot[t]] = acc;
}

struct ParsedTerm {
  uint64_t x, z;
  int ny;
};

qc_status parse_pauli(int n, const char* str, ParsedTerm* out) {
  if (!str || int(strlen(str)) != n) {
    set_error("Pauli string must have exactly n=%d characters", n);
    return QC_ERR_INVALID_ARG;
  }
  ParsedTerm t{0, 0, 0};
  for (int q = 0; q < n; ++q) {
    const uint64_t b = uint64_t(1) << (n - 1 - q);
    switch (str[q]) {
      case 'I': case 'i': break;
      case 'X': case 'x': t.x |= b; break;
      case 'Z': case 'z': t.z |= b; break;
      case 'Y': case 'y': t.x |= b; t.z |= b; t.ny++; break;
      default:
        set_error("invalid Pauli character '%c'", str[q]);
        return QC_ERR_INVALID_ARG;
    }
  }
  *out = t;
  return QC_OK;
}

// Resident k_pauli_z blocks per SM (1..32), queried once per (kernel, device): kind 0
// complex64, 1 complex128 in FP64, 2 complex128 in double-float.
static int z_blocks_per_sm(int kind, int device) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find({kind, device});
  if (it != cache.end()) return it->second;
  int per_sm = 0;
  if (kind == 0)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pauli_z<float>, kZBlock, 0);
  else if (kind == 1)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pauli_z<double>, kZBlock, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pauli_z_df, kZBlock, 0);
  per_sm = std::min(std::max(per_sm, 1), 32);
  cache[{kind, device}] = per_sm;
  return per_sm;
}

// Z-only strings z[0..nt) (N >= 64), values to vals[slot[j]]: passes of up to 32 terms,
// each a k_pauli_z launch (one resident wave of blocks looping over 2^K virtual threads
// that take 2^kbits chunks of 32 amplitudes each; at most max_blocks blocks, whose
// partials go to `part`) and a k_sum_zterms launch.
static void launch_z_strings(qc_state* s, const uint64_t* z, const int* slot, int nt, double* part,
                             size_t max_blocks, double* vals) {
  const uint64_t N = state_len(s);
  const int cbits = s->n - 5;  // log2 of the chunk count
  const int K = std::max(7, std::min(cbits, kZMaxThreadBits));
  const int per_sm = z_blocks_per_sm(s->dtype == QC_C64 ? 0 : s->n >= kDfMinQubits ? 2 : 1, s->device);
  uint64_t gz = std::min<uint64_t>(uint64_t(1) << (K - 7), uint64_t(per_sm) * device_sm_count());
  gz = std::max<uint64_t>(1, std::min<uint64_t>(gz, max_blocks));
  for (int beg = 0; beg < nt; beg += kMaxZTerms) {
    ZGroup zg{};
    zg.nt = std::min(kMaxZTerms, nt - beg);
    zg.hshift = cbits;
    zg.kbits_base = K;
    zg.kbits = std::max(0, cbits - K);
    for (int j = 0; j < zg.nt; ++j) {
      zg.z[j] = z[beg + j];
      zg.slot[j] = slot[beg + j];
      for (int b = 0; b < zg.kbits; ++b)
        if ((zg.z[j] >> (K + b)) & 1) zg.flip[b] |= 1u << j;
    }
    if (s->dtype == QC_C64)
      QC_COUNT(), k_pauli_z<float><<<unsigned(gz), kZBlock, 0, s->stream>>>(reinterpret_cast<const float*>(s->amps),
                                                                          N, zg, part);
    else if (s->n >= kDfMinQubits)
      QC_COUNT(), k_pauli_z_df<<<unsigned(gz), kZBlock, 0, s->stream>>>(reinterpret_cast<const double*>(s->amps), N,
                                                                       zg, part);
    else
      QC_COUNT(), k_pauli_z<double><<<unsigned(gz), kZBlock, 0, s->stream>>>(reinterpret_cast<const double*>(s->amps),
                                                                           N, zg, part);
    QC_COUNT(), k_sum_zterms<<<zg.nt, 256, 0, s->stream>>>(part, int(gz), zg, vals);
  }
}

// values[t] = <psi|P_t|psi> (no coefficients) into a device buffer of nterms doubles:
// `dev_vals`, or with dev_vals == nullptr the end of the state's scratch (returned in
// *vals_out; valid until the next call that uses the scratch).
qc_status expect_terms_device(qc_state* s, const ParsedTerm* terms, int nterms, double* dev_vals,
                              double** vals_out = nullptr) {
  const uint64_t N = state_len(s);
  std::map<uint64_t, std::vector<int>> groups;
  for (int t = 0; t < nterms; ++t) groups[terms[t].x].push_back(t);
  const int B = 256;
  const unsigned g = stream_grid(N, B, 8);
  // block partials: the X/Y-string kernels use g blocks, the Z-string kernel at most
  // one resident wave (below 32 blocks per SM)
  const size_t nblk = std::max<size_t>(g, size_t(32) * device_sm_count());
  void* scr = nullptr;
  if (qc_status st = state_scratch(s, sizeof(double) * (nblk * kMaxZTerms + size_t(nterms)) + 256, &scr))
    return st;
  double* part = reinterpret_cast<double*>(scr);
  if (!dev_vals) dev_vals = part + nblk * kMaxZTerms;
  if (vals_out) *vals_out = dev_vals;
  for (auto& kv : groups) {
    const std::vector<int>& idx = kv.second;
    if (kv.first == 0 && N >= 64) {  // Z-only strings
      std::vector<uint64_t> z(idx.size());
      for (size_t j = 0; j < idx.size(); ++j) z[j] = terms[idx[j]].z;
      launch_z_strings(s, z.data(), idx.data(), int(idx.size()), part, nblk, dev_vals);
      continue;
    }
    for (size_t beg = 0; beg < idx.size(); beg += kMaxTermsPerPass) {
      PauliGroup pg{};
      pg.xmask = kv.first;
      pg.hbit = kv.first ? __builtin_ctzll(kv.first) : -1;
      pg.nt = int(std::min<size_t>(kMaxTermsPerPass, idx.size() - beg));
      for (int j = 0; j < pg.nt; ++j) {
        pg.z[j] = terms[idx[beg + j]].z;
        pg.mode[j] = terms[idx[beg + j]].ny & 3;
        pg.slot[j] = idx[beg + j];
      }
      if (s->dtype == QC_C64)
        QC_COUNT(), k_pauli<float><<<g, B, 0, s->stream>>>(reinterpret_cast<const float*>(s->amps), N, pg, part);
      else
        QC_COUNT(), k_pauli<double><<<g, B, 0, s->stream>>>(reinterpret_cast<const double*>(s->amps), N, pg, part);
      QC_COUNT(), k_sum_terms<<<pg.nt, 256, 0, s->stream>>>(part, int(g), pg, dev_vals);
    }
  }
  return check_launch("Pauli expectation");
}

}  // namespace qcgb

using namespace qcgb;

extern "C" qc_status qc_expect_pauli(const qc_state* cs, const char* const* strings, const double* coeffs,
                                     int nterms, double* host_out) {
  clear_error();
  qc_state* s = const_cast<qc_state*>(cs);
  if (!s || !s->amps || nterms < 0 || (nterms > 0 && (!strings || !host_out))) {
    set_error("qc_expect_pauli: invalid arguments");
    return QC_ERR_INVALID_ARG;
  }
  if (nterms == 0) return QC_OK;
  std::vector<ParsedTerm> terms(nterms);
  for (int t = 0; t < nterms; ++t)
    if (qc_status st = parse_pauli(s->n, strings[t], &terms[t])) return st;
  double* dev = nullptr;  // values at the end of the state's scratch
  qc_status st = expect_terms_device(s, terms.data(), nterms, nullptr, &dev);
  std::vector<double> vals(nterms);
  if (st == QC_OK)
    st = check_cuda(cudaMemcpyAsync(vals.data(), dev, sizeof(double) * nterms, cudaMemcpyDeviceToHost, s->stream),
                    "D2H");
  if (st == QC_OK) st = check_cuda(cudaStreamSynchronize(s->stream), "qc_expect_pauli");
  if (st != QC_OK) return st;
  for (int t = 0; t < nterms; ++t) host_out[t] = vals[t] * (coeffs ? coeffs[t] : 1.0);
  return QC_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the expectation entry point.
//
// Some callers cannot allocate device memory at the time they need an expectation
// value: a process whose device memory is already reserved in full by another
// allocator (for example a framework's caching allocator sized to the whole GPU),
// or a service that must not risk an allocation failure, or the device-wide
// synchronisation cudaMalloc/cudaFree can cause, once it is running.  For them
// qc_expect_pauli_noalloc uses a fixed scratch array that lives in this library's
// device image instead of the state's lazily allocated scratch.
// ---------------------------------------------------------------------------
namespace qcgb {

constexpr int kNoAllocMaxBlocks = 1216;  // grid cap of the reduction (8 blocks per SM on 152 SMs)
constexpr int kNoAllocMaxTerms = 256;    // terms per call
constexpr size_t kNoAllocDoubles = size_t(kNoAllocMaxBlocks) * kMaxTermsPerPass + kNoAllocMaxTerms;

// 1216*16 + 256 doubles = 157,696 bytes, held by every device that loads the library
// until the process exits.  Shared by all calls: each call overwrites it.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

// Device address of g_noalloc_scratch on `device`, looked up on every call (the
// lookup allocates nothing; a cached address would go stale after a device reset).
static qc_status noalloc_scratch(int device, double** out) {
  int cur = -1;
  if (qc_status st = check_cuda(cudaGetDevice(&cur), "cudaGetDevice")) return st;
  if (cur != device)
    if (qc_status st = check_cuda(cudaSetDevice(device), "cudaSetDevice")) return st;
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (cur != device) cudaSetDevice(cur);
  if (qc_status st = check_cuda(e, "cudaGetSymbolAddress(noalloc scratch)")) return st;
  *out = static_cast<double*>(p);
  return QC_OK;
}

}  // namespace qcgb

extern "C" qc_status qc_expect_pauli_noalloc(const qc_state* cs, const char* const* strings, const double* coeffs,
                                             int nterms, double* host_out) {
  clear_error();
  qc_state* s = const_cast<qc_state*>(cs);
  if (!s || !s->amps || nterms < 0 || (nterms > 0 && (!strings || !host_out))) {
    set_error("qc_expect_pauli_noalloc: invalid arguments");
    return QC_ERR_INVALID_ARG;
  }
  if (nterms > kNoAllocMaxTerms) {
    set_error("qc_expect_pauli_noalloc: %d terms exceed the fixed scratch limit of %d terms per call", nterms,
              kNoAllocMaxTerms);
    return QC_ERR_INVALID_ARG;
  }
  if (nterms == 0) return QC_OK;
  ParsedTerm terms[kNoAllocMaxTerms];
  for (int t = 0; t < nterms; ++t)
    if (qc_status st = parse_pauli(s->n, strings[t], &terms[t])) return st;
  double* scratch = nullptr;
  if (qc_status st = noalloc_scratch(s->device, &scratch)) return st;
  double* part = scratch;                                              // blocks x 16
  double* vals = scratch + size_t(kNoAllocMaxBlocks) * kMaxTermsPerPass;  // nterms
  // group terms by X mask without heap use: order term indices by xmask
  int order[kNoAllocMaxTerms];
  for (int t = 0; t < nterms; ++t) order[t] = t;
  for (int i = 1; i < nterms; ++i) {
    const int v = order[i];
    int j = i - 1;
    while (j >= 0 && terms[order[j]].x > terms[v].x) {
      order[j + 1] = order[j];
      --j;
    }
    order[j + 1] = v;
  }
  const uint64_t N = state_len(s);
  const int B = 256;
  unsigned g = stream_grid(N, B, 8);
  if (g > unsigned(kNoAllocMaxBlocks)) g = kNoAllocMaxBlocks;
  int beg = 0;
  while (beg < nterms) {
    PauliGroup pg{};
    pg.xmask = terms[order[beg]].x;
    pg.hbit = pg.xmask ? __builtin_ctzll(pg.xmask) : -1;
    pg.nt = 0;
    while (beg + pg.nt < nterms && pg.nt < kMaxTermsPerPass && terms[order[beg + pg.nt]].x == pg.xmask) {
      const int t = order[beg + pg.nt];
      pg.z[pg.nt] = terms[t].z;
      pg.mode[pg.nt] = terms[t].ny & 3;
      pg.slot[pg.nt] = t;
      ++pg.nt;
    }
    if (pg.xmask == 0 && N >= 64) {
      // Z-only strings: all of them (they are contiguous in `order`) in the Z kernel,
      // its block partials within the same fixed scratch
      int nz = pg.nt;
      while (beg + nz < nterms && terms[order[beg + nz]].x == 0) ++nz;
      uint64_t z[kNoAllocMaxTerms];
      for (int j = 0; j < nz; ++j) z[j] = terms[order[beg + j]].z;
      launch_z_strings(s, z, order + beg, nz, part, size_t(kNoAllocMaxBlocks) * kMaxTermsPerPass / kMaxZTerms,
                       vals);
      beg += nz;
      continue;
    }
    if (s->dtype == QC_C64)
      QC_COUNT(), k_pauli<float><<<g, B, 0, s->stream>>>(reinterpret_cast<const float*>(s->amps), N, pg, part);
    else
      QC_COUNT(), k_pauli<double><<<g, B, 0, s->stream>>>(reinterpret_cast<const double*>(s->amps), N, pg, part);
    QC_COUNT(), k_sum_terms<<<pg.nt, 256, 0, s->stream>>>(part, int(g), pg, vals);
    beg += pg.nt;
  }
  if (qc_status st = check_launch("qc_expect_pauli_noalloc")) return st;
  double host_vals[kNoAllocMaxTerms];
  if (qc_status st = check_cuda(cudaMemcpyAsync(host_vals, vals, sizeof(double) * nterms, cudaMemcpyDeviceToHost,
                                                s->stream),
                                "D2H"))
    return st;
  if (qc_status st = check_cuda(cudaStreamSynchronize(s->stream), "qc_expect_pauli_noalloc")) return st;
  for (int t = 0; t < nterms; ++t) host_out[t] = host_vals[t] * (coeffs ? coeffs[t] : 1.0);
  return QC_OK;
}
