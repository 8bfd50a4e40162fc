// Subsystem readouts: the reduced state vector of the unmeasured qubits (QCLAB Sec. 5.1,
// reducedStatevector) and marginal outcome probabilities of a qubit subset (the
// distribution behind counts(shots) of Sec. 5.2 when only some qubits are measured).
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace qcgb {

struct GatherSpec {
  uint64_t fixed;      // index bits of the known qubits
  int nrest;
  int8_t rest[40];     // bit positions of the remaining qubits, ascending significance of r
};

// out[r] = amps[fixed | deposit(r, rest)]; r's bit k goes to bit rest[k]
template <typename R>
__global__ void k_gather(const R* __restrict__ amps, uint64_t M, GatherSpec g, R* __restrict__ out) {
  for (uint64_t r = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; r < M; r += uint64_t(gridDim.x) * blockDim.x) {
    uint64_t i = g.fixed;
    for (int k = 0; k < g.nrest; ++k)
      if ((r >> k) & 1) i |= uint64_t(1) << g.rest[k];
    st_amp<R>(out, r, ld_amp<R>(amps, i));
  }
}

// Marginal over m <= 12 qubits: per-block histograms of p_i (FP64) in shared memory,
// written per block; a second kernel adds the blocks in a fixed order.
struct MarginalSpec {
  int m;
  int8_t bit[12];  // index bit of marginal bit k (k = 0 is the least significant outcome bit)
};

template <typename R>
__global__ void __launch_bounds__(256) k_marginal_partials(const R* __restrict__ amps, uint64_t N, MarginalSpec s,
                                                           double* __restrict__ partials) {
  extern __shared__ double hist[];
  const int B = 1 << s.m;
  for (int i = threadIdx.x; i < B; i += blockDim.x) hist[i] = 0.0;
  __syncthreads();
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < N; i += uint64_t(gridDim.x) * blockDim.x) {
    const Cplx<R> v = ld_amp<R>(amps, i);
    const double p = prob_fp64(v.re, v.im);
    int x = 0;
    for (int k = 0; k < s.m; ++k) x |= int((i >> s.bit[k]) & 1) << k;
    atomicAdd(&hist[x], p);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < B; i += blockDim.x) partials[size_t(blockIdx.x) * B + i] = hist[i];
}

__global__ void k_marginal_sum(const double* __restrict__ partials, int nblocks, int B, double* __restrict__ out) {
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < B; x += gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int b = 0; b < nblocks; ++b) a += partials[size_t(b) * B + x];
    out[x] = a;
  }
}

}  // namespace qcgb

using namespace qcgb;

extern "C" qc_status qc_reduced_state(const qc_state* cs, const int* known, const int* bits, int m, void* dev_out) {
  clear_error();
  qc_state* s = const_cast<qc_state*>(cs);
  if (!s || !s->amps || m < 0 || m >= s->n || (m > 0 && (!known || !bits)) || !dev_out ||
      (reinterpret_cast<uintptr_t>(dev_out) & 15)) {
    set_error("qc_reduced_state: invalid arguments");
    return QC_ERR_INVALID_ARG;
  }
  GatherSpec g{};
  std::vector<bool> is_known(s->n, false);
  for (int j = 0; j < m; ++j) {
    if (known[j] < 0 || known[j] >= s->n || is_known[known[j]] || (bits[j] != 0 && bits[j] != 1)) {
      set_error("qc_reduced_state: bad known qubit or bit");
      return QC_ERR_INVALID_ARG;
    }
    is_known[known[j]] = true;
    if (bits[j]) g.fixed |= uint64_t(1) << (s->n - 1 - known[j]);
  }
  // remaining qubits keep their order: the last remaining qubit is the least significant
  for (int q = s->n - 1; q >= 0; --q)
    if (!is_known[q]) g.rest[g.nrest++] = int8_t(s->n - 1 - q);
  const uint64_t M = uint64_t(1) << g.nrest;
  const unsigned grid = stream_grid(M, 256);
  if (s->dtype == QC_C64)
    QC_COUNT(), k_gather<float><<<grid, 256, 0, s->stream>>>(reinterpret_cast<const float*>(s->amps), M, g,
                                                             reinterpret_cast<float*>(dev_out));
  else
    QC_COUNT(), k_gather<double><<<grid, 256, 0, s->stream>>>(reinterpret_cast<const double*>(s->amps), M, g,
                                                              reinterpret_cast<double*>(dev_out));
  return check_launch("qc_reduced_state");
}

extern "C" qc_status qc_marginal_probs(const qc_state* cs, const int* qubits, int m, double* dev_out) {
  clear_error();
  qc_state* s = const_cast<qc_state*>(cs);
  if (!s || !s->amps || m < 1 || m > 12 || m > s->n || !qubits || !dev_out) {
    set_error("qc_marginal_probs: invalid arguments (1 <= m <= 12)");
    return QC_ERR_INVALID_ARG;
  }
  MarginalSpec ms{};
  ms.m = m;
  std::vector<bool> seen(s->n, false);
  for (int j = 0; j < m; ++j) {
    if (qubits[j] < 0 || qubits[j] >= s->n || seen[qubits[j]]) {
      set_error("qc_marginal_probs: qubits must be distinct and in range");
      return QC_ERR_INVALID_ARG;
    }
    seen[qubits[j]] = true;
    // outcome index: qubits[0] is the most significant outcome bit
    ms.bit[m - 1 - j] = int8_t(s->n - 1 - qubits[j]);
  }
  const uint64_t N = state_len(s);
  const int B = 1 << m;
  const unsigned grid = stream_grid(N, 256, 2);
  void* scr = nullptr;
  if (qc_status st = state_scratch(s, sizeof(double) * size_t(grid) * B, &scr)) return st;
  double* part = reinterpret_cast<double*>(scr);
  const size_t smem = sizeof(double) * B;
  if (s->dtype == QC_C64)
    QC_COUNT(), k_marginal_partials<float><<<grid, 256, smem, s->stream>>>(reinterpret_cast<const float*>(s->amps),
                                                                            N, ms, part);
  else
    QC_COUNT(), k_marginal_partials<double><<<grid, 256, smem, s->stream>>>(reinterpret_cast<const double*>(s->amps),
                                                                             N, ms, part);
  QC_COUNT(), k_marginal_sum<<<(B + 255) / 256, 256, 0, s->stream>>>(part, int(grid), B, dev_out);
  return check_launch("qc_marginal_probs");
}
