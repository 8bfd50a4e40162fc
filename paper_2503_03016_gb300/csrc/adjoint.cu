// Adjoint (reverse-sweep) gradient of E(theta) = <psi(theta)| H |psi(theta)>.
//
// The circuit is the paper's gate sequence (Sec. 3.2) with rotation gates
// U_l = exp(-i theta_l G_l / 2), G in {X, Y, Z}.  With psi_l the state after gate l and
// lambda_l = U_{l+1}^dag ... U_L^dag H psi_L, dE/dtheta_l = 2 Re <lambda_l| dpsi_l/dtheta_l>
// = 2 Re <lambda_l| (-i G_l / 2) |psi_l> = Im <lambda_l| G_l |psi_l>.
// Sweep: psi = U_L ... U_1 |0>, lambda = H psi, E = Re <psi|lambda>; then for l = L..1:
// g_l = Im <lambda|G_l|psi>, psi <- U_l^dag psi, lambda <- U_l^dag lambda.  For a
// rotation gate the inner product and both un-applications are one pass over the
// pairs of the target bit (read 2 states, write 2 states); block partial sums are
// FP64 and reduced in a fixed order.
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <vector>

#include "adjoint_tiles.cuh"
#include "circuit.cuh"
#include "common.cuh"
#include "kernels.cuh"
#include "tiles_df.cuh"

namespace qcgb {

struct ParsedTermA {
  uint64_t x, z;
  int ny;
};

qc_status parse_pauli_a(int n, const char* str, ParsedTermA* out) {
  if (!str || int(strlen(str)) != n) {
    set_error("Pauli string must have exactly n=%d characters", n);
    return QC_ERR_INVALID_ARG;
  }
  ParsedTermA t{0, 0, 0};
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

constexpr int kHTerms = 32;
struct HGroup {
  int nt;
  int first;                          // nonzero: overwrite lambda instead of accumulating
  uint64_t x[kHTerms];                // X-or-Y mask of each term; equal masks are adjacent
  uint64_t z[kHTerms];
  double cre[kHTerms], cim[kHTerms];  // coeff * i^nY
  float fre[kHTerms], fim[kHTerms];   // the same, rounded to FP32 (complex64 states; the hi parts)
  float lre[kHTerms], lim[kHTerms];   // the rest rounded to FP32 (double-float lo parts)
};

// lambda_k (+)= sum_t c_t i^nY (-1)^popc((k^x_t) & z_t) psi_{k^x_t} over up to kHTerms
// terms of one or more X masks, so that lambda is read and written once per launch and
// psi is read once per distinct mask.  Two neighbouring k per step (k even): their
// sources k^x and (k+1)^x are the two halves of one aligned pair, read with one access
// and swapped when x has bit 0.  The coefficient sums and products are formed at the
// state's precision (complex64: FP32, whose result is stored in FP32 anyway;
// complex128: FP64); a term's sign is a select, not a product.
template <typename R>
__device__ __forceinline__ R hsum_re(const HGroup& g, int t) {
  if constexpr (sizeof(R) == 4) return g.fre[t]; else return g.cre[t];
}
template <typename R>
__device__ __forceinline__ R hsum_im(const HGroup& g, int t) {
  if constexpr (sizeof(R) == 4) return g.fim[t]; else return g.cim[t];
}

template <typename R>
__global__ void __launch_bounds__(256) k_apply_hsum(const R* __restrict__ psi, R* __restrict__ lam, uint64_t N,
                                                    HGroup g) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  const uint64_t tid = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x;
  if (N < 2) {  // a single amplitude (every x is 0)
    if (tid == 0) {
      const Cplx<R> p = ld_amp<R>(psi, 0);
      R fr = R(0), fi = R(0);
      for (int t = 0; t < g.nt; ++t) {
        fr += hsum_re<R>(g, t);
        fi += hsum_im<R>(g, t);
      }
      Cplx<R> out{fr * p.re - fi * p.im, fr * p.im + fi * p.re};
      if (!g.first) {
        const Cplx<R> o = ld_amp<R>(lam, 0);
        out.re += o.re;
        out.im += o.im;
      }
      st_amp<R>(lam, 0, out);
    }
    return;
  }
  for (uint64_t it = tid; it < N / 2; it += stride) {
    const uint64_t k = 2 * it;
    Cplx<R> o0{R(0), R(0)}, o1{R(0), R(0)};
    if (!g.first) ld_amp2<R>(lam, k, o0, o1);
    int t = 0;
    while (t < g.nt) {
      // the terms of one X mask (the same for every thread: no divergence)
      const uint64_t x = g.x[t];
      const uint64_t j0 = k ^ x;  // source of k; (k + 1)'s source is j0 ^ 1
      Cplx<R> a, b;
      ld_amp2<R>(psi, j0 & ~uint64_t(1), a, b);
      const Cplx<R> p0 = (x & 1) ? b : a, p1 = (x & 1) ? a : b;
      R f0r = R(0), f0i = R(0), f1r = R(0), f1i = R(0);
      do {
        const R cr = hsum_re<R>(g, t), ci = hsum_im<R>(g, t);
        const bool s0 = __popcll(j0 & g.z[t]) & 1;
        const bool s1 = s0 ^ bool(g.z[t] & 1);
        f0r += s0 ? -cr : cr;
        f0i += s0 ? -ci : ci;
        f1r += s1 ? -cr : cr;
        f1i += s1 ? -ci : ci;
      } while (++t < g.nt && g.x[t] == x);
      o0.re += f0r * p0.re - f0i * p0.im;
      o0.im += f0r * p0.im + f0i * p0.re;
      o1.re += f1r * p1.re - f1i * p1.im;
      o1.im += f1r * p1.im + f1i * p1.re;
    }
    st_amp2<R>(lam, k, o0, o1);
  }
}

// The same lambda (+)= H psi for complex128 states of 2^kDfMinQubits amplitudes or more
// in double-float arithmetic: amplitudes split into FP32 pairs, each X mask's signed
// coefficient sum added with TwoSum, its product with psi and the sum over masks as
// packed double-float terms, lambda joined back to binary64.
__global__ void __launch_bounds__(256) k_apply_hsum_df(const double* __restrict__ psi, double* __restrict__ lam,
                                                       uint64_t N, HGroup g) {
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t it = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; it < N / 2; it += stride) {
    const uint64_t k = 2 * it;
    DF2Acc o0{make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)}, o1 = o0;
    if (!g.first) {
      Cplx<double> a, b;
      ld_amp2<double>(lam, k, a, b);
      const DFC A = dfc_of(a), B = dfc_of(b);
      o0 = DF2Acc{A.hi, A.lo};
      o1 = DF2Acc{B.hi, B.lo};
    }
    int t = 0;
    while (t < g.nt) {
      const uint64_t x = g.x[t];
      const uint64_t j0 = k ^ x;
      Cplx<double> a, b;
      ld_amp2<double>(psi, j0 & ~uint64_t(1), a, b);
      const DFC p0 = dfc_of((x & 1) ? b : a), p1 = dfc_of((x & 1) ? a : b);
      DF2Acc f0, f1;
      bool first = true;
      do {
        const float2 ch = make_float2(g.fre[t], g.fim[t]), cl = make_float2(g.lre[t], g.lim[t]);
        const float2 nh = make_float2(-ch.x, -ch.y), nl = make_float2(-cl.x, -cl.y);
        const bool s0 = __popcll(j0 & g.z[t]) & 1;
        const bool s1 = s0 ^ bool(g.z[t] & 1);
        if (first) {
          f0 = DF2Acc{s0 ? nh : ch, s0 ? nl : cl};
          f1 = DF2Acc{s1 ? nh : ch, s1 ? nl : cl};
          first = false;
        } else {
          df2_add(f0, s0 ? nh : ch, s0 ? nl : cl);
          df2_add(f1, s1 ? nh : ch, s1 ? nl : cl);
        }
      } while (++t < g.nt && g.x[t] == x);
      const DF2 c0 = df2_result(f0), c1 = df2_result(f1);
      // o += c p: lanes (c.re, c.re) (p.re, p.im) + (-c.im, c.im) (p.im, p.re)
      df2_mac(o0, make_float2(c0.hi.x, c0.hi.x), make_float2(-c0.hi.x, -c0.hi.x), make_float2(c0.lo.x, c0.lo.x), dfc_x(p0));
      df2_mac(o0, make_float2(-c0.hi.y, c0.hi.y), make_float2(c0.hi.y, -c0.hi.y), make_float2(-c0.lo.y, c0.lo.y), dfc_sw(p0));
      df2_mac(o1, make_float2(c1.hi.x, c1.hi.x), make_float2(-c1.hi.x, -c1.hi.x), make_float2(c1.lo.x, c1.lo.x), dfc_x(p1));
      df2_mac(o1, make_float2(-c1.hi.y, c1.hi.y), make_float2(c1.hi.y, -c1.hi.y), make_float2(-c1.lo.y, c1.lo.y), dfc_sw(p1));
    }
    const DF2 r0 = df2_result(o0), r1 = df2_result(o1);
    st_amp2<double>(lam, k, Cplx<double>{df_join(r0.hi.x, r0.lo.x), df_join(r0.hi.y, r0.lo.y)},
                    Cplx<double>{df_join(r1.hi.x, r1.lo.x), df_join(r1.hi.y, r1.lo.y)});
  }
}

// Re and Im of <a|b>, block partials
template <typename R>
__global__ void __launch_bounds__(256) k_inner_partials(const R* __restrict__ a, const R* __restrict__ b, uint64_t N,
                                                        double* partials) {
  double sr = 0.0, si = 0.0;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < N; i += stride) {
    const Cplx<R> x = ld_amp<R>(a, i), y = ld_amp<R>(b, i);
    // each term at the state's precision, the sums in FP64
    const R tr = x.re * y.re + x.im * y.im, ti = x.re * y.im - x.im * y.re;
    if constexpr (sizeof(R) == 4) {
      sr += widen_exact(tr);
      si += widen_exact(ti);
    } else {
      sr += tr;
      si += ti;
    }
  }
  sr = block_sum(sr);
  si = block_sum(si);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = sr;
    partials[2 * blockIdx.x + 1] = si;
  }
}

// One reverse step of a rotation on bit `p` with generator G (0 X, 1 Y, 2 Z):
// partial[block] = Im <lambda|G|psi>; then psi <- Ud psi, lambda <- Ud lambda.
template <typename R>
__global__ void __launch_bounds__(256) k_adjoint_rot(R* __restrict__ psi, R* __restrict__ lam, uint64_t half, int p,
                                                     int gen, Mat2<R> ud, double* __restrict__ partial) {
  const Cplx<R> u00{ud.m[0], ud.m[1]}, u01{ud.m[2], ud.m[3]}, u10{ud.m[4], ud.m[5]}, u11{ud.m[6], ud.m[7]};
  const uint64_t m = uint64_t(1) << p, lo = m - 1;
  double acc = 0.0;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t it = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; it < half; it += stride) {
    const uint64_t i0 = ((it & ~lo) << 1) | (it & lo), i1 = i0 | m;
    const Cplx<R> a0 = ld_amp<R>(psi, i0), a1 = ld_amp<R>(psi, i1);
    const Cplx<R> l0 = ld_amp<R>(lam, i0), l1 = ld_amp<R>(lam, i1);
    // (G psi) on the pair; then Im sum conj(l) * (G psi), the pair's share formed at the
    // state's precision and added to the FP64 accumulator
    R gr0, gi0, gr1, gi1;
    if (gen == 0) {  // X
      gr0 = a1.re; gi0 = a1.im; gr1 = a0.re; gi1 = a0.im;
    } else if (gen == 1) {  // Y: (G psi)_0 = -i a1, (G psi)_1 = i a0
      gr0 = a1.im; gi0 = -a1.re; gr1 = -a0.im; gi1 = a0.re;
    } else {  // Z
      gr0 = a0.re; gi0 = a0.im; gr1 = -a1.re; gi1 = -a1.im;
    }
    const R share = l0.re * gi0 - l0.im * gr0 + l1.re * gi1 - l1.im * gr1;
    if constexpr (sizeof(R) == 4)
      acc += widen_exact(share);
    else
      acc += share;
    st_amp<R>(psi, i0, cmul2(u00, a0, u01, a1));
    st_amp<R>(psi, i1, cmul2(u10, a0, u11, a1));
    st_amp<R>(lam, i0, cmul2(u00, l0, u01, l1));
    st_amp<R>(lam, i1, cmul2(u10, l0, u11, l1));
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// grad[param[g]] += sum_b partials[g][b] for every recorded rotation g (fixed order)
// sum of each rotation's block partials into its first slot; k_collect_grads then adds
// the rotations that share a parameter, serially in gate order
__global__ void k_reduce_grads(double* partials, int nblocks, int nrot) {
  for (int g = blockIdx.x; g < nrot; g += gridDim.x) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) acc += partials[size_t(g) * nblocks + b];
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[size_t(g) * nblocks] = acc;
    __syncthreads();
  }
}

__global__ void k_sum2_adj(const double* partials, int count, double* out) {
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

// grad[p] = the sum of the recorded rotations g with params[g] == p, added in gate order
// (the order a serial loop over g would use, so the result does not depend on the
// launch); one thread per parameter.
__global__ void k_collect_grads(const double* partials, int nblocks, const int* params, int nrot, double* grad,
                                int nparams) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nparams; p += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int g = 0; g < nrot; ++g)
      if (params[g] == p) acc += partials[size_t(g) * nblocks];
    grad[p] = acc;
  }
}

// Per-process device workspace of the adjoint sweep (three state buffers and partials).
struct AdjWork {
  int device = -1;
  size_t bytes = 0;
  void* p = nullptr;
  void* scratch = nullptr;  // the psi handle's plan and reduction scratch, kept between calls
  size_t scratch_bytes = 0;
  cudaEvent_t done = nullptr;  // recorded after a call's last use of the workspace
  bool pending = false;
};
static AdjWork g_adj;
static AdjPlanBuf g_adj_plan;
// The workspace above belongs to the process: calls are serialised from workspace
// sizing to their last use of it (a concurrent call could otherwise free or overwrite
// the buffers while another call's kernels still use them).
static std::mutex g_adj_mu;

template <typename R>
static qc_status adjoint_impl(const qc_circuit* c, const double* params, int nparams,
                              const std::vector<ParsedTermA>& terms, const double* coeffs, qc_dtype dtype,
                              cudaStream_t stream, double* host_energy, double* host_grad, double* dev_energy,
                              double* dev_grad) {
  const int n = c->n;
  const uint64_t N = uint64_t(1) << n;
  const size_t sbytes = N * 2 * sizeof(R);
  // rotations, in order, with their parameter
  std::vector<ResolvedOp> rops(c->nops);
  std::vector<int> gen(c->nops, -1), pidx(c->nops, -1);
  int nrot = 0;
  for (int i = 0; i < c->nops; ++i) {
    const qc_op& op = c->ops[i];
    if (qc_status st = resolve_op(c, op, params, &rops[i])) return st;
    if (op.param >= 0) {
      if (op.kind != QC_GATE_RX && op.kind != QC_GATE_RY && op.kind != QC_GATE_RZ) {
        set_error("qc_adjoint_grad: parameterised op %d must be RX, RY or RZ", i);
        return QC_ERR_UNSUPPORTED;
      }
      if (op.param >= nparams) {
        set_error("qc_adjoint_grad: op %d uses parameter %d >= nparams", i, op.param);
        return QC_ERR_INVALID_ARG;
      }
      gen[i] = op.kind == QC_GATE_RX ? 0 : op.kind == QC_GATE_RY ? 1 : 2;
      pidx[i] = op.param;
      ++nrot;
    }
  }
  const int B = 256;
  const unsigned grid = stream_grid(N / 2, B, 8);
  // registers of 12 qubits and more take the fused sweep (tile passes over both
  // states), which writes one partial per rotation and SM; the per-rotation kernels
  // write one per block of `grid`.  (Complex128 is bound by GB300's FP64 rate either
  // way; with runs of CZ as sign ops the fused passes still come out ahead.)
  const bool fused = n >= adjoint_tiles_min_qubits();
  const unsigned pg = std::max<unsigned>(grid, unsigned(device_sm_count()));
  const size_t pbytes = sizeof(double) * (size_t(std::max(nrot, 1)) * pg + 2 * grid + 2 + nparams) + sizeof(int) * (nrot + 1);
  const size_t need = 2 * sbytes + ((pbytes + 255) & ~size_t(255)) + 256;
  int dev = 0;
  cudaGetDevice(&dev);
  if (g_adj.device != dev) {
    if (g_adj.p || g_adj.scratch) cudaDeviceSynchronize();
    if (g_adj.p) cudaFree(g_adj.p);
    if (g_adj.scratch) cudaFree(g_adj.scratch);
    g_adj = AdjWork();
    if (qc_status st = check_cuda(cudaEventCreateWithFlags(&g_adj.done, cudaEventDisableTiming), "adjoint event"))
      return st;
    g_adj.device = dev;
  }
  // a previous call (possibly on another stream) is done with the workspace first
  if (g_adj.pending)
    if (qc_status st = check_cuda(cudaStreamWaitEvent(stream, g_adj.done, 0), "adjoint ordering")) return st;
  if (g_adj.bytes < need) {
    if (g_adj.p) {
      cudaDeviceSynchronize();
      cudaFree(g_adj.p);
      g_adj.p = nullptr;
    }
    if (qc_status st = check_cuda(cudaMalloc(&g_adj.p, need), "adjoint workspace")) return st;
    g_adj.bytes = need;
    g_adj.device = dev;
  }
  char* w = static_cast<char*>(g_adj.p);
  R* lam = reinterpret_cast<R*>(w);
  double* part = reinterpret_cast<double*>(w + sbytes);
  double* inner = part + size_t(std::max(nrot, 1)) * pg;
  double* grad = inner + 2 * grid + 2;
  int* dparams = reinterpret_cast<int*>(grad + nparams);
  // psi: a state handle over the workspace so that the gate kernels can run on it
  qc_state s{};
  s.n = n;
  s.dtype = dtype;
  s.amps = w + sbytes + ((pbytes + 255) & ~size_t(255));
  s.stream = stream;
  s.device = dev;
  s.scratch = g_adj.scratch;
  s.scratch_bytes = g_adj.scratch_bytes;
  qc_state sl = s;
  sl.amps = lam;
  qc_status st = QC_OK;
  // forward
  if ((st = qc_state_init_basis(&s, 0))) goto done;
  // (the energy and the gradient do not see the forward state's global phase)
  if ((st = n >= 10 ? run_fused(&s, c, params, QC_PREC_AUTO, /*drop_global_phase=*/true)
                    : run_per_gate(&s, c, params)))
    goto done;
  {
    // lambda = H psi: the terms ordered by X mask, up to kHTerms per launch
    std::vector<int> order(terms.size());
    for (size_t t = 0; t < terms.size(); ++t) order[t] = int(t);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return terms[a].x < terms[b].x; });
    bool first = true;
    const unsigned g2 = stream_grid(N / 2 ? N / 2 : 1, B);
    for (size_t b0 = 0; b0 < order.size(); b0 += kHTerms) {
      HGroup hg{};
      hg.first = first ? 1 : 0;
      first = false;
      hg.nt = int(std::min<size_t>(kHTerms, order.size() - b0));
      for (int j = 0; j < hg.nt; ++j) {
        const ParsedTermA& t = terms[order[b0 + j]];
        const double cf = coeffs ? coeffs[order[b0 + j]] : 1.0;
        const int ny = t.ny & 3;  // i^ny
        hg.x[j] = t.x;
        hg.z[j] = t.z;
        hg.cre[j] = ny == 0 ? cf : ny == 2 ? -cf : 0.0;
        hg.cim[j] = ny == 1 ? cf : ny == 3 ? -cf : 0.0;
        hg.fre[j] = float(hg.cre[j]);
        hg.fim[j] = float(hg.cim[j]);
        hg.lre[j] = float(hg.cre[j] - double(hg.fre[j]));
        hg.lim[j] = float(hg.cim[j] - double(hg.fim[j]));
      }
      if (sizeof(R) == 8 && n >= kDfMinQubits)
        QC_COUNT(), k_apply_hsum_df<<<g2, B, 0, stream>>>(reinterpret_cast<const double*>(s.amps),
                                                          reinterpret_cast<double*>(lam), N, hg);
      else
        QC_COUNT(), k_apply_hsum<R><<<g2, B, 0, stream>>>(reinterpret_cast<const R*>(s.amps), lam, N, hg);
    }
    if (first) {  // empty Hamiltonian
      cudaMemsetAsync(lam, 0, sbytes, stream);
    }
    QC_COUNT(), k_inner_partials<R><<<grid, B, 0, stream>>>(reinterpret_cast<const R*>(s.amps), lam, N, inner);
    QC_COUNT(), k_sum2_adj<<<1, 1024, 0, stream>>>(inner, int(grid), inner + 2 * grid);
  }
  {
    // reverse sweep
    std::vector<int> rot_params;
    int r = nrot;
    int pgrid = int(grid);  // blocks whose partials each rotation sums
    std::vector<ResolvedOp> rev;
    std::vector<int> rgrad, rgen;
    for (int i = c->nops - 1; i >= 0; --i) {
      ResolvedOp ud = rops[i];
      const int dim = ud.form == FORM_2Q ? 4 : 2;
      // U^dagger
      double t[32];
      for (int a = 0; a < dim; ++a)
        for (int b = 0; b < dim; ++b) {
          t[2 * (a * dim + b)] = ud.m[2 * (b * dim + a)];
          t[2 * (a * dim + b) + 1] = -ud.m[2 * (b * dim + a) + 1];
        }
      memcpy(ud.m, t, sizeof(double) * 2 * dim * dim);
      if (fused) {
        // collected and run as tile passes below
        rev.push_back(ud);
        rgrad.push_back(gen[i] >= 0 ? --r : -1);
        rgen.push_back(gen[i]);
        if (gen[i] >= 0) rot_params.push_back(pidx[i]);
        continue;
      }
      if (gen[i] >= 0) {
        --r;
        Mat2<R> m;
        for (int e = 0; e < 8; ++e) m.m[e] = R(ud.m[e]);
        QC_COUNT(), k_adjoint_rot<R><<<grid, B, 0, stream>>>(reinterpret_cast<R*>(s.amps), lam, N / 2, ud.bits[0],
                                                             gen[i], m, part + size_t(r) * grid);
        rot_params.push_back(pidx[i]);
      } else {
        if ((st = apply_resolved(&s, ud))) goto done;
        if ((st = apply_resolved(&sl, ud))) goto done;
      }
    }
    if (fused && (st = adjoint_reverse_tiles<R>(n, rev, rgrad, rgen, reinterpret_cast<R*>(s.amps), lam, stream,
                                                 &g_adj_plan, part, &pgrid)))
      goto done;
    std::reverse(rot_params.begin(), rot_params.end());
    if (nrot > 0) {
      if ((st = check_cuda(cudaMemcpyAsync(dparams, rot_params.data(), sizeof(int) * nrot, cudaMemcpyHostToDevice,
                                           stream),
                           "upload")))
        goto done;
      QC_COUNT(), k_reduce_grads<<<std::min(nrot, 1024), 1024, 0, stream>>>(part, pgrid, nrot);
    }
    QC_COUNT(), k_collect_grads<<<unsigned(std::max(1, (nparams + 255) / 256)), 256, 0, stream>>>(part, pgrid, dparams,
                                                                                                nrot, grad, nparams);
    if ((st = check_launch("adjoint sweep"))) goto done;
    if (dev_energy) {
      // device outputs, asynchronous on the stream
      if ((st = check_cuda(cudaMemcpyAsync(dev_energy, inner + 2 * grid, sizeof(double), cudaMemcpyDeviceToDevice,
                                           stream),
                           "energy output")))
        goto done;
      if (nparams > 0 &&
          (st = check_cuda(cudaMemcpyAsync(dev_grad, grad, sizeof(double) * nparams, cudaMemcpyDeviceToDevice, stream),
                           "gradient output")))
        goto done;
    } else {
      std::vector<double> e(2);
      if ((st = check_cuda(cudaMemcpyAsync(e.data(), inner + 2 * grid, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                           stream),
                           "D2H")))
        goto done;
      if ((st = check_cuda(cudaMemcpyAsync(host_grad, grad, sizeof(double) * nparams, cudaMemcpyDeviceToHost,
                                           stream),
                           "D2H")))
        goto done;
      if ((st = check_cuda(cudaStreamSynchronize(stream), "qc_adjoint_grad"))) goto done;
      *host_energy = e[0];
    }
  }
done:
  // the psi handle's scratch stays with the workspace for the next call
  g_adj.scratch = s.scratch;
  g_adj.scratch_bytes = s.scratch_bytes;
  if (cudaEventRecord(g_adj.done, stream) == cudaSuccess) g_adj.pending = true;
  return st;
}

}  // namespace qcgb

using namespace qcgb;

extern "C" qc_status qc_adjoint_grad(const qc_circuit* c, const double* params, int nparams,
                                     const char* const* strings, const double* coeffs, int nterms, qc_dtype dtype,
                                     void* stream, double* host_energy, double* host_grad) {
  clear_error();
  if (!c || c->n < 1 || c->n > 32 || (c->nops > 0 && !c->ops) || nparams < 0 || (nparams > 0 && (!params || !host_grad)) ||
      nterms < 0 || (nterms > 0 && !strings) || !host_energy || (dtype != QC_C64 && dtype != QC_C128)) {
    set_error("qc_adjoint_grad: invalid arguments");
    return QC_ERR_INVALID_ARG;
  }
  std::vector<ParsedTermA> terms(nterms);
  for (int t = 0; t < nterms; ++t)
    if (qc_status st = parse_pauli_a(c->n, strings[t], &terms[t])) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_adj_mu);
  if (dtype == QC_C64)
    return adjoint_impl<float>(c, params, nparams, terms, coeffs, dtype, s, host_energy, host_grad, nullptr, nullptr);
  return adjoint_impl<double>(c, params, nparams, terms, coeffs, dtype, s, host_energy, host_grad, nullptr, nullptr);
}

extern "C" qc_status qc_inner(const qc_state* ca, const qc_state* cb, double* host_out) {
  clear_error();
  qc_state* a = const_cast<qc_state*>(ca);
  if (!a || !cb || !a->amps || !cb->amps || !host_out || a->n != cb->n || a->dtype != cb->dtype) {
    set_error("qc_inner: invalid arguments (same n and dtype required)");
    return QC_ERR_INVALID_ARG;
  }
  const uint64_t N = state_len(a);
  const int B = 256;
  const unsigned grid = stream_grid(N, B, 8);
  void* scr = nullptr;
  if (qc_status st = state_scratch(a, sizeof(double) * (2 * size_t(grid) + 2), &scr)) return st;
  double* part = static_cast<double*>(scr);
  if (a->dtype == QC_C64)
    QC_COUNT(), k_inner_partials<float><<<grid, B, 0, a->stream>>>(reinterpret_cast<const float*>(a->amps),
                                                                   reinterpret_cast<const float*>(cb->amps), N, part);
  else
    QC_COUNT(), k_inner_partials<double><<<grid, B, 0, a->stream>>>(reinterpret_cast<const double*>(a->amps),
                                                                    reinterpret_cast<const double*>(cb->amps), N, part);
  QC_COUNT(), k_sum2_adj<<<1, 1024, 0, a->stream>>>(part, int(grid), part + 2 * grid);
  if (qc_status st = check_launch("qc_inner")) return st;
  double h[2];
  if (qc_status st = check_cuda(cudaMemcpyAsync(h, part + 2 * grid, sizeof(h), cudaMemcpyDeviceToHost, a->stream),
                                "D2H"))
    return st;
  if (qc_status st = check_cuda(cudaStreamSynchronize(a->stream), "qc_inner")) return st;
  host_out[0] = h[0];
  host_out[1] = h[1];
  return QC_OK;
}

extern "C" qc_status qc_adjoint_grad_dev(const qc_circuit* c, const double* dev_params, int nparams,
                                         const qc_hamiltonian* H, qc_dtype dtype, void* stream, double* dev_energy,
                                         double* dev_grad) {
  clear_error();
  if (!c || c->n < 1 || c->n > 32 || (c->nops > 0 && !c->ops) || nparams < 0 ||
      (nparams > 0 && (!dev_params || !dev_grad)) || !H || H->nterms < 0 || (H->nterms > 0 && !H->terms) ||
      !dev_energy || (dtype != QC_C64 && dtype != QC_C128)) {
    set_error("qc_adjoint_grad_dev: invalid arguments");
    return QC_ERR_INVALID_ARG;
  }
  const uint64_t lim = c->n >= 64 ? ~uint64_t(0) : (uint64_t(1) << c->n);
  std::vector<ParsedTermA> terms(H->nterms);
  std::vector<double> coeffs(H->nterms);
  for (int t = 0; t < H->nterms; ++t) {
    const qc_pauli_term& T = H->terms[t];
    if (T.xmask >= lim || T.zmask >= lim) {
      set_error("qc_adjoint_grad_dev: term %d acts outside the %d qubits", t, c->n);
      return QC_ERR_INVALID_ARG;
    }
    terms[t] = ParsedTermA{T.xmask, T.zmask, __builtin_popcountll(T.xmask & T.zmask)};
    coeffs[t] = T.coeff;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // the plan is built on the host from the parameter values: one copy, waited for
  std::vector<double> params(size_t(std::max(nparams, 1)));
  if (nparams > 0) {
    if (qc_status st = check_cuda(cudaMemcpyAsync(params.data(), dev_params, sizeof(double) * nparams,
                                                  cudaMemcpyDeviceToHost, s),
                                  "parameter read"))
      return st;
    if (qc_status st = check_cuda(cudaStreamSynchronize(s), "parameter read")) return st;
  }
  std::lock_guard<std::mutex> lock(g_adj_mu);
  if (dtype == QC_C64)
    return adjoint_impl<float>(c, params.data(), nparams, terms, coeffs.data(), dtype, s, nullptr, nullptr,
                               dev_energy, dev_grad);
  return adjoint_impl<double>(c, params.data(), nparams, terms, coeffs.data(), dtype, s, nullptr, nullptr, dev_energy,
                              dev_grad);
}
