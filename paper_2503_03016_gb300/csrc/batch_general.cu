// General batched circuits in one persistent launch (qc_run_batch).
//
// Each circuit is an ordered gate list (QCLAB Sec. 2) applied to its own register from
// |0...0> (Sec. 3.2: every gate acts as I_l (x) U' (x) I_r on the whole register),
// followed by the expectation value of its Pauli sum.  The host resolves every op to
// its bit positions and matrix (the CUDA path's own gate definitions in circuit.cu);
// matrices of parameterised ops are formed on the device from the caller's FP64
// angles, so a batch whose parameters live in device memory needs no host round trip
// for them.  Complex64 states, FP32 gate arithmetic.
//
// Work split: persistent blocks (as many as fit on every SM) take circuits from an
// atomic counter, largest first.  A circuit of at most 13 qubits stays in the block's
// shared memory (64 KiB) from the initial state to its expectation value; a larger one
// runs in a per-block slice of a device workspace (or directly in the caller's output
// buffer for its state), one block-wide sweep per gate.  Between gates the block
// synchronises; within a gate, thread t takes the amplitude pairs (or quads) t,
// t + 256, ... so that neighbouring threads touch neighbouring amplitudes.
//
// Expectation values: the terms of a circuit's Pauli sum are grouped by X mask; for a
// group with mask x the value is Re sum_j conj(psi_{j^x}) psi_j W(j), where
// W(j) = sum_t c_t i^{|x & z_t|} (-1)^{|j & z_t|} (from P|j> = i^{|x&z|} (-1)^{|j&z|}
// |j^x>).  W and the per-amplitude products are formed in FP32, added in FP32 over 16
// amplitudes, then in FP64; the block total is a fixed-order FP64 reduction.
#include <string.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <map>
#include <mutex>
#include <vector>

#include "circuit.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace qcgb {

constexpr int kGbSmemBits = 13;  // complex64 state of up to 13 qubits in shared memory
constexpr int kGbMaxN = 20;
constexpr int kGbThreads = 256;
constexpr size_t kGbSmem = sizeof(float2) << kGbSmemBits;

struct GbOp {  // 16 bytes
  uint8_t type;  // 0: 2x2 on bit a, where the bits of cm read cv; 1: 4x4 on (a, b), row 2 b_a + b_b
  int8_t a, b;
  uint8_t pad;
  uint32_t cm, cv;
  uint32_t mat;  // float offset of the matrix (8 or 32 floats, row-major (re, im))
};
static_assert(sizeof(GbOp) == 16, "GbOp must be 16 bytes");

struct GbFix {  // a parameterised op: its matrix is formed on the device
  uint32_t mat;
  int32_t kind;
  int32_t adjoint;
  int32_t pad;
  int64_t param;  // index of its first angle in dev_params
};

struct GbCirc {
  int32_t n, out;
  int64_t op0;
  int32_t nops, g0;
  int32_t ngroups, state;  // state: index into the state pointers, or -1
};

struct GbGroup {
  uint64_t x;
  int32_t t0, nt;
};
struct GbTerm {
  uint64_t z;
  float cre, cim;  // coeff * i^{|x & z|}
};

// ---------------------------------------------------------------------------
// device
// ---------------------------------------------------------------------------

// Matrices of the parameterised ops from the FP64 angles (the gate definitions of
// resolve_op: RX, RY, RZ = exp(-i t G/2), U3 per OpenQASM, CP = diag(1, e^{i phi}) on
// the target), conjugate-transposed for adjoint ops, rounded to FP32.
__global__ void k_gb_resolve(const GbFix* __restrict__ fix, int nfix, const double* __restrict__ params,
                             float* __restrict__ pool) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nfix) return;
  const GbFix f = fix[i];
  const double t = params[f.param];
  double m[8];
  double c, s;
  switch (f.kind) {
    case QC_GATE_RX:
      sincos(0.5 * t, &s, &c);
      m[0] = c; m[1] = 0; m[2] = 0; m[3] = -s; m[4] = 0; m[5] = -s; m[6] = c; m[7] = 0;
      break;
    case QC_GATE_RY:
      sincos(0.5 * t, &s, &c);
      m[0] = c; m[1] = 0; m[2] = -s; m[3] = 0; m[4] = s; m[5] = 0; m[6] = c; m[7] = 0;
      break;
    case QC_GATE_RZ:
      sincos(0.5 * t, &s, &c);
      m[0] = c; m[1] = -s; m[2] = 0; m[3] = 0; m[4] = 0; m[5] = 0; m[6] = c; m[7] = s;
      break;
    case QC_GATE_CP:
      sincos(t, &s, &c);
      m[0] = 1; m[1] = 0; m[2] = 0; m[3] = 0; m[4] = 0; m[5] = 0; m[6] = c; m[7] = s;
      break;
    default: {  // U3(theta, phi, lambda)
      const double ph = params[f.param + 1], la = params[f.param + 2];
      sincos(0.5 * t, &s, &c);
      double sl, cl, sp, cp, spl, cpl;
      sincos(la, &sl, &cl);
      sincos(ph, &sp, &cp);
      sincos(ph + la, &spl, &cpl);
      m[0] = c; m[1] = 0;
      m[2] = -cl * s; m[3] = -sl * s;
      m[4] = cp * s; m[5] = sp * s;
      m[6] = cpl * c; m[7] = spl * c;
      break;
    }
  }
  if (f.adjoint) {  // U^dagger: transpose and conjugate
    double a[8] = {m[0], -m[1], m[4], -m[5], m[2], -m[3], m[6], -m[7]};
    for (int e = 0; e < 8; ++e) m[e] = a[e];
  }
  float* d = pool + f.mat;
  for (int e = 0; e < 8; ++e) d[e] = float(m[e]);
}

__device__ __forceinline__ float2 gb_cma(float2 a, float2 x, float2 b, float2 y) {
  float2 r;
  r.x = fmaf(a.x, x.x, fmaf(-a.y, x.y, fmaf(b.x, y.x, -b.y * y.y)));
  r.y = fmaf(a.x, x.y, fmaf(a.y, x.x, fmaf(b.x, y.y, b.y * y.x)));
  return r;
}

// Every op of a circuit on the state S (shared memory or global), one block-wide sweep
// per op, the block synchronised between ops.
__device__ __forceinline__ void gb_apply(float2* S, int n, const GbOp* __restrict__ ops, int nops,
                                         const float* __restrict__ pool) {
  const uint32_t N = 1u << n;
  for (int k = 0; k < nops; ++k) {
    const GbOp o = ops[k];
    const float* m = pool + o.mat;
    if (o.type == 0) {
      const float2 m00 = make_float2(m[0], m[1]), m01 = make_float2(m[2], m[3]);
      const float2 m10 = make_float2(m[4], m[5]), m11 = make_float2(m[6], m[7]);
      const uint32_t tb = 1u << o.a, lo = tb - 1u;
      for (uint32_t p = threadIdx.x; p < N / 2; p += blockDim.x) {
        const uint32_t i0 = ((p & ~lo) << 1) | (p & lo);
        if ((i0 & o.cm) != o.cv) continue;
        const uint32_t i1 = i0 | tb;
        const float2 x0 = S[i0], x1 = S[i1];
        S[i0] = gb_cma(m00, x0, m01, x1);
        S[i1] = gb_cma(m10, x0, m11, x1);
      }
    } else {
      float2 M[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) M[e] = make_float2(m[2 * e], m[2 * e + 1]);
      const uint32_t ba = 1u << o.a, bb = 1u << o.b;
      const int pl = o.a < o.b ? o.a : o.b, ph = o.a < o.b ? o.b : o.a;
      const uint32_t ll = (1u << pl) - 1u, hl = (1u << ph) - 1u;
      for (uint32_t p = threadIdx.x; p < N / 4; p += blockDim.x) {
        uint32_t i = ((p & ~ll) << 1) | (p & ll);
        i = ((i & ~hl) << 1) | (i & hl);
        const uint32_t ix[4] = {i, i | bb, i | ba, i | ba | bb};
        float2 x[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) x[r] = S[ix[r]];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float2 y0 = gb_cma(M[4 * r], x[0], M[4 * r + 1], x[1]);
          const float2 y1 = gb_cma(M[4 * r + 2], x[2], M[4 * r + 3], x[3]);
          S[ix[r]] = make_float2(y0.x + y1.x, y0.y + y1.y);
        }
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ double gb_observable(const float2* S, int n, const GbGroup* __restrict__ groups, int ng,
                                                const GbTerm* __restrict__ terms) {
  const uint32_t N = 1u << n;
  double acc = 0.0;
  for (int g = 0; g < ng; ++g) {
    const GbGroup G = groups[g];
    const uint32_t x = uint32_t(G.x);
    float part = 0.0f;
    int cnt = 0;
    for (uint32_t j = threadIdx.x; j < N; j += blockDim.x) {
      float wr = 0.0f, wi = 0.0f;
      for (int t = 0; t < G.nt; ++t) {
        const GbTerm T = terms[G.t0 + t];
        const bool neg = __popc(j & uint32_t(T.z)) & 1;
        wr += neg ? -T.cre : T.cre;
        wi += neg ? -T.cim : T.cim;
      }
      const float2 a = S[j ^ x], b = S[j];
      const float pr = fmaf(a.x, b.x, a.y * b.y), pi = fmaf(a.x, b.y, -a.y * b.x);
      part += fmaf(pr, wr, -pi * wi);
      if (++cnt == 16) {
        acc += double(part);
        part = 0.0f;
        cnt = 0;
      }
    }
    acc += double(part);
  }
  return block_sum(acc);
}

__global__ void __launch_bounds__(kGbThreads) k_batch_general(const GbCirc* __restrict__ circs, int ncirc,
                                                              const GbOp* __restrict__ ops,
                                                              const float* __restrict__ pool,
                                                              const GbGroup* __restrict__ groups,
                                                              const GbTerm* __restrict__ terms,
                                                              float2* const* __restrict__ states, float2* work,
                                                              uint64_t work_per_block, unsigned* counter,
                                                              double* __restrict__ out) {
  extern __shared__ float2 sS[];
  __shared__ int s_next;
  for (;;) {
    if (threadIdx.x == 0) s_next = int(atomicAdd(counter, 1u));
    __syncthreads();
    const int ci = s_next;
    __syncthreads();  // every thread has read s_next before it is overwritten
    if (ci >= ncirc) break;
    const GbCirc C = circs[ci];
    const uint32_t N = 1u << C.n;
    float2* dst = C.state >= 0 ? states[C.state] : nullptr;
    if (C.n <= kGbSmemBits) {
      for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) sS[i] = make_float2(i == 0 ? 1.0f : 0.0f, 0.0f);
      __syncthreads();
      gb_apply(sS, C.n, ops + C.op0, C.nops, pool);
      if (C.ngroups > 0) {
        const double v = gb_observable(sS, C.n, groups + C.g0, C.ngroups, terms);
        if (threadIdx.x == 0) out[C.out] = v;
      }
      if (dst)
        for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) dst[i] = sS[i];
    } else {
      float2* G = dst ? dst : work + uint64_t(blockIdx.x) * work_per_block;
      for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) G[i] = make_float2(i == 0 ? 1.0f : 0.0f, 0.0f);
      __syncthreads();
      gb_apply(G, C.n, ops + C.op0, C.nops, pool);
      if (C.ngroups > 0) {
        const double v = gb_observable(G, C.n, groups + C.g0, C.ngroups, terms);
        if (threadIdx.x == 0) out[C.out] = v;
      }
    }
    __syncthreads();
  }
}

__global__ void k_f64_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    b[i] = float(a[i]);
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------

// Process-wide workspace: the uploaded tables, the per-block states of circuits above
// 13 qubits and the FP32 angles of the ansatz fast path.  Calls are serialised; an
// event orders a call's uploads after the previous call's kernels on any stream.
struct GbWork {
  int device = -1;
  void* tables = nullptr;
  size_t tables_bytes = 0;
  void* states = nullptr;
  size_t states_bytes = 0;
  float* f32 = nullptr;
  size_t f32_len = 0;
  unsigned* counter = nullptr;
  cudaEvent_t done = nullptr;
  bool pending = false;
};
static GbWork g_gb;
static std::mutex g_gb_mu;
static thread_local int g_last_batch_path = 0;

static qc_status gb_grow(void** p, size_t* have, size_t need, const char* what) {
  if (*have >= need) return QC_OK;
  if (*p) {
    if (g_gb.pending) cudaEventSynchronize(g_gb.done);
    cudaFree(*p);
    *p = nullptr;
    *have = 0;
  }
  if (qc_status st = check_cuda(cudaMalloc(p, need), what)) return st;
  *have = need;
  return QC_OK;
}

// The layered ansatz of the fast path: per layer RY then RZ on every qubit (parameters
// layer*2n + 2q + {0, 1}), then CZ(q, q+1) for q = 0..n-2.
static bool is_ansatz(const qc_circuit& c, int* layers) {
  const int n = c.n;
  if (n < 6 || n > kGbMaxN || c.nops <= 0) return false;
  const int per = 3 * n - 1;
  if (c.nops % per) return false;
  const int L = c.nops / per;
  int k = 0;
  for (int l = 0; l < L; ++l) {
    for (int q = 0; q < n; ++q)
      for (int r = 0; r < 2; ++r) {
        const qc_op& o = c.ops[k++];
        if (o.kind != (r ? QC_GATE_RZ : QC_GATE_RY) || o.nq != 1 || o.qubits[0] != q || o.adjoint ||
            o.param != l * 2 * n + 2 * q + r)
          return false;
      }
    for (int q = 0; q + 1 < n; ++q) {
      const qc_op& o = c.ops[k++];
      if (o.kind != QC_GATE_CZ || o.nq != 2 || o.qubits[0] != q || o.qubits[1] != q + 1) return false;
    }
  }
  *layers = L;
  return true;
}

static bool is_zz_chain(const qc_hamiltonian* H, int n) {
  if (!H || H->nterms != n - 1 || !H->terms) return false;
  std::vector<uint64_t> z;
  for (int t = 0; t < H->nterms; ++t) {
    const qc_pauli_term& T = H->terms[t];
    if (T.xmask != 0 || T.coeff != 1.0) return false;
    z.push_back(T.zmask);
  }
  std::sort(z.begin(), z.end());
  for (int i = 0; i < n - 1; ++i)
    if (z[i] != (uint64_t(3) << i)) return false;
  return true;
}

// The ansatz kernel's fast path: the FP64 angles rounded to FP32 into the workspace,
// then qc_run_ansatz_batch.
static qc_status gb_fast_path(const qc_batch* b, int layers, cudaStream_t stream, double* dev_out) {
  std::vector<int32_t> ns(b->count);
  std::vector<int64_t> offs(b->count);
  for (int i = 0; i < b->count; ++i) {
    ns[i] = b->circuits[i].n;
    offs[i] = b->param_offset ? b->param_offset[i] : 0;
  }
  void* p = g_gb.f32;
  size_t have = g_gb.f32_len * sizeof(float);
  if (qc_status st = gb_grow(&p, &have, size_t(std::max<int64_t>(b->nparams, 1)) * sizeof(float), "batch angles"))
    return st;
  g_gb.f32 = static_cast<float*>(p);
  g_gb.f32_len = have / sizeof(float);
  if (b->nparams > 0)
    QC_COUNT(), k_f64_to_f32<<<stream_grid(uint64_t(b->nparams), 256, 4), 256, 0, stream>>>(b->dev_params, g_gb.f32,
                                                                                           b->nparams);
  if (qc_status st = check_launch("batch angles")) return st;
  qc_ansatz_batch ab{b->count, layers, ns.data(), offs.data(), g_gb.f32, b->nparams};
  return qc_run_ansatz_batch(&ab, stream, dev_out);
}

static size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace qcgb

using namespace qcgb;

extern "C" int qc_last_batch_path(void) { return g_last_batch_path; }

extern "C" qc_status qc_run_batch(const qc_batch* b, void* stream_v, double* dev_out) {
  clear_error();
  if (!b || b->count < 0 || b->nparams < 0 || (b->count > 0 && !b->circuits) ||
      (b->count > 0 && b->observables && !dev_out)) {
    set_error("qc_run_batch: invalid arguments");
    return QC_ERR_INVALID_ARG;
  }
  if (b->count == 0) return QC_OK;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_v);
  auto obs = [&](int i) -> const qc_hamiltonian* {
    if (!b->observables) return nullptr;
    return b->shared_observable ? &b->observables[0] : &b->observables[i];
  };
  bool any_states = false;
  int64_t max_param = -1;
  for (int i = 0; i < b->count; ++i) {
    const qc_circuit& c = b->circuits[i];
    if (c.n < 1 || c.n > kGbMaxN || c.nops < 0 || (c.nops > 0 && !c.ops)) {
      set_error("qc_run_batch: circuit %d: n=%d (supported 1..%d) or its op list is invalid", i, c.n, kGbMaxN);
      return c.n > kGbMaxN ? QC_ERR_UNSUPPORTED : QC_ERR_INVALID_ARG;
    }
    if (const qc_hamiltonian* H = obs(i)) {
      if (H->nterms < 0 || (H->nterms > 0 && !H->terms)) {
        set_error("qc_run_batch: observable of circuit %d is invalid", i);
        return QC_ERR_INVALID_ARG;
      }
      const uint64_t lim = uint64_t(1) << c.n;
      for (int t = 0; t < H->nterms; ++t)
        if (H->terms[t].xmask >= lim || H->terms[t].zmask >= lim) {
          set_error("qc_run_batch: term %d of circuit %d acts outside its %d qubits", t, i, c.n);
          return QC_ERR_INVALID_ARG;
        }
    }
    if (b->dev_states && b->dev_states[i]) {
      if (reinterpret_cast<uintptr_t>(b->dev_states[i]) & 15u) {
        set_error("qc_run_batch: state buffer of circuit %d is not 16-byte aligned", i);
        return QC_ERR_INVALID_ARG;
      }
      any_states = true;
    }
    const int64_t poff = b->param_offset ? b->param_offset[i] : 0;
    for (int k = 0; k < c.nops; ++k) {
      const qc_op& o = c.ops[k];
      const bool rot = o.kind == QC_GATE_RX || o.kind == QC_GATE_RY || o.kind == QC_GATE_RZ ||
                       o.kind == QC_GATE_U3 || o.kind == QC_GATE_CP;
      if (!rot || o.param < 0) continue;
      const int64_t last = poff + o.param + (o.kind == QC_GATE_U3 ? 2 : 0);
      if (!b->dev_params || poff + o.param < 0 || last >= b->nparams) {
        set_error("qc_run_batch: op %d of circuit %d reads parameter %lld outside dev_params (%lld)", k, i,
                  (long long)last, (long long)b->nparams);
        return QC_ERR_INVALID_ARG;
      }
      max_param = std::max<int64_t>(max_param, o.param + 2);
    }
  }
  std::lock_guard<std::mutex> lock(g_gb_mu);
  int dev = 0;
  if (qc_status st = check_cuda(cudaGetDevice(&dev), "cudaGetDevice")) return st;
  if (g_gb.device != dev) {
    if (g_gb.device >= 0 && g_gb.pending) cudaEventSynchronize(g_gb.done);
    g_gb = GbWork();
    g_gb.device = dev;
    if (qc_status st = check_cuda(cudaEventCreateWithFlags(&g_gb.done, cudaEventDisableTiming), "batch event"))
      return st;
  }
  // the workspace is reused: this call's uploads and kernels follow the previous call's
  if (g_gb.pending)
    if (qc_status st = check_cuda(cudaStreamWaitEvent(stream, g_gb.done, 0), "batch ordering")) return st;

  // fast path: every circuit the layered ansatz with the same depth, observable the chain
  int layers = -1;
  bool fast = b->observables && !any_states && b->dev_params;
  for (int i = 0; fast && i < b->count; ++i) {
    int L = 0;
    fast = is_ansatz(b->circuits[i], &L) && (layers < 0 || L == layers) && is_zz_chain(obs(i), b->circuits[i].n);
    layers = L;
  }
  if (fast) {
    qc_status st = gb_fast_path(b, layers, stream, dev_out);
    if (st == QC_OK) st = check_cuda(cudaEventRecord(g_gb.done, stream), "batch event");
    g_gb.pending = st == QC_OK;
    g_last_batch_path = 1;
    return st;
  }

  // general path: encode every circuit's ops, parameter fixes and term groups
  std::vector<int> order(b->count);
  for (int i = 0; i < b->count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return b->circuits[x].n > b->circuits[y].n; });
  std::vector<double> zeros(size_t(std::max<int64_t>(max_param + 1, 3)), 0.0);
  std::vector<GbCirc> circs;
  std::vector<GbOp> ops;
  std::vector<float> pool;
  std::vector<GbFix> fixes;
  std::vector<GbGroup> groups;
  std::vector<GbTerm> terms;
  std::vector<void*> sptr;
  std::map<std::vector<float>, uint32_t> shared_mats;  // matrices of fixed gates, stored once
  int max_work_n = 0;
  for (int i : order) {
    const qc_circuit& c = b->circuits[i];
    const int64_t poff = b->param_offset ? b->param_offset[i] : 0;
    GbCirc C{};
    C.n = c.n;
    C.out = i;
    C.op0 = int64_t(ops.size());
    C.nops = c.nops;
    C.state = -1;
    if (b->dev_states && b->dev_states[i]) {
      C.state = int(sptr.size());
      sptr.push_back(b->dev_states[i]);
    } else if (c.n > kGbSmemBits) {
      max_work_n = std::max(max_work_n, c.n);
    }
    for (int k = 0; k < c.nops; ++k) {
      const qc_op& o = c.ops[k];
      ResolvedOp r;
      if (qc_status st = resolve_op(&c, o, zeros.data(), &r)) {
        set_error("qc_run_batch: circuit %d, op %d is invalid", i, k);
        return st;
      }
      GbOp g{};
      int dim = 2;
      if (r.form == FORM_2Q) {
        g.type = 1;
        g.a = int8_t(r.bits[0]);
        g.b = int8_t(r.bits[1]);
        dim = 4;
      } else {
        g.type = 0;
        const int nc = r.form == FORM_CTRL ? r.nq - 1 : 0;
        g.a = int8_t(r.bits[nc]);
        for (int j = 0; j < nc; ++j) {
          g.cm |= 1u << r.bits[j];
          if ((r.cstate >> j) & 1u) g.cv |= 1u << r.bits[j];
        }
      }
      const bool param_op = o.param >= 0 && (o.kind == QC_GATE_RX || o.kind == QC_GATE_RY ||
                                             o.kind == QC_GATE_RZ || o.kind == QC_GATE_U3 || o.kind == QC_GATE_CP);
      std::vector<float> m(2 * dim * dim);
      for (size_t e = 0; e < m.size(); ++e) m[e] = float(r.m[e]);
      if (param_op) {
        g.mat = uint32_t(pool.size());
        pool.insert(pool.end(), m.begin(), m.end());
        fixes.push_back(GbFix{g.mat, o.kind, o.adjoint ? 1 : 0, 0, poff + o.param});
      } else {
        auto it = shared_mats.find(m);
        if (it == shared_mats.end()) {
          it = shared_mats.emplace(m, uint32_t(pool.size())).first;
          pool.insert(pool.end(), m.begin(), m.end());
        }
        g.mat = it->second;
      }
      ops.push_back(g);
    }
    C.g0 = int(groups.size());
    if (const qc_hamiltonian* H = obs(i)) {
      std::vector<int> to(H->nterms);
      for (int t = 0; t < H->nterms; ++t) to[t] = t;
      std::stable_sort(to.begin(), to.end(), [&](int x, int y) { return H->terms[x].xmask < H->terms[y].xmask; });
      for (int t : to) {
        const qc_pauli_term& T = H->terms[t];
        if (groups.size() == size_t(C.g0) || groups.back().x != T.xmask)
          groups.push_back(GbGroup{T.xmask, int32_t(terms.size()), 0});
        const int ny = __builtin_popcountll(T.xmask & T.zmask) & 3;  // i^ny
        const double cre = ny == 0 ? T.coeff : ny == 2 ? -T.coeff : 0.0;
        const double cim = ny == 1 ? T.coeff : ny == 3 ? -T.coeff : 0.0;
        terms.push_back(GbTerm{T.zmask, float(cre), float(cim)});
        groups.back().nt++;
      }
    }
    C.ngroups = int(groups.size()) - C.g0;
    circs.push_back(C);
  }
  if (pool.size() >= (size_t(1) << 32)) {
    set_error("qc_run_batch: too many gate matrices in one batch");
    return QC_ERR_UNSUPPORTED;
  }
  // one device buffer for every table
  const size_t o_circ = 0;
  const size_t o_ops = o_circ + al256(circs.size() * sizeof(GbCirc));
  const size_t o_pool = o_ops + al256(std::max<size_t>(ops.size(), 1) * sizeof(GbOp));
  const size_t o_fix = o_pool + al256(std::max<size_t>(pool.size(), 1) * sizeof(float));
  const size_t o_grp = o_fix + al256(std::max<size_t>(fixes.size(), 1) * sizeof(GbFix));
  const size_t o_term = o_grp + al256(std::max<size_t>(groups.size(), 1) * sizeof(GbGroup));
  const size_t o_sptr = o_term + al256(std::max<size_t>(terms.size(), 1) * sizeof(GbTerm));
  const size_t total = o_sptr + al256(std::max<size_t>(sptr.size(), 1) * sizeof(void*)) + 256;
  if (qc_status st = gb_grow(&g_gb.tables, &g_gb.tables_bytes, total, "batch tables")) return st;
  if (!g_gb.counter) {
    void* p = nullptr;
    if (qc_status st = check_cuda(cudaMalloc(&p, 256), "batch counter")) return st;
    g_gb.counter = static_cast<unsigned*>(p);
  }
  std::vector<char> host(total, 0);
  auto put = [&](size_t off, const void* src, size_t bytes) {
    if (bytes) memcpy(host.data() + off, src, bytes);
  };
  put(o_circ, circs.data(), circs.size() * sizeof(GbCirc));
  put(o_ops, ops.data(), ops.size() * sizeof(GbOp));
  put(o_pool, pool.data(), pool.size() * sizeof(float));
  put(o_fix, fixes.data(), fixes.size() * sizeof(GbFix));
  put(o_grp, groups.data(), groups.size() * sizeof(GbGroup));
  put(o_term, terms.data(), terms.size() * sizeof(GbTerm));
  put(o_sptr, sptr.data(), sptr.size() * sizeof(void*));
  char* d = static_cast<char*>(g_gb.tables);
  if (qc_status st = check_cuda(cudaMemcpyAsync(d, host.data(), total, cudaMemcpyHostToDevice, stream),
                                "batch table upload"))
    return st;
  if (qc_status st = check_cuda(cudaFuncSetAttribute(k_batch_general, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     int(kGbSmem)),
                                "batch shared memory"))
    return st;
  int per_sm = 0;
  if (qc_status st = check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_general, kGbThreads,
                                                                             kGbSmem),
                                "batch occupancy"))
    return st;
  const int grid = std::max(1, std::min(per_sm, 3)) * device_sm_count();
  const uint64_t wpb = max_work_n ? (uint64_t(1) << max_work_n) : 0;
  if (wpb)
    if (qc_status st = gb_grow(&g_gb.states, &g_gb.states_bytes, size_t(grid) * wpb * sizeof(float2),
                               "batch state workspace"))
      return st;
  float* dpool = reinterpret_cast<float*>(d + o_pool);
  if (!fixes.empty())
    QC_COUNT(), k_gb_resolve<<<unsigned((fixes.size() + 255) / 256), 256, 0, stream>>>(
                    reinterpret_cast<const GbFix*>(d + o_fix), int(fixes.size()), b->dev_params, dpool);
  if (qc_status st = check_cuda(cudaMemsetAsync(g_gb.counter, 0, sizeof(unsigned), stream), "batch counter reset"))
    return st;
  QC_COUNT(), k_batch_general<<<unsigned(grid), kGbThreads, kGbSmem, stream>>>(
                  reinterpret_cast<const GbCirc*>(d + o_circ), int(circs.size()),
                  reinterpret_cast<const GbOp*>(d + o_ops), dpool, reinterpret_cast<const GbGroup*>(d + o_grp),
                  reinterpret_cast<const GbTerm*>(d + o_term), reinterpret_cast<float2* const*>(d + o_sptr),
                  static_cast<float2*>(g_gb.states), wpb, g_gb.counter, dev_out);
  if (qc_status st = check_launch("general batch kernel")) return st;
  if (qc_status st = check_cuda(cudaEventRecord(g_gb.done, stream), "batch event")) return st;
  g_gb.pending = true;
  g_last_batch_path = 0;
  return QC_OK;
}
