// Circuits: gate matrices, dense k-qubit blocks and the circuit runner.
//
// QCLAB Sec. 2 builds a circuit as an ordered list of gates (push_back, nested
// sub-circuits flattened in order); Sec. 3.2 applies each gate to the whole register.
// QC_RUN_PER_GATE does exactly that, one sweep per gate.  QC_RUN_FUSED hands the list
// to the planner (planner.cu), which groups gates into shared-memory tile passes and
// fused blocks with the same product.
#include <string.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "circuit.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace qcgb {

using cd = std::complex<double>;

// ---------------------------------------------------------------------------
// gate matrices (OpenQASM 2 definitions for the gates the paper does not spell out)
// ---------------------------------------------------------------------------
static void put2(double* m, cd a, cd b, cd c, cd d) {
  m[0] = a.real(); m[1] = a.imag(); m[2] = b.real(); m[3] = b.imag();
  m[4] = c.real(); m[5] = c.imag(); m[6] = d.real(); m[7] = d.imag();
}

static void adjoint_inplace(double* m, int dim) {
  std::vector<double> t(2 * dim * dim);
  for (int r = 0; r < dim; ++r)
    for (int c = 0; c < dim; ++c) {
      t[2 * (r * dim + c)] = m[2 * (c * dim + r)];
      t[2 * (r * dim + c) + 1] = -m[2 * (c * dim + r) + 1];
    }
  memcpy(m, t.data(), sizeof(double) * t.size());
}

qc_status op_angles(const qc_op& op, const double* params, double* ang) {
  const int cnt = op.kind == QC_GATE_U3 ? 3 : 1;
  for (int i = 0; i < cnt; ++i) {
    if (op.param >= 0) {
      if (!params) {
        set_error("op uses parameter %d but no parameter vector was given", op.param);
        return QC_ERR_INVALID_ARG;
      }
      ang[i] = params[op.param + i];
    } else {
      ang[i] = op.angle[i];
    }
  }
  return QC_OK;
}

qc_status resolve_op(const qc_circuit* c, const qc_op& op, const double* params, ResolvedOp* out) {
  ResolvedOp r{};
  const double h = 1.0 / std::sqrt(2.0);
  const cd I(0, 1);
  double ang[3] = {0, 0, 0};
  const int k = op.kind;
  if (k == QC_GATE_RX || k == QC_GATE_RY || k == QC_GATE_RZ || k == QC_GATE_U3 || k == QC_GATE_CP)
    if (qc_status st = op_angles(op, params, ang)) return st;
  int need = 1;
  switch (k) {
    case QC_GATE_MATRIX1:
    case QC_GATE_MATRIX2:
    case QC_GATE_CTRL_MATRIX1: {
      const int dim = k == QC_GATE_MATRIX2 ? 4 : 2;
      if (op.matrix < 0 || !c->pool || op.matrix + 2 * dim * dim > c->pool_len) {
        set_error("op matrix offset %lld out of the pool", (long long)op.matrix);
        return QC_ERR_INVALID_ARG;
      }
      memcpy(r.m, c->pool + op.matrix, sizeof(double) * 2 * dim * dim);
      r.form = k == QC_GATE_MATRIX2 ? FORM_2Q : (k == QC_GATE_MATRIX1 ? FORM_1Q : FORM_CTRL);
      need = k == QC_GATE_MATRIX2 ? 2 : (k == QC_GATE_MATRIX1 ? 1 : 2);
      break;
    }
    case QC_GATE_H: put2(r.m, h, h, h, -h); r.form = FORM_1Q; break;
    case QC_GATE_X: put2(r.m, 0, 1, 1, 0); r.form = FORM_1Q; break;
    case QC_GATE_Y: put2(r.m, 0, -I, I, 0); r.form = FORM_1Q; break;
    case QC_GATE_Z: put2(r.m, 1, 0, 0, -1); r.form = FORM_1Q; break;
    case QC_GATE_S: put2(r.m, 1, 0, 0, I); r.form = FORM_1Q; break;
    case QC_GATE_SDG: put2(r.m, 1, 0, 0, -I); r.form = FORM_1Q; break;
    case QC_GATE_T: put2(r.m, 1, 0, 0, std::exp(I * (M_PI / 4))); r.form = FORM_1Q; break;
    case QC_GATE_TDG: put2(r.m, 1, 0, 0, std::exp(-I * (M_PI / 4))); r.form = FORM_1Q; break;
    case QC_GATE_RX: {
      const double cs = std::cos(ang[0] / 2), sn = std::sin(ang[0] / 2);
      put2(r.m, cs, -I * sn, -I * sn, cs);
      r.form = FORM_1Q;
      break;
    }
    case QC_GATE_RY: {
      const double cs = std::cos(ang[0] / 2), sn = std::sin(ang[0] / 2);
      put2(r.m, cs, -sn, sn, cs);
      r.form = FORM_1Q;
      break;
    }
    case QC_GATE_RZ:
      put2(r.m, std::exp(-I * (ang[0] / 2)), 0, 0, std::exp(I * (ang[0] / 2)));
      r.form = FORM_1Q;
      break;
    case QC_GATE_U3: {
      const double cs = std::cos(ang[0] / 2), sn = std::sin(ang[0] / 2);
      put2(r.m, cs, -std::exp(I * ang[2]) * sn, std::exp(I * ang[1]) * sn, std::exp(I * (ang[1] + ang[2])) * cs);
      r.form = FORM_1Q;
      break;
    }
    case QC_GATE_CNOT: put2(r.m, 0, 1, 1, 0); r.form = FORM_CTRL; need = 2; break;
    case QC_GATE_CZ: put2(r.m, 1, 0, 0, -1); r.form = FORM_CTRL; need = 2; break;
    case QC_GATE_CP: put2(r.m, 1, 0, 0, std::exp(I * ang[0])); r.form = FORM_CTRL; need = 2; break;
    case QC_GATE_MCX: put2(r.m, 0, 1, 1, 0); r.form = FORM_CTRL; need = 2; break;
    case QC_GATE_SWAP: {
      memset(r.m, 0, sizeof(r.m));
      r.m[0] = 1; r.m[2 * (1 * 4 + 2)] = 1; r.m[2 * (2 * 4 + 1)] = 1; r.m[2 * 15] = 1;
      r.form = FORM_2Q;
      need = 2;
      break;
    }
    default:
      set_error("unknown gate kind %d", k);
      return QC_ERR_INVALID_ARG;
  }
  if (op.nq < need || op.nq > QC_MAX_OP_QUBITS || (r.form != FORM_CTRL && op.nq != need)) {
    set_error("gate kind %d has %d qubits", k, op.nq);
    return QC_ERR_INVALID_ARG;
  }
  for (int i = 0; i < op.nq; ++i) {
    if (op.qubits[i] < 0 || op.qubits[i] >= c->n) {
      set_error("qubit %d out of range", op.qubits[i]);
      return QC_ERR_INVALID_ARG;
    }
    for (int j = 0; j < i; ++j)
      if (op.qubits[i] == op.qubits[j]) {
        set_error("repeated qubit %d in one gate", op.qubits[i]);
        return QC_ERR_INVALID_ARG;
      }
    r.bits[i] = c->n - 1 - op.qubits[i];
  }
  r.nq = op.nq;
  r.cstate = (k == QC_GATE_MCX || k == QC_GATE_CTRL_MATRIX1) ? op.ctrl_states : 0xFFFFFFFFu;
  if (op.adjoint) adjoint_inplace(r.m, r.form == FORM_2Q ? 4 : 2);
  *out = r;
  return QC_OK;
}

qc_status apply_resolved(qc_state* s, const ResolvedOp& r) {
  if (r.form == FORM_1Q) return apply_1q_bits(s, r.bits[0], nullptr, nullptr, 0, r.m);
  if (r.form == FORM_2Q) return apply_2q_bits(s, r.bits[0], r.bits[1], r.m);
  const int nc = r.nq - 1;
  int cv[QC_MAX_OP_QUBITS];
  for (int j = 0; j < nc; ++j) cv[j] = (r.cstate >> j) & 1;
  return apply_1q_bits(s, r.bits[nc], r.bits, cv, nc, r.m);
}

// ---------------------------------------------------------------------------
// dense k-qubit block, native precision: a CTA takes 32 consecutive groups of 2^k
// amplitudes, stages them in shared memory as [row][group], and every thread forms
// out[r][g] = sum_c U[r][c] v[c][g] with U broadcast from shared memory.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_kq_native(R* __restrict__ a, uint64_t ngroups, int k, KqSpec sp,
                                                   const R* __restrict__ Ug, bool u_in_smem) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int D = 1 << k;
  // U (D*D) is staged in shared memory when it fits, else read through the caches
  Cplx<R>* Us = reinterpret_cast<Cplx<R>*>(smem_raw);
  Cplx<R>* V = u_in_smem ? Us + D * D : Us;  // D rows x 32 groups
  if (u_in_smem)
    for (int i = threadIdx.x; i < D * D; i += blockDim.x) Us[i] = Cplx<R>{Ug[2 * i], Ug[2 * i + 1]};
  const Cplx<R>* U = u_in_smem ? Us : reinterpret_cast<const Cplx<R>*>(Ug);
  const int per = D * 32 / blockDim.x > 0 ? D * 32 / blockDim.x : 1;
  const uint64_t nchunks = (ngroups + 31) / 32;
  for (uint64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    __syncthreads();
    for (int e = threadIdx.x; e < D * 32; e += blockDim.x) {
      const int g = e & 31, r = e >> 5;
      const uint64_t gi = ch * 32 + g;
      if (gi < ngroups) {
        const uint64_t base = insert_zero_bits(gi, sp.pos, sp.cnt);
        V[r * 32 + g] = ld_amp<R>(a, base | sp.off[r]);
      }
    }
    __syncthreads();
    Cplx<R> out[16];
    for (int j = 0; j < per && j < 16; ++j) {
      const int e = threadIdx.x + j * blockDim.x;
      if (e >= D * 32) break;
      const int g = e & 31, r = e >> 5;
      R sr = 0, si = 0;
      for (int c = 0; c < D; ++c) {
        const Cplx<R> u = U[r * D + c], v = V[c * 32 + g];
        sr = fma(u.re, v.re, fma(-u.im, v.im, sr));
        si = fma(u.re, v.im, fma(u.im, v.re, si));
      }
      out[j] = Cplx<R>{sr, si};
    }
    for (int j = 0; j < per && j < 16; ++j) {
      const int e = threadIdx.x + j * blockDim.x;
      if (e >= D * 32) break;
      const int g = e & 31, r = e >> 5;
      const uint64_t gi = ch * 32 + g;
      if (gi < ngroups) {
        const uint64_t base = insert_zero_bits(gi, sp.pos, sp.cnt);
        st_amp<R>(a, base | sp.off[r], out[j]);
      }
    }
  }
}

qc_status apply_kq_native(qc_state* s, const int* bits, int k, const double* U) {
  if (k < 1 || k > 7 || k > s->n) {
    set_error("fused block size k=%d out of range", k);
    return QC_ERR_INVALID_ARG;
  }
  KqSpec sp{};
  std::vector<int> sorted(bits, bits + k);
  std::sort(sorted.begin(), sorted.end());
  sp.cnt = k;
  for (int j = 0; j < k; ++j) sp.pos[j] = int8_t(sorted[j]);
  const int D = 1 << k;
  for (int r = 0; r < D; ++r) {
    uint64_t off = 0;
    for (int j = 0; j < k; ++j)
      if ((r >> (k - 1 - j)) & 1) off |= uint64_t(1) << bits[j];
    sp.off[r] = off;
  }
  const uint64_t ngroups = state_len(s) >> k;
  const size_t esz = s->dtype == QC_C64 ? 8 : 16;
  size_t smem = esz * (size_t(D) * D + size_t(D) * 32);
  const bool u_in_smem = smem <= 200 * 1024;
  if (!u_in_smem) smem = esz * size_t(D) * 32;
  // the matrix goes through a small device buffer in the state's precision
  void* scr = nullptr;
  if (qc_status st = state_scratch(s, esz * D * D, &scr)) return st;
  std::vector<float> uf;
  if (s->dtype == QC_C64) {
    uf.resize(2 * D * D);
    for (int i = 0; i < 2 * D * D; ++i) uf[i] = float(U[i]);
    if (qc_status st = check_cuda(cudaMemcpyAsync(scr, uf.data(), esz * D * D, cudaMemcpyHostToDevice, s->stream),
                                  "block upload"))
      return st;
  } else {
    if (qc_status st = check_cuda(cudaMemcpyAsync(scr, U, esz * D * D, cudaMemcpyHostToDevice, s->stream),
                                  "block upload"))
      return st;
  }
  const unsigned grid = stream_grid((ngroups + 31) / 32, 1, 4);
  if (s->dtype == QC_C64) {
    cudaFuncSetAttribute(k_kq_native<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    QC_COUNT(), k_kq_native<float><<<grid, 256, smem, s->stream>>>(reinterpret_cast<float*>(s->amps), ngroups, k, sp,
                                                       reinterpret_cast<const float*>(scr), u_in_smem);
  } else {
    cudaFuncSetAttribute(k_kq_native<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    QC_COUNT(), k_kq_native<double><<<grid, 256, smem, s->stream>>>(reinterpret_cast<double*>(s->amps), ngroups, k, sp,
                                                        reinterpret_cast<const double*>(scr), u_in_smem);
  }
  return check_launch("fused block");
}

qc_status apply_kq_bits(qc_state* s, const int* bits, int k, const double* U, qc_prec prec) {
  if (prec == QC_PREC_TF32X3) return apply_kq_tf32x3(s, bits, k, U);
  return apply_kq_native(s, bits, k, U);
}

qc_status run_per_gate(qc_state* s, const qc_circuit* c, const double* params) {
  for (int i = 0; i < c->nops; ++i) {
    ResolvedOp r;
    if (qc_status st = resolve_op(c, c->ops[i], params, &r)) return st;
    if (qc_status st = apply_resolved(s, r)) return st;
  }
  return QC_OK;
}

}  // namespace qcgb

using namespace qcgb;

extern "C" {

qc_status qc_apply_fused_k(qc_state* s, const int* qubits, int k, const double* U, qc_prec prec) {
  clear_error();
  if (!s || !s->amps || !qubits || !U || k < 1 || k > 7 || k > s->n) {
    set_error("qc_apply_fused_k: invalid arguments");
    return QC_ERR_INVALID_ARG;
  }
  int bits[8];
  for (int j = 0; j < k; ++j) {
    if (qubits[j] < 0 || qubits[j] >= s->n) {
      set_error("qc_apply_fused_k: qubit %d out of range", qubits[j]);
      return QC_ERR_INVALID_ARG;
    }
    for (int i = 0; i < j; ++i)
      if (qubits[i] == qubits[j]) {
        set_error("qc_apply_fused_k: repeated qubit %d", qubits[j]);
        return QC_ERR_INVALID_ARG;
      }
    bits[j] = s->n - 1 - qubits[j];
  }
  if (prec == QC_PREC_BF16X3) {
    set_error("qc_apply_fused_k: BF16x3 products keep about 16 significant bits, too few for 1e-5");
    return QC_ERR_UNSUPPORTED;
  }
  if (prec == QC_PREC_AUTO) prec = QC_PREC_NATIVE;  // one block: nothing to choose between passes
  if (prec != QC_PREC_NATIVE && prec != QC_PREC_TF32X3) {
    set_error("qc_apply_fused_k: unknown precision mode %d", int(prec));
    return QC_ERR_INVALID_ARG;
  }
  if (prec == QC_PREC_TF32X3 && (s->dtype != QC_C64 || k < 2 || k > 6)) {
    set_error("qc_apply_fused_k: TF32x3 blocks need a complex64 state and 2 <= k <= 6");
    return QC_ERR_UNSUPPORTED;
  }
  return apply_kq_bits(s, bits, k, U, prec);
}

qc_status qc_run_circuit(qc_state* s, const qc_circuit* c, const double* params, qc_run_mode mode, qc_prec prec) {
  clear_error();
  if (!s || !s->amps || !c || (c->nops > 0 && !c->ops) || c->n != s->n) {
    set_error("qc_run_circuit: invalid arguments (circuit n must equal state n)");
    return QC_ERR_INVALID_ARG;
  }
  if (prec == QC_PREC_BF16X3) {
    set_error("qc_run_circuit: BF16x3 products keep about 16 significant bits, too few for 1e-5");
    return QC_ERR_UNSUPPORTED;
  }
  if (prec != QC_PREC_NATIVE && prec != QC_PREC_TF32X3 && prec != QC_PREC_AUTO) {
    set_error("qc_run_circuit: unknown precision mode %d", int(prec));
    return QC_ERR_INVALID_ARG;
  }
  if (mode == QC_RUN_PER_GATE) return run_per_gate(s, c, params);
  if (mode == QC_RUN_FUSED) return run_fused(s, c, params, prec);
  set_error("qc_run_circuit: unknown mode %d", int(mode));
  return QC_ERR_INVALID_ARG;
}

}  // extern "C"
