// Placeholder definitions for the fused paths (replaced as they are implemented).
#include "circuit.cuh"

namespace qcgb {
qc_status run_fused(qc_state* s, const qc_circuit* c, const double* params, qc_prec prec) {
  (void)prec;
  return run_per_gate(s, c, params);
}
qc_status apply_kq_tf32x3(qc_state* s, const int* bits, int k, const double* U) {
  (void)s; (void)bits; (void)k; (void)U;
  set_error("TF32x3 fused blocks are not built yet");
  return QC_ERR_UNSUPPORTED;
}
}  // namespace qcgb

extern "C" qc_status qc_adjoint_grad(const qc_circuit*, const double*, int, const char* const*, const double*, int,
                                     qc_dtype, void*, double*, double*) {
  qcgb::set_error("qc_adjoint_grad is not built yet");
  return QC_ERR_UNSUPPORTED;
}
extern "C" qc_status qc_run_batch(const qc_batch*, void*, double*) {
  qcgb::set_error("qc_run_batch is not built yet");
  return QC_ERR_UNSUPPORTED;
}
