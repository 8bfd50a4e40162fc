// Circuit-level declarations shared by circuit.cu, planner.cu and the fused kernels.
#pragma once

#include <vector>

#include "common.cuh"

namespace qcgb {

enum OpForm { FORM_1Q = 0, FORM_2Q = 1, FORM_CTRL = 2 };

// A gate with its FP64 matrix and bit positions (bit = n-1-qubit).
// FORM_1Q: m is 2x2 on bits[0].  FORM_2Q: m is 4x4 on (bits[0], bits[1]), row index
// 2*b(bits[0]) + b(bits[1]).  FORM_CTRL: m is 2x2 on bits[nq-1], applied where the
// control bits bits[0..nq-2] read cstate (bit j of cstate for control j).
struct ResolvedOp {
  int form;
  int nq;
  int bits[QC_MAX_OP_QUBITS];
  uint32_t cstate;
  double m[32];
};

// k-qubit block: zero bits inserted at pos[0..cnt) (ascending) give a group's base;
// member r of the group sits at base | off[r].
struct KqSpec {
  int cnt;
  int8_t pos[8];
  uint64_t off[128];
};

qc_status resolve_op(const qc_circuit* c, const qc_op& op, const double* params, ResolvedOp* out);
qc_status apply_resolved(qc_state* s, const ResolvedOp& r);
qc_status run_per_gate(qc_state* s, const qc_circuit* c, const double* params);
// drop_global_phase: the constant of every unconditioned phase op is left out (the
// result differs by a global phase; for callers that only form expectation values)
qc_status run_fused(qc_state* s, const qc_circuit* c, const double* params, qc_prec prec,
                    bool drop_global_phase = false);
// complex64 tile passes whose stages run as 32 x 32 blocks on the tensor cores (TF32x3);
// *handled is false (nothing applied) when a stage's op depends on bits outside its slots
qc_status run_tiles_tc(qc_state* s, const std::vector<ResolvedOp>& rops, bool* handled);
qc_status apply_kq_native(qc_state* s, const int* bits, int k, const double* U);
qc_status apply_kq_tf32x3(qc_state* s, const int* bits, int k, const double* U);
// a dense block of k <= 5 qubits (bits[0] the most significant bit of U's index) as one
// tensor-core tile pass of a single stage whose tiles move as boxes; *handled is false
// (nothing applied) where it does not apply (complex128, fewer than 12 qubits, a tile
// that no box plan covers)
qc_status apply_block_tile_tc(qc_state* s, const int* bits, int k, const double* U, bool* handled);

}  // namespace qcgb
