// Fused reverse sweep of the adjoint gradient (adjoint_tiles.cu).
#pragma once

#include <vector>

#include "circuit.cuh"
#include "common.cuh"

namespace qcgb {

// Device buffer for the sweep's plan, kept between calls.
struct AdjPlanBuf {
  void* p = nullptr;
  size_t bytes = 0;
  std::vector<char> host;
};

// Smallest register the fused sweep handles (its tile is 2^12 / 2^11 amplitudes).
int adjoint_tiles_min_qubits();

// Applies `rev` (the daggered gates in reverse order) to psi and lambda with tile
// passes; for each op i with grad[i] >= 0 (a rotation with generator gen[i]: 0 X, 1 Y,
// 2 Z) it first records the block sums of Im <lambda|G|psi> into
// gpart[grad[i] * grid + block].  grid (blocks per pass) is returned in *grid_out;
// gpart must hold (max grad + 1) x device_sm_count() doubles.  Stream-ordered.
template <typename R>
qc_status adjoint_reverse_tiles(int n, const std::vector<ResolvedOp>& rev, const std::vector<int>& grad,
                                const std::vector<int>& gen, R* psi, R* lam, cudaStream_t stream, AdjPlanBuf* buf,
                                double* gpart, int* grid_out);

}  // namespace qcgb
