// Batched ansatz circuits in one persistent launch (qc_run_ansatz_batch, and the fast
// path of qc_run_batch).
//
// Each circuit is the paper's gate sequence (Sec. 3.2) on its own register: per layer
// RY(t) then RZ(t') on every qubit, then CZ(i, i+1) for i = 0..n-2; the result is
// <psi| sum_{i<n-1} Z_i Z_{i+1} |psi>.
//
// Work split: one block per SM takes circuits from an atomic counter, largest first.
// A circuit of n <= 13 qubits stays in shared memory for its whole run; a larger one
// lives in a per-block global buffer and goes through tile passes of 2^13 amplitudes
// that alternate between the 13 low index bits and the remaining high bits plus enough
// low bits for 512-byte runs, zig-zagging over the layers (layers + 1 passes).  Within
// a tile, register stages of SB bits apply the layer's fused 2x2 gates U = RZ(t') RY(t)
// (up to a global phase); the CZ chain is the diagonal (-1)^popc(i & i>>1)
// and Z_iZ_{i+1} the sign (n-1) - 2 popc((i ^ i>>1) & (2^(n-1)-1)) of index i, both
// folded into the last stage.  The stage width SB (the fusion width) is chosen by the
// autotuner; the launch is recorded once in a CUDA graph and replayed.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace qcgb {

constexpr int kBatchTileBits = 13;  // 64 KiB complex64 tile
constexpr int kBatchMaxN = 20;
constexpr int kBatchMinN = 6;

struct BatchCirc {
  int32_t n;
  int32_t out;      // output slot
  int64_t poff;     // parameter offset
};

__device__ __forceinline__ uint32_t bswz(uint32_t r) {
  uint32_t x = r >> 4;
  return r ^ ((x ^ (x >> 4) ^ (x >> 8)) & 15u);
}

// Fused layer gate of qubit q: U = RZ(t') RY(t) up to its global phase e^{-it'/2}, which
// no output of the batch sees (each circuit yields <sum Z_i Z_i+1>): U' = diag(1, e) RY(t)
// with e = e^{it'}, RY(t) = [[c, -s], [s, c]], (c, s) = cos/sin(t/2).  Row 0 is real;
// row 1 is e times a real combination.  Kept as packed pairs: cc = (c, c), ms = (-s, -s),
// ss = (s, s), er = (Re e, Re e), ei = (-Im e, Im e), so that per pair
//   out0 = cc x0 + ms x1,   t = ss x0 + cc x1,   out1 = er t + ei (t_im, t_re):
// six packed operations, against eight for a general complex 2x2.
struct GateP {
  float2 cc, ms, ss, er, ei;
};

__device__ __forceinline__ GateP layer_gate(const float* p) {
  float s, c, sz, cz;
  sincosf(0.5f * p[0], &s, &c);
  sincosf(p[1], &sz, &cz);
  GateP g;
  g.cc = make_float2(c, c);
  g.ms = make_float2(-s, -s);
  g.ss = make_float2(s, s);
  g.er = make_float2(cz, cz);
  g.ei = make_float2(-sz, sz);
  return g;
}

// One stage over `nbits_local` local bits of a buffer of 2^nl amplitudes (shared memory):
// slots = local bits sl[0..SB), thread groups enumerate the other bits.  Applies the
// fused gate of every slot whose qubit is active, optionally the CZ-chain sign and the
// ZZ accumulation (these need the global index: local index -> global via `gbase` and
// the local->global bit map `gbit`).
template <int SB>
__device__ __forceinline__ void batch_stage(Cplx<float>* buf, int nl, const int8_t (&sl)[SB],
                                            const GateP* gates, const int8_t (&slot_q)[SB], bool phase, bool zz,
                                            int n, uint64_t gbase, const int8_t* gbit, double* zz_acc) {
  constexpr int NA = 1 << SB;
  const int ngroups = 1 << (nl - SB);
  // non-slot local bits in ascending order
  int8_t rest[kBatchTileBits];
  int nr = 0;
  for (int b = 0; b < nl; ++b) {
    bool is_slot = false;
#pragma unroll
    for (int k = 0; k < SB; ++k) is_slot |= (sl[k] == b);
    if (!is_slot) rest[nr++] = int8_t(b);
  }
  uint32_t sw[SB];
#pragma unroll
  for (int k = 0; k < SB; ++k) sw[k] = bswz(1u << sl[k]);
  const uint64_t zmask = (uint64_t(1) << (n - 1)) - 1;
  for (int g = threadIdx.x; g < ngroups; g += blockDim.x) {
    uint32_t r0 = 0;
    for (int k = 0; k < nr; ++k) r0 |= ((uint32_t(g) >> k) & 1u) << rest[k];
    const uint32_t p0 = bswz(r0);
    Cplx<float> v[NA];
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      uint32_t o = 0;
#pragma unroll
      for (int k = 0; k < SB; ++k)
        if ((j >> k) & 1) o ^= sw[k];
      v[j] = buf[p0 ^ o];
    }
#pragma unroll
    for (int k = 0; k < SB; ++k) {
      if (slot_q[k] < 0) continue;
      const GateP& u = gates[slot_q[k]];
      const float2 cc = u.cc, ms = u.ms, ss = u.ss, er = u.er, ei = u.ei;
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        if (j & (1 << k)) continue;
        const int j1 = j | (1 << k);
        const float2 x = f2(v[j]), y = f2(v[j1]);
        const float2 t = __ffma2_rn(cc, y, __fmul2_rn(ss, x));
        v[j] = c2(__ffma2_rn(ms, y, __fmul2_rn(cc, x)));
        v[j1] = c2(__ffma2_rn(ei, make_float2(t.y, t.x), __fmul2_rn(er, t)));
      }
    }
    if (phase || zz) {
      // global index of element j: gbase | map(r0 | slot bits of j)
      uint64_t gr0 = gbase;
      for (int k = 0; k < nr; ++k)
        if ((r0 >> rest[k]) & 1) gr0 |= uint64_t(1) << gbit[rest[k]];
      uint64_t gs[SB];
#pragma unroll
      for (int k = 0; k < SB; ++k) gs[k] = uint64_t(1) << gbit[sl[k]];
      float zg = 0.0f;  // this group's share, added to the FP64 accumulator once
#pragma unroll
      for (int j = 0; j < NA; ++j) {
        uint64_t gi = gr0;
#pragma unroll
        for (int k = 0; k < SB; ++k)
          if ((j >> k) & 1) gi |= gs[k];
        if (phase && (__popcll(gi & (gi >> 1) & zmask) & 1)) {
          v[j].re = -v[j].re;
          v[j].im = -v[j].im;
        }
        if (zz) {
          const float pj = v[j].re * v[j].re + v[j].im * v[j].im;
          zg += pj * float((n - 1) - 2 * __popcll((gi ^ (gi >> 1)) & zmask));
        }
      }
      if (zz) *zz_acc += double(zg);
    }
#pragma unroll
    for (int j = 0; j < NA; ++j) {
      uint32_t o = 0;
#pragma unroll
      for (int k = 0; k < SB; ++k)
        if ((j >> k) & 1) o ^= sw[k];
      buf[p0 ^ o] = v[j];
    }
  }
}

// Applies one layer's gates on the local bits of a buffer: the local bits are split
// into stages of SB; `qubit_of_local[b]` is the qubit of local bit b, or -1 if this
// pass applies no gate there.  The CZ phase / ZZ readout go into the last stage.
template <int SB>
__device__ void batch_layer_on_buffer(Cplx<float>* buf, int nl, const int8_t* qubit_of_local, const GateP* gates,
                                      bool phase, bool zz, int n, uint64_t gbase, const int8_t* gbit,
                                      double* zz_acc) {
  // local bits with gates, in order
  int8_t act[kBatchTileBits];
  int na = 0;
  for (int b = 0; b < nl; ++b)
    if (qubit_of_local[b] >= 0) act[na++] = int8_t(b);
  const int nst = na > 0 ? (na + SB - 1) / SB : 1;
  for (int st = 0; st < nst; ++st) {
    int8_t sl[SB], sq[SB];
    int used = 0;
    for (int k = 0; k < SB && st * SB + k < na; ++k) {
      sl[k] = act[st * SB + k];
      sq[k] = qubit_of_local[sl[k]];
      ++used;
    }
    // pad the stage with other local bits (no gate)
    for (int b = 0; used < SB && b < nl; ++b) {
      bool taken = false;
      for (int k = 0; k < used; ++k) taken |= (sl[k] == b);
      if (!taken) {
        sl[used] = int8_t(b);
        sq[used] = -1;
        ++used;
      }
    }
    const bool last = st == nst - 1;
    batch_stage<SB>(buf, nl, sl, gates, sq, phase && last, zz && last, n, gbase, gbit, zz_acc);
    __syncthreads();
  }
}

// MINB: blocks per SM the register budget is sized for (each holds a 64 KiB tile)
template <int SB, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_batch(const BatchCirc* __restrict__ circs, int ncirc, int layers, const float* __restrict__ params,
            unsigned* __restrict__ counter, float2* __restrict__ scratch, size_t scratch_per_block,
            double* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cplx<float>* tile = reinterpret_cast<Cplx<float>*>(smem_raw);  // 2^13 amplitudes
  __shared__ GateP gates[kBatchMaxN], gates2[kBatchMaxN];
  __shared__ int8_t qol[kBatchTileBits], gbit[kBatchTileBits];
  __shared__ int s_idx;
  __shared__ double red[32];
  Cplx<float>* gstate = reinterpret_cast<Cplx<float>*>(scratch + size_t(blockIdx.x) * scratch_per_block);
  for (;;) {
    if (threadIdx.x == 0) s_idx = int(atomicAdd(counter, 1u));
    __syncthreads();
    const int idx = s_idx;
    if (idx >= ncirc) break;
    const BatchCirc C = circs[idx];
    const int n = C.n;
    const float* p = params + C.poff;
    double zz = 0.0;
    if (n <= kBatchTileBits) {
      // whole state in shared memory: |0...0>
      for (int i = threadIdx.x; i < (1 << n); i += blockDim.x) tile[i] = Cplx<float>{0.f, 0.f};
      __syncthreads();
      if (threadIdx.x == 0) tile[bswz(0)] = Cplx<float>{1.f, 0.f};
      if (threadIdx.x < kBatchTileBits) {
        qol[threadIdx.x] = threadIdx.x < n ? int8_t(n - 1 - threadIdx.x) : int8_t(-1);
        gbit[threadIdx.x] = int8_t(threadIdx.x);
      }
      for (int l = 0; l < layers; ++l) {
        __syncthreads();
        for (int q = threadIdx.x; q < n; q += blockDim.x) gates[q] = layer_gate(p + l * 2 * n + 2 * q);
        __syncthreads();
        batch_layer_on_buffer<SB>(tile, n, qol, gates, true, l == layers - 1, n, 0, gbit, &zz);
      }
    } else {
      // global state, two tile passes per layer
      const uint64_t N = uint64_t(1) << n;
      for (uint64_t i = threadIdx.x; i < N; i += blockDim.x) gstate[i] = Cplx<float>{0.f, 0.f};
      __syncthreads();
      if (threadIdx.x == 0) gstate[0] = Cplx<float>{1.f, 0.f};
      __threadfence_block();
      const int h = n - kBatchTileBits;  // high bits for pass B
      const int lowB = kBatchTileBits - h;  // low bits kept in pass B
      // Zig-zag over the layers: pass pp (0 .. layers) takes the low tile (pass A, the 13
      // low index bits) for even pp and the high tile (pass B) for odd pp, and applies
      // the second part of layer pp - 1 (its gates on this tile's qubits, then its CZ
      // chain, which follows the other part done by the previous pass) and the first part
      // of layer pp.  layers + 1 passes over the state instead of two per layer.
      for (int pp = 0; pp <= layers; ++pp) {
        const int pass = pp & 1;
        const int l0 = pp - 1, l1 = pp;
        __syncthreads();
        for (int q = threadIdx.x; q < n; q += blockDim.x) {
          if (l0 >= 0) gates[q] = layer_gate(p + l0 * 2 * n + 2 * q);
          if (l1 < layers) gates2[q] = layer_gate(p + l1 * 2 * n + 2 * q);
        }
        {
          // local bit -> global bit map and the qubit each local bit carries a gate for
          if (threadIdx.x < kBatchTileBits) {
            const int b = threadIdx.x;
            if (pass == 0) {
              gbit[b] = int8_t(b);
              qol[b] = int8_t(n - 1 - b);
            } else {
              gbit[b] = b < lowB ? int8_t(b) : int8_t(kBatchTileBits + (b - lowB));
              qol[b] = b < lowB ? int8_t(-1) : int8_t(n - 1 - (kBatchTileBits + (b - lowB)));
            }
          }
          __syncthreads();
          const int ntiles = 1 << h;
          for (int t = 0; t < ntiles; ++t) {
            // tile t: pass 0 -> high bits = t; pass 1 -> bits lowB..12 = t
            uint64_t gbase;
            if (pass == 0)
              gbase = uint64_t(t) << kBatchTileBits;
            else
              gbase = uint64_t(t) << lowB;
            {
              // neighbouring amplitude pairs as 16-byte loads, CH of them issued before
              // their stores
              constexpr int PER = (1 << (kBatchTileBits - 1)) / NT;
              constexpr int CH = PER < 8 ? PER : 8;
#pragma unroll
              for (int k0 = 0; k0 < PER; k0 += CH) {
                float4 buf[CH];
#pragma unroll
                for (int k = 0; k < CH; ++k) {
                  const uint32_t r = 2u * (threadIdx.x + (k0 + k) * NT);
                  const uint64_t gi = gbase | (pass == 0 ? uint64_t(r)
                                                        : (uint64_t(r & ((1u << lowB) - 1)) |
                                                           (uint64_t(r >> lowB) << kBatchTileBits)));
                  buf[k] = reinterpret_cast<const float4*>(gstate)[gi >> 1];
                }
#pragma unroll
                for (int k = 0; k < CH; ++k) {
                  const uint32_t r = 2u * (threadIdx.x + (k0 + k) * NT);
                  const uint32_t ps = bswz(r);
                  tile[ps] = Cplx<float>{buf[k].x, buf[k].y};
                  tile[ps ^ 1u] = Cplx<float>{buf[k].z, buf[k].w};
                }
              }
            }
            __syncthreads();
            if (l0 >= 0)
              batch_layer_on_buffer<SB>(tile, kBatchTileBits, qol, gates, true, l0 == layers - 1, n, gbase, gbit,
                                        &zz);
            if (l1 < layers)
              batch_layer_on_buffer<SB>(tile, kBatchTileBits, qol, gates2, false, false, n, gbase, gbit, &zz);
            {
              constexpr int PER = (1 << (kBatchTileBits - 1)) / NT;
#pragma unroll
              for (int k = 0; k < PER; ++k) {
                const uint32_t r = 2u * (threadIdx.x + k * NT);
                const uint64_t gi = gbase | (pass == 0 ? uint64_t(r)
                                                      : (uint64_t(r & ((1u << lowB) - 1)) |
                                                         (uint64_t(r >> lowB) << kBatchTileBits)));
                const uint32_t ps = bswz(r);
                const Cplx<float> a = tile[ps], b = tile[ps ^ 1u];
                reinterpret_cast<float4*>(gstate)[gi >> 1] = make_float4(a.re, a.im, b.re, b.im);
              }
            }
            __syncthreads();
          }
        }
      }
    }
    // block reduction of the ZZ value (FP64)
    double v = double(zz);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
      double w = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
      if (threadIdx.x == 0) out[C.out] = w;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// host: plan cache, autotuner, CUDA graph
// ---------------------------------------------------------------------------
// Launch shapes the autotuner chooses from: register-stage width SB (the fusion width:
// 2^SB amplitudes per thread per stage) and threads per block.
struct BatchShape {
  int sb, nt, minb;
};
constexpr BatchShape kBatchShapes[] = {{4, 256, 2}, {4, 128, 3}, {5, 128, 2}};
constexpr int kNumBatchShapes = int(sizeof(kBatchShapes) / sizeof(kBatchShapes[0]));

template <int SH>
struct ShapeKernel {
  static constexpr BatchShape S = kBatchShapes[SH];
  static constexpr auto fn = k_batch<S.sb, S.nt, S.minb>;
};

template <int SH>
static int batch_blocks_per_sm(size_t smem) {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ShapeKernel<SH>::fn, kBatchShapes[SH].nt, smem);
  return b < 1 ? 1 : b;
}


struct BatchPlan {
  std::string key;
  int device = -1;
  int shape = 0;
  int grid_of[kNumBatchShapes] = {};
  BatchCirc* d_circs = nullptr;
  unsigned* d_counter = nullptr;
  float2* d_scratch = nullptr;
  size_t scratch_per_block = 0;
  int ncirc = 0, layers = 0;
  const float* params = nullptr;
  double* out = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t capture = nullptr;
};
static std::mutex g_batch_mu;
static BatchPlan g_batch;
static std::map<std::string, int> g_tuned;  // autotuner results (fusion width SB)

static void free_plan(BatchPlan& p) {
  if (p.exec) cudaGraphExecDestroy(p.exec);
  if (p.d_circs) cudaFree(p.d_circs);
  if (p.d_counter) cudaFree(p.d_counter);
  if (p.d_scratch) cudaFree(p.d_scratch);
  if (p.capture) cudaStreamDestroy(p.capture);
  p = BatchPlan();
}

static qc_status launch_batch(const BatchPlan& p, int shape, cudaStream_t stream) {
  const size_t smem = sizeof(Cplx<float>) << kBatchTileBits;
  cudaError_t e = cudaMemsetAsync(p.d_counter, 0, sizeof(unsigned), stream);
  if (e != cudaSuccess) return check_cuda(e, "batch counter reset");
  const unsigned grid = unsigned(p.grid_of[shape]);
  const unsigned nt = unsigned(kBatchShapes[shape].nt);
#define QC_BATCH_LAUNCH(SH)                                                                                  \
  QC_COUNT(), ShapeKernel<SH>::fn<<<grid, nt, smem, stream>>>(p.d_circs, p.ncirc, p.layers, p.params,        \
                                                               p.d_counter, p.d_scratch, p.scratch_per_block, \
                                                               p.out)
  switch (shape) {
    case 0: QC_BATCH_LAUNCH(0); break;
    case 1: QC_BATCH_LAUNCH(1); break;
    default: QC_BATCH_LAUNCH(2); break;
  }
#undef QC_BATCH_LAUNCH
  return check_launch("batch kernel");
}

// Autotuner: times each launch shape (fusion width SB, block size) once on the real
// batch (CUDA events) and keeps the fastest; results are kept per (GPU, workload shape)
// and, if QC_AUTOTUNE_CACHE names a file, appended to it as "key shape" lines and read
// back by later processes.
static int autotune_shape(const BatchPlan& p, cudaStream_t stream, const std::string& key) {
  auto it = g_tuned.find(key);
  if (it != g_tuned.end()) return it->second;
  const char* path = getenv("QC_AUTOTUNE_CACHE");
  if (path) {
    FILE* f = fopen(path, "r");
    if (f) {
      char k[512];
      int v;
      while (fscanf(f, "%511s %d", k, &v) == 2)
        if (key == k && v >= 0 && v < kNumBatchShapes) {
          fclose(f);
          g_tuned[key] = v;
          return v;
        }
      fclose(f);
    }
  }
  int best = 0;
  float best_ms = 1e30f;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int sh = 0; sh < kNumBatchShapes; ++sh) {
    cudaEventRecord(e0, stream);
    if (launch_batch(p, sh, stream) != QC_OK) continue;
    cudaEventRecord(e1, stream);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = sh;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g_tuned[key] = best;
  if (path) {
    FILE* f = fopen(path, "a");
    if (f) {
      fprintf(f, "%s %d\n", key.c_str(), best);
      fclose(f);
    }
  }
  return best;
}

static int g_last_batch_sb = 0;

}  // namespace qcgb

using namespace qcgb;

extern "C" int qc_batch_fusion_width(void) { return g_last_batch_sb; }

extern "C" qc_status qc_run_ansatz_batch(const qc_ansatz_batch* b, void* stream_v, double* dev_out) {
  clear_error();
  if (!b || b->count < 0 || b->layers < 0 || (b->count > 0 && (!b->n || !b->param_offset || !b->dev_params || !dev_out))) {
    set_error("qc_run_ansatz_batch: invalid arguments");
    return QC_ERR_INVALID_ARG;
  }
  if (b->count == 0) return QC_OK;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_v);
  int maxn = 0;
  for (int i = 0; i < b->count; ++i) {
    const int n = b->n[i];
    if (n < kBatchMinN || n > kBatchMaxN) {
      set_error("qc_run_ansatz_batch: circuit %d has n=%d (supported %d..%d)", i, n, kBatchMinN, kBatchMaxN);
      return QC_ERR_UNSUPPORTED;
    }
    if (b->param_offset[i] < 0 || b->param_offset[i] + int64_t(b->layers) * 2 * n > b->nparams) {
      set_error("qc_run_ansatz_batch: parameters of circuit %d exceed nparams", i);
      return QC_ERR_INVALID_ARG;
    }
    maxn = std::max(maxn, n);
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, dev);
  // the key: device, shape of the batch, and the device buffers it reads and writes
  std::string key = std::string(prop.name) + "|" + std::to_string(b->count) + "|" + std::to_string(b->layers);
  {
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < b->count; ++i) {
      h = (h ^ uint64_t(b->n[i])) * 1099511628211ull;
      h = (h ^ uint64_t(b->param_offset[i])) * 1099511628211ull;
    }
    key += "|" + std::to_string(h);
  }
  for (char& ch : key)
    if (ch == ' ') ch = '_';
  const std::string full_key = key + "|" + std::to_string(reinterpret_cast<uintptr_t>(b->dev_params)) + "|" +
                               std::to_string(reinterpret_cast<uintptr_t>(dev_out));
  std::lock_guard<std::mutex> lock(g_batch_mu);
  if (g_batch.key != full_key || g_batch.device != dev) {
    free_plan(g_batch);
    BatchPlan& p = g_batch;
    p.key = full_key;
    p.device = dev;
    p.ncirc = b->count;
    p.layers = b->layers;
    p.params = b->dev_params;
    p.out = dev_out;
    // largest circuits first
    std::vector<BatchCirc> circs(b->count);
    for (int i = 0; i < b->count; ++i) circs[i] = BatchCirc{b->n[i], i, b->param_offset[i]};
    std::stable_sort(circs.begin(), circs.end(), [](const BatchCirc& x, const BatchCirc& y) { return x.n > y.n; });
    const size_t smem = sizeof(Cplx<float>) << kBatchTileBits;
    qc_status st = QC_OK;
    for (auto fn : {ShapeKernel<0>::fn, ShapeKernel<1>::fn, ShapeKernel<2>::fn})
      if (st == QC_OK)
        st = check_cuda(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)),
                        "batch smem");
    p.grid_of[0] = prop.multiProcessorCount * batch_blocks_per_sm<0>(smem);
    p.grid_of[1] = prop.multiProcessorCount * batch_blocks_per_sm<1>(smem);
    p.grid_of[2] = prop.multiProcessorCount * batch_blocks_per_sm<2>(smem);
    const int max_grid = std::max(p.grid_of[0], std::max(p.grid_of[1], p.grid_of[2]));
    p.scratch_per_block = maxn > kBatchTileBits ? (size_t(1) << maxn) : 1;
    if (st == QC_OK) st = check_cuda(cudaMalloc(&p.d_circs, sizeof(BatchCirc) * circs.size()), "batch table");
    if (st == QC_OK) st = check_cuda(cudaMalloc(&p.d_counter, 256), "batch counter");
    if (st == QC_OK)
      st = check_cuda(cudaMalloc(&p.d_scratch, sizeof(float2) * p.scratch_per_block * max_grid), "batch scratch");
    if (st == QC_OK)
      st = check_cuda(cudaMemcpy(p.d_circs, circs.data(), sizeof(BatchCirc) * circs.size(), cudaMemcpyHostToDevice),
                      "batch table upload");
    if (st != QC_OK) {
      free_plan(g_batch);
      return st;
    }
    p.shape = autotune_shape(p, stream, key);
    // record [counter reset, kernel] once in a CUDA graph on a private stream
    st = check_cuda(cudaStreamCreateWithFlags(&p.capture, cudaStreamNonBlocking), "capture stream");
    cudaGraph_t graph = nullptr;
    if (st == QC_OK) st = check_cuda(cudaStreamBeginCapture(p.capture, cudaStreamCaptureModeThreadLocal), "capture");
    if (st == QC_OK) {
      qc_status ls = launch_batch(p, p.shape, p.capture);
      cudaError_t e = cudaStreamEndCapture(p.capture, &graph);
      st = ls != QC_OK ? ls : check_cuda(e, "end capture");
    }
    if (st == QC_OK) st = check_cuda(cudaGraphInstantiate(&p.exec, graph, 0), "graph instantiate");
    if (graph) cudaGraphDestroy(graph);
    if (st != QC_OK) {
      free_plan(g_batch);
      return st;
    }
  }
  g_last_batch_sb = kBatchShapes[g_batch.shape].sb;
  QC_COUNT();  // the graph's kernel
  return check_cuda(cudaGraphLaunch(g_batch.exec, stream), "batch graph launch");
}
