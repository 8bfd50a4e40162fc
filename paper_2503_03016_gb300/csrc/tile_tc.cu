// Tile passes with tensor-core stages (QC_PREC_TF32X3, complex64).
//
// A tile of 2^12 amplitudes (the pass's bit set B, as for the CUDA-core passes) goes
// through the pass's stages.  A stage owns 5 of the tile's bits (its slots); every op of
// the stage acts on, and is conditioned on, slot bits only, so the stage is one 32 x 32
// block U_s = G_k ... G_1 (Sec. 3.2's U' of each gate, embedded on the slots and
// multiplied on the host in FP64).  With the 2^7 combinations of the tile's other bits
// as rows, a stage is the real GEMM D = A B (A[r][2c + ri] = (re, im) of block index c
// in row r; B the real form of U_s^T), M = 128, N = K = 64, with the TF32 split
// a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi (a_hi = RN_tf32(a), a_lo = a - a_hi, which the
// tensor cores read to TF32 precision; B split with round-to-nearest on the host),
// accumulated in FP32.
//
// Kernel: one CTA per SM, 288 threads: two epilogue groups of 128 threads (warps 0-3
// and 4-7), each working on its own tile, and one MMA warp (warp 8) whose first lane
// issues every tcgen05.mma.  Thread r of a group owns row r of its tile's current
// stage, which is TMEM lane r: it reads its row's 32 amplitudes from the group's tile
// in shared memory (byte offsets formed in Gray-code order, one XOR each, and kept for
// the write-back), splits them and writes A_hi and A_lo into TMEM (tcgen05.st), so A
// never passes through shared memory as an operand (the tensor cores read only B
// there), and arrives on the group's mbarrier of that half of the columns: the MMA warp
// starts the K steps of the first half while the second half is being gathered.  The MMA warp
// issues the stage's 16 products (A from TMEM, B from shared memory) into two FP32
// accumulators and commits them to the group's mbarrier.  The group reads its rows of
// D back (tcgen05.ld), adds the two partial sums, writes the outputs into the tile at
// this stage's positions (the transposition between stages' row and slot bits) and,
// after a group barrier, gathers the next stage's rows.  While one group's products
// run on the tensor cores the other group moves its tile, so the tensor pipe is fed
// from both.  A group's memory traffic also runs in the windows where it waits for its
// products: the write-back of its previous tile (16-byte stores from shared memory)
// during stage 0, the load of its next tile (cp.async into the buffer just written
// back) during the following stages.
//
// Products and accumulation: per K step, a_hi [b_hi | b_lo] is one product of N = 128
// (the image holds each K slice as B_hi's rows followed by B_lo's, one 128-row operand),
// whose first 64 columns accumulate the large products a_hi b_hi and the other 64 the
// small products a_hi b_lo, and a_lo b_hi (N = 64) adds into the second accumulator: 16
// products per stage instead of 24 of N = 64, which the tensor cores run at half the
// rate of N = 128.  The tensor cores truncate the FP32 accumulator toward zero after each
// product step, which a circuit's stages compound into a norm loss; the large and small
// products are kept apart and added on the CUDA cores with round-to-nearest, and the
// passes restore the register's norm (below).
//
// B images (host-built, already in the K-major 128-byte-swizzled layout, 32 KiB per
// stage) stream through two shared-memory buffers by bulk copies with mbarrier
// transaction counts; buffer (x & 1) serves the x-th stage execution of the CTA, and
// the next image is loaded into the other buffer as soon as both groups have issued
// stage x (both then have finished x - 1, whose products read that buffer).  Passes
// with one or two stages keep them resident.
//
// Every wait is bounded and also watches a CTA-wide abort word: a wait that runs out
// sets it, so every other waiter leaves too (the group votes on the outcome in a
// barrier, so the group's threads leave together); before TMEM is released the MMA thread commits and waits
// (bounded) for its outstanding products, and every bulk copy in flight is waited for.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <complex>
#include <mutex>
#include <vector>

#include "circuit.cuh"
#include "common.cuh"
#include "kernels.cuh"
#include "tc_common.cuh"
#include "tiles.cuh"

namespace qcgb {

constexpr int kTtM = 12;                        // tile bits
constexpr int kTtL = 4;                         // lowest index bits always in the tile
constexpr int kTtSB = 5;                        // stage (block) bits
constexpr int kTtRows = 1 << (kTtM - kTtSB);    // 128 rows = MMA M = TMEM lanes
constexpr int kTtGroups = 2;                    // tiles in flight per CTA
constexpr int kTtGroupThreads = kTtRows;        // one thread per row
constexpr int kTtThreads = kTtGroups * kTtGroupThreads + 32;  // + the MMA warp
constexpr int kTtMmaWarp = kTtGroups * kTtGroupThreads / 32;
constexpr int kTtCols = 2 << kTtSB;             // 64 real columns (K = N)
constexpr int kTtBregion = kTtCols * 128;       // one 32-column K slice of B_hi or B_lo: 8 KiB
// B image of one stage, 32 KiB: per K slice s, B_hi's 64 rows then B_lo's 64 rows (16 KiB
// at s * 16 KiB), so that the slice is also one 128-row operand [B_hi; B_lo]
constexpr int kTtBimg = 2 * 2 * kTtBregion;
constexpr int kTtImgFloats = kTtBimg / 4;
constexpr int kTtTileBytes = (1 << kTtM) * 8;   // complex64 tile: 32 KiB
constexpr int kTtMaxStages = kMaxPassOps;
// Deferred phase factors.  The non-slot part of a phase op conditioned on at most one
// slot bit -- exp(i sum beta_b b_b) over row and tile-number bits, applied where the
// slot bit has its value -- commutes with the rest of its stage when no later op of
// the stage acts densely on that slot, so it is applied after the stage's product: per
// output (row r, block index c) one factor F(r, c) = F0(r) prod_k G_k,c_k(r), each
// factor a row table (128 entries) times a per-tile value from three tile-number chunk
// tables (3 x 256 entries), all FP64-built on the host and rounded to FP32.
constexpr int kTtMaxDefStage = 11;  // factors per stage: unconditioned + 5 slots x 2 values
constexpr int kTtMaxDefPass = 64;   // factors per pass (per-tile values in shared memory)
// stage cuts searched this many stages ahead (each stage block costs a full round of
// transposition and products, so fewer blocks pay more than the host search costs)
constexpr int kTtStageLookahead = 2;
constexpr int kTtHi = 1 << (kTtM - kTtL);       // 128-byte runs per tile
// TMEM columns of a group: A_hi [0, 64), A_lo [64, 128), accumulators [128, 256)
constexpr int kTmemPerGroup = 256;
constexpr int kTmemCols = kTtGroups * kTmemPerGroup;  // 512

struct TcStage {
  int32_t img;          // index of the stage's B image
  uint32_t swz[5];      // byte offset in the swizzled tile of block-index bit k
  int8_t lane_bit[7];   // local bit receiving bit k of the row index
  int8_t ndef;          // deferred phase factors of the stage (0: none)
  int32_t def0;         // global index of its first factor (row and tile-number tables)
  int8_t dkey[kTtMaxDefStage];  // per factor: -1 unconditioned, else 2 slot + slot value
  int8_t pad;
};
static_assert(sizeof(TcStage) == 48, "TcStage must be 48 bytes");

constexpr size_t kTtSmem = 1024 /* alignment slack */ + 2 * kTtBimg + 2 * kTtGroups * kTtTileBytes +
                           kTtHi * sizeof(uint64_t) + kTileNumberTab * sizeof(uint64_t) +
                           kTtMaxStages * sizeof(TcStage) + 256;

// A pass whose tile moves as boxes of the state for the tensor memory accelerator: the
// state's index bits grouped into at most 5 dimensions of consecutive bits (dimension
// 0: bits 0..3, 16 amplitudes = 128 bytes); a dimension whose bits all lie in the tile
// is copied whole, any other one element at a time.  Tile bits inside such a
// dimension are box coordinates: the tile is 2^nc boxes (at least 1 KiB each), box j
// at byte j * (tile bytes >> nc) with the coordinate bits of j, so the tile's local
// bits are dimension 0, the whole dimensions' bits in ascending order, then the
// coordinate bits.  Boxes land in shared memory with the 128-byte swizzle (16-byte
// chunk c of 128-byte row r at chunk c ^ (r & 7)).
struct TcTma {
  int32_t tma;         // 1: tiles move by cp.async.bulk.tensor, 0: by cp.async
  int8_t start[5];     // first index bit of dimension d
  int8_t len[5];       // its bits (0: a padding dimension of size 1)
  int8_t tile[5];      // 1: dimension d is copied whole (coordinate 0)
  int8_t nc;           // tile bits taken as box coordinates (at most kTtMaxCoordBits)
  int8_t cdim[5];      // dimension of coordinate bit q
  int8_t coff[5];      // its bit within that dimension
};
// Boxes of at least 8 KiB: with 16 boxes of 2 KiB per tile the one pass of the 28-qubit
// brickwork that took them ran slower than with per-amplitude copies
constexpr int kTtMaxCoordBits = 2;

// Norm restoration across the passes of a circuit.  The tensor cores truncate their
// FP32 accumulator toward zero, so every stage shrinks the amplitudes slightly (a
// 28-qubit brickwork: about 9e-6 of norm in all, nearly all of its error), while a
// unitary circuit keeps the norm exactly.  The first pass sums the norm of its input,
// every pass the norm of its output (per block, in a fixed order, into norms[]), and a
// later pass multiplies each amplitude it loads by sqrt(input norm / previous output
// norm), formed in FP64 from those sums.
struct TcNorm {
  int32_t first;        // this pass sums the circuit's input norm
  int32_t apply;        // this pass scales its input (a previous pass wrote out_prev)
  int32_t nblocks;      // blocks of the previous pass (partials in in_part / out_prev)
  int32_t pad;
  double* in_part;      // [nblocks] input norm per block (written by the first pass)
  double* out_prev;     // [nblocks] output norm per block of the previous pass
  double* out_cur;      // [gridDim.x] output norm per block of this pass
};

// byte offset of local index u in a tile with the 128-byte swizzle (XOR-linear in u)
__host__ __device__ __forceinline__ uint32_t tma_swz_bytes(uint32_t u) {
  return ((u >> 4) << 7) | ((((u >> 1) ^ (u >> 4)) & 7u) << 4) | ((u & 1u) << 3);
}

// bounded mbarrier wait that also gives up when another thread has set *abort
__device__ __forceinline__ bool mbar_wait_ab(uint32_t bar, uint32_t parity, const volatile int* abort) {
  for (long long it = 0; it < kTcSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 63) == 63 && *abort) return false;
  }
  return false;
}

// one bulk copy global -> shared, completion counted in bytes on `bar`
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// barrier of one epilogue group (named barrier 1 + g, all its threads), with an OR vote
__device__ __forceinline__ bool group_sync_or(int g, bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"(v ? 1u : 0u), "r"(1 + g), "n"(kTtGroupThreads)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(1 + g), "n"(kTtGroupThreads) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
      "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
      "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}

__device__ __forceinline__ float2 lds2(uint32_t addr) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(addr));
  return v;
}
__device__ __forceinline__ void sts2(uint32_t addr, float2 v) {
  asm volatile("st.shared.v2.f32 [%0], {%1, %2};\n" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}

// D (+)= A B with A in TMEM (M = 128 lanes, K = 8 TF32 columns from a_tmem), B from
// shared memory (descriptor)
__device__ __forceinline__ void tc_mma_ts(uint32_t dtm, uint32_t atm, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(dtm),
      "r"(atm), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

// tiles of group g of this CTA: 2 blockIdx + g + k (2 gridDim), k = 0, 1, ...
__device__ __forceinline__ uint32_t group_tiles(uint64_t ntiles, int g) {
  const uint64_t t0 = 2 * uint64_t(blockIdx.x) + g, step = 2 * uint64_t(gridDim.x);
  return t0 < ntiles ? uint32_t((ntiles - 1 - t0) / step + 1) : 0u;
}

// coordinates of tile t's box: its base index's bits in the dimensions outside the tile
__device__ __forceinline__ void tma_coords(uint64_t base, const TcTma& tm, int32_t (&c)[5]) {
#pragma unroll
  for (int d = 0; d < 5; ++d)
    c[d] = tm.tile[d] || tm.len[d] == 0 ? 0 : int32_t((base >> tm.start[d]) & ((uint64_t(1) << tm.len[d]) - 1));
}

// the coordinates of box j of a tile whose first box is at c (every index static, so
// that cj stays in registers)
__device__ __forceinline__ void tma_box_coords(const TcTma& tm, const int32_t (&c)[5], uint32_t j, int32_t (&cj)[5]) {
#pragma unroll
  for (int d = 0; d < 5; ++d) cj[d] = c[d];
#pragma unroll
  for (int q = 0; q < kTtMaxCoordBits; ++q)
    if (q < tm.nc && ((j >> q) & 1u)) {
#pragma unroll
      for (int d = 0; d < 5; ++d)
        if (tm.cdim[q] == d) cj[d] += int32_t(1) << tm.coff[q];
    }
}

// the tile's boxes -> shared memory at dst, completion counted in bytes on `bar`
__device__ __forceinline__ void tma_load_tile(uint32_t dst, const CUtensorMap* map, const int32_t (&c)[5],
                                              uint32_t bar, const TcTma& tm) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(uint32_t(kTtTileBytes))
               : "memory");
  const uint32_t nb = 1u << tm.nc, bytes = uint32_t(kTtTileBytes) >> tm.nc;
  for (uint32_t j = 0; j < nb; ++j) {
    int32_t cj[5];
    tma_box_coords(tm, c, j, cj);
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5, %6}], [%7];\n" ::"r"(dst + j * bytes),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(cj[0]), "r"(cj[1]), "r"(cj[2]), "r"(cj[3]), "r"(cj[4]), "r"(bar)
        : "memory");
  }
}

// the tile's boxes from shared memory at src -> the state, as one bulk group
__device__ __forceinline__ void tma_store_tile(uint32_t src, const CUtensorMap* map, const int32_t (&c)[5],
                                               const TcTma& tm) {
  const uint32_t nb = 1u << tm.nc, bytes = uint32_t(kTtTileBytes) >> tm.nc;
  for (uint32_t j = 0; j < nb; ++j) {
    int32_t cj[5];
    tma_box_coords(tm, c, j, cj);
    asm volatile(
        "cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4, %5}], [%6];\n" ::"l"(
            reinterpret_cast<uint64_t>(map)),
        "r"(cj[0]), "r"(cj[1]), "r"(cj[2]), "r"(cj[3]), "r"(cj[4]), "r"(src + j * bytes)
        : "memory");
  }
  asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// DEFER: the pass has stages with deferred phase factors (rowtab, gtab; the pass's
// factors are global indices [P.pool0, P.pool0 + P.npool))
template <bool TMA, bool DEFER>
__global__ void __launch_bounds__(kTtThreads, 1) k_tile_pass_tc(float* __restrict__ amps, const TilePass P,
                                                                 const TcStage* __restrict__ stages,
                                                                 const float* __restrict__ imgs,
                                                                 int* __restrict__ status,
                                                                 const __grid_constant__ CUtensorMap tmap,
                                                                 const TcTma tm, const TcNorm nrm,
                                                                 const float2* __restrict__ rowtab,
                                                                 const float2* __restrict__ gtab) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* bbuf = base;  // two stage images
  Cplx<float>* tiles = reinterpret_cast<Cplx<float>*>(bbuf + 2 * kTtBimg);  // [group][buffer]
  uint64_t* hioff = reinterpret_cast<uint64_t*>(bbuf + 2 * kTtBimg + 2 * kTtGroups * kTtTileBytes);
  uint64_t* tnt = hioff + kTtHi;  // tile number -> base
  TcStage* sst = reinterpret_cast<TcStage*>(tnt + kTileNumberTab);
  // mbarriers: full[2][2] (half h of the group's rows' columns is in TMEM: one arrival
  // per row), done[2] (products complete),
  // bfull[2] (B image landed), fin (the MMA thread's last products), bfree[2] (the
  // products of the last execution that read B buffer b are complete), tload[2] (a
  // group's tile landed)
  uint64_t* bars = reinterpret_cast<uint64_t*>(sst + kTtMaxStages);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 13);
  volatile int* abort_word = reinterpret_cast<volatile int*>(tmem_slot + 1);
  __shared__ int8_t sbits[16], ssorted[16];  // the tile's bits in local order / ascending
  __shared__ int8_t srbit[16];                // relabeled SWAPs: see TilePass::rbit
  __shared__ float s_fac;                                 // this pass's input scale
  __shared__ double s_norm[2][kTtGroups * kTtGroupThreads];  // per-thread norm sums
  __shared__ float2 s_gfac[DEFER ? kTtGroups : 1][DEFER ? kTtMaxDefPass : 1];  // per-tile factor values
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int m = kTtM, L = kTtL;
  constexpr uint32_t T = 1u << m;
  const int S = P.nstages;

  if (tid == 0) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      sbits[k] = ssorted[k] = P.bits[k];
      srbit[k] = P.rbit[k];
    }
    for (int k = 1; k < m; ++k)  // insertion sort of the m tile bits
      for (int j = k; j > 0 && ssorted[j - 1] > ssorted[j]; --j) {
        const int8_t x = ssorted[j];
        ssorted[j] = ssorted[j - 1];
        ssorted[j - 1] = x;
      }
    for (int b = 0; b < 13; ++b) {
      const uint32_t cnt = b < 4 ? uint32_t(kTtGroupThreads) : 1u;
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bars + b)), "r"(cnt) : "memory");
    }
    *abort_word = 0;
    double f = 1.0;
    if (nrm.apply) {  // fixed-order FP64 sums of the previous partials
      double a = 0.0, b = 0.0;
      for (int i = 0; i < nrm.nblocks; ++i) {
        a += nrm.in_part[i];
        b += nrm.out_prev[i];
      }
      if (a > 0.0 && b > 0.0) f = sqrt(a / b);
    }
    s_fac = float(f);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  for (int i = tid; i < S; i += kTtThreads) sst[i] = stages[P.stage0 + i];
  __syncthreads();
  for (int h = tid; h < kTtHi; h += kTtThreads) {
    uint64_t o = 0;
    for (int k = 0; k < m - L; ++k)
      if ((h >> k) & 1) o |= uint64_t(1) << sbits[L + k];
    hioff[h] = o;
  }
  build_tile_number_tables(tnt, ssorted, m, __ffsll(static_cast<long long>(P.ntiles)) - 1);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t full0 = smem_u32(bars), done0 = smem_u32(bars + 4), bfull0 = smem_u32(bars + 6),
                 fin = smem_u32(bars + 8), bfree0 = smem_u32(bars + 9), tload0 = smem_u32(bars + 11);
  const uint32_t K0 = group_tiles(P.ntiles, 0), K1 = group_tiles(P.ntiles, 1);

  if (warp == kTtMmaWarp) {
    // ------------------------------------------------------------------ MMA warp
    if (lane == 0) {
      constexpr uint32_t idesc = tf32_idesc(kTtRows, kTtCols), idesc2 = tf32_idesc(kTtRows, 2 * kTtCols);
      const bool resident = S <= 2;
      uint32_t bpar = 0, inflight = 0;
      uint32_t fpar_b = 0, freeing = 0;  // bfree[b]: parity of its next phase; a commit not yet waited for
      auto load_b = [&](int b, int s) {
        bulk_load(smem_u32(bbuf + b * kTtBimg), imgs + size_t(sst[s].img) * kTtImgFloats, kTtBimg, bfull0 + 8u * b);
        inflight |= 1u << b;
      };
      if (S > 0) {
        load_b(0, 0);
        if (S == 2) load_b(1, 1);
      }
      uint32_t fpar = 0;  // bit g: parity of group g's next full phase
      bool issued = false, ok = true;
      uint64_t x = 0;  // stage executions of this CTA
      const uint32_t Kmax = K0 > K1 ? K0 : K1;
      for (uint32_t k = 0; k < Kmax && ok; ++k) {
        for (int s = 0; s < S && ok; ++s, ++x) {
          const int b = resident ? s : int(x & 1);
          if ((inflight >> b) & 1u) {
            ok = mbar_wait_ab(bfull0 + 8u * b, (bpar >> b) & 1u, abort_word);
            if (!ok) break;
            bpar ^= 1u << b;
            inflight &= ~(1u << b);
          }
          const uint32_t bimg = smem_u32(bbuf + b * kTtBimg);
          for (int g = 0; g < kTtGroups; ++g) {
            if (k >= (g ? K1 : K0)) continue;
            const uint32_t gb = tmem + uint32_t(g * kTmemPerGroup);
            for (int h = 0; h < 2 && ok; ++h) {
              // the K steps of half h read A columns [32h, 32h + 32) (+ 64): they start
              // as soon as every row has written that half
              ok = mbar_wait_ab(full0 + 8u * (2 * g + h), (fpar >> g) & 1u, abort_word);
              if (!ok) break;
              asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
              // per K step: a_hi [b_hi | b_lo] as one N = 128 product (columns 128..191
              // take a_hi b_hi, 192..255 a_hi b_lo), then a_lo b_hi into 192..255
              for (int ks = 4 * h; ks < 4 * h + 4; ++ks) {
                const uint64_t bd = sw128_desc(bimg + uint32_t(h * 2 * kTtBregion + (ks & 3) * 32), kTcAtom);
                tc_mma_ts(gb + 128u, gb + uint32_t(8 * ks), bd, idesc2, ks == 0 ? 0u : 1u);
                tc_mma_ts(gb + 192u, gb + 64u + uint32_t(8 * ks), bd, idesc, 1u);
              }
            }
            if (!ok) break;
            fpar ^= 1u << g;
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             done0 + 8u * g)
                         : "memory");
            issued = true;
          }
          if (!ok) break;
          if (!resident) {
            // completion of this execution's products frees buffer b
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             bfree0 + 8u * b)
                         : "memory");
            freeing |= 1u << b;
            // the next execution's image goes into the other buffer once the products
            // of the execution before this one (the last to read it) are complete
            const bool more = (s + 1 < S) || (k + 1 < Kmax);
            const int nb = b ^ 1;
            if (more) {
              if ((freeing >> nb) & 1u) {
                ok = mbar_wait_ab(bfree0 + 8u * nb, (fpar_b >> nb) & 1u, abort_word);
                if (!ok) break;
                fpar_b ^= 1u << nb;
                freeing &= ~(1u << nb);
              }
              load_b(nb, s + 1 < S ? s + 1 : 0);
            }
          }
        }
      }
      if (!ok) *abort_word = 1;
      // outstanding products and copies finish before the block leaves (bounded)
      if (issued) {
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(fin)
                     : "memory");
        const volatile int never = 0;
        if (!mbar_wait_ab(fin, 0, &never)) *abort_word = 1;
      }
      for (int b = 0; b < 2; ++b)
        if ((inflight >> b) & 1u) {
          const volatile int never = 0;
          mbar_wait_ab(bfull0 + 8u * b, (bpar >> b) & 1u, &never);
        }
    }
  } else {
    // ------------------------------------------------------------ epilogue groups
    const int g = warp >> 2;                        // group
    const int row = tid & (kTtRows - 1);            // this thread's row = TMEM lane
    const uint32_t Kg = g ? K1 : K0;
    Cplx<float>* buf0 = tiles + size_t(g) * 2 * T;
    const uint32_t ta = tmem + (uint32_t(32 * (warp & 3)) << 16) + uint32_t(g * kTmemPerGroup);
    const uint64_t G2 = 2 * uint64_t(gridDim.x);
    const uint64_t t0 = 2 * uint64_t(blockIdx.x) + g;
    constexpr uint32_t lowmask = (1u << L) - 1;
    uint32_t dpar = 0;
    bool failed = false;
    // this thread's share (elements i = part, part + parts, ... of its row's stride) of
    // the asynchronous load of tile t into dst
    auto prefetch = [&](Cplx<float>* dst, uint64_t t, int part, int parts) {
      const float* src = amps + 2 * tile_base(t, tnt);
      for (uint32_t r = row + uint32_t(part) * kTtGroupThreads; r < T; r += uint32_t(parts) * kTtGroupThreads)
        cp_async_amp<float>(dst + tile_swz(r), src + 2 * (hioff[r >> L] | (r & lowmask)));
    };
    // write-back of tile t from src, two amplitudes (16 bytes) per store
    auto store = [&](const Cplx<float>* src, uint64_t t) {
      const uint64_t tbase = tile_base(t, tnt);
      for (uint32_t e = row; e < T / 2; e += kTtGroupThreads) {
        const uint32_t r = 2 * e;
        const uint64_t gi = tbase | hioff[r >> L] | (r & lowmask);
        const uint32_t p = tile_swz(r);
        st_amp2<float>(amps, gi, src[p], src[p ^ 1u]);
      }
    };
    constexpr bool tma = TMA;
    const bool elect = row == 0;
    const uint32_t tload = tload0 + 8u * g;
    uint32_t nload = 0, nwait = 0;  // (TMA) tile loads issued (elected thread) / waited for
    const float fac = s_fac;
    double nin = 0.0, nout = 0.0;   // this thread's norm sums (input of a first pass, output)
    if (Kg > 0) {
      if (!tma) {
        prefetch(buf0, t0, 0, 1);
      } else if (elect) {
        int32_t c[5];
        tma_coords(tile_base(t0, tnt), tm, c);
        tma_load_tile(smem_u32(buf0), &tmap, c, tload, tm);
        ++nload;
      }
    }
    cp_async_commit();
    // Tile k works in buffer k & 1.  Its write-back is deferred to the wait for the
    // products of stage 0 of tile k + 1, and the load of tile k + 1 (into the buffer
    // just written back) is spread over the waits of the stages after stage 0 of tile k
    // (after the group barrier that ends stage 0), so both overlap the tensor cores.
    for (uint32_t k = 0; k < Kg && !failed; ++k) {
      Cplx<float>* cur = buf0 + (k & 1) * T;
      Cplx<float>* other = buf0 + ((k + 1) & 1) * T;
      const uint32_t curs = smem_u32(cur);  // shared-window address of the tile
      const uint64_t t = t0 + k * G2;
      const bool next = k + 1 < Kg;
      const int nparts = S >= 3 ? 2 : 1;  // load windows: stages 1 .. nparts
      if constexpr (DEFER) {
        // this tile's values of the pass's deferred factors (the previous tile's last
        // stage ended with a group barrier; the barrier below publishes these)
        for (int i = row; i < P.npool; i += kTtGroupThreads) {
          const float2* gt = gtab + size_t(P.pool0 + i) * 768;
          s_gfac[g][i] = cmulf(cmulf(gt[t & 255], gt[256 + ((t >> 8) & 255)]), gt[512 + ((t >> 16) & 255)]);
        }
      }
      if (tma) {
        if (!mbar_wait_ab(tload, k & 1u, abort_word))
          failed = true;
        else
          ++nwait;
        if (group_sync_or(g, failed)) {
          failed = true;
          break;
        }
      } else {
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        group_sync(g);
      }
      bool loaded = false;  // (TMA) the load of tile k + 1 is issued
      auto tma_next = [&]() {
        if (elect && next) {
          // the write-back of tile k - 1 has read `other` before it is refilled
          asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
          int32_t c[5];
          tma_coords(tile_base(t + G2, tnt), tm, c);
          tma_load_tile(smem_u32(other), &tmap, c, tload, tm);
          ++nload;
        }
        loaded = true;
      };
      for (int s = 0; s < S; ++s) {
        const TcStage& st = sst[s];
        uint32_t r0 = 0;
#pragma unroll
        for (int b = 0; b < 7; ++b) r0 |= uint32_t((row >> b) & 1) << st.lane_bit[b];
        uint32_t sw[5];
#pragma unroll
        for (int b = 0; b < 5; ++b) sw[b] = st.swz[b];
        // byte offsets of block indices c = i ^ (i >> 1) (Gray order: one XOR each);
        // formed again for the write-back of this stage's outputs (not kept in
        // registers over the wait, whose window runs the memory traffic)
        const uint32_t off0 = tma ? tma_swz_bytes(r0) : tile_swz(r0) * 8u;
        uint32_t off[32];
        off[0] = off0;
#pragma unroll
        for (int i = 1; i < 32; ++i) off[i] = off[i - 1] ^ sw[(i & 1) ? 0 : (i & 2) ? 1 : (i & 4) ? 2 : (i & 8) ? 3 : 4];
        // this row's 32 amplitudes -> TF32 hi / lo in TMEM (A_hi columns 0..63, A_lo
        // columns 64..127, column 2c + ri); chunk q holds c in [16q, 16q + 16)
        float sin_ = 0.0f;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          uint32_t hi[32], lo[32];
#pragma unroll
          for (int i = 16 * q; i < 16 * q + 16; ++i) {
            const int c = (i ^ (i >> 1)) - 16 * q;
            float2 v = lds2(curs + off[i]);
            if (s == 0) {  // the tile as loaded: its norm (first pass), the pass's scale
              sin_ = fmaf(v.x, v.x, fmaf(v.y, v.y, sin_));
              v.x *= fac;
              v.y *= fac;
            }
            // round to the nearest TF32 value, ties away from zero, in integer arithmetic
            // (the same value as cvt.rna.tf32 for every finite input; amplitudes are far
            // below the overflow range)
            const float hr = __uint_as_float((__float_as_uint(v.x) + 0x1000u) & 0xFFFFE000u);
            const float hm = __uint_as_float((__float_as_uint(v.y) + 0x1000u) & 0xFFFFE000u);
            hi[2 * c] = __float_as_uint(hr);
            hi[2 * c + 1] = __float_as_uint(hm);
            lo[2 * c] = __float_as_uint(v.x - hr);
            lo[2 * c + 1] = __float_as_uint(v.y - hm);
          }
          tmem_st32(ta + uint32_t(32 * q), hi);
          tmem_st32(ta + 64u + uint32_t(32 * q), lo);
          // this half of the row is in TMEM: its K steps may start (one arrival per
          // warp, counting its 32 rows)
          asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
          asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
          __syncwarp();
          if (lane == 0)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], 32;\n" ::"r"(full0 + 8u * (2 * g + q)) : "memory");
        }
        if (s == 0) nin += double(sin_);
        // work for the memory system while the products run
        if (tma) {
          if (s == 0) tma_next();
        } else {
          if (s == 0 && k > 0) store(other, t - G2);
          if (next && s >= 1 && s <= nparts) prefetch(other, t + G2, s - 1, nparts);
        }
        const bool ok = mbar_wait_ab(done0 + 8u * g, dpar, abort_word);
        dpar ^= 1u;
        if (group_sync_or(g, !ok)) {
          failed = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        // deferred phase factors of this stage: F(c) = A[c & 7] B[c >> 3]
        float2 fa[8], fb[4];
        bool defer = false;
        if constexpr (DEFER) {
          if (st.ndef > 0) {
            defer = true;
            float2 f0 = make_float2(1.0f, 0.0f), gk[5][2];
#pragma unroll
            for (int b = 0; b < 5; ++b) gk[b][0] = gk[b][1] = f0;
            for (int d = 0; d < st.ndef; ++d) {
              const int src = st.def0 + d;
              const float2 f = cmulf(rowtab[size_t(src) * kTtRows + row], s_gfac[g][src - P.pool0]);
              const int key = st.dkey[d];
              if (key < 0) f0 = cmulf(f0, f);
#pragma unroll
              for (int kv = 0; kv < 10; ++kv)
                if (key == kv) gk[kv >> 1][kv & 1] = cmulf(gk[kv >> 1][kv & 1], f);
            }
            float2 t01[4], f2[2];
#pragma unroll
            for (int c = 0; c < 4; ++c) t01[c] = cmulf(gk[0][c & 1], gk[1][c >> 1]);
#pragma unroll
            for (int c = 0; c < 2; ++c) f2[c] = cmulf(f0, gk[2][c]);
#pragma unroll
            for (int c = 0; c < 8; ++c) fa[c] = cmulf(t01[c & 3], f2[c >> 2]);
#pragma unroll
            for (int c = 0; c < 4; ++c) fb[c] = cmulf(gk[3][c & 1], gk[4][c >> 1]);
          }
        }
        // the row of D: the two partial sums added, written into the tile at this
        // stage's positions (for the next stage's gather, or the write-back)
        off[0] = off0;
#pragma unroll
        for (int i = 1; i < 32; ++i) off[i] = off[i - 1] ^ sw[(i & 1) ? 0 : (i & 2) ? 1 : (i & 4) ? 2 : (i & 8) ? 3 : 4];
        float sout = 0.0f;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          uint32_t d0[32], d1[32];
          tmem_ld32(ta + 128u + uint32_t(32 * q), d0);
          tmem_ld32(ta + 192u + uint32_t(32 * q), d1);
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
          for (int i = 16 * q; i < 16 * q + 16; ++i) {
            const int c = (i ^ (i >> 1)) - 16 * q;
            float2 y = make_float2(__uint_as_float(d0[2 * c]) + __uint_as_float(d1[2 * c]),
                                   __uint_as_float(d0[2 * c + 1]) + __uint_as_float(d1[2 * c + 1]));
            if constexpr (DEFER) {
              if (defer) {
                const int cf = i ^ (i >> 1);
                y = cmulf(y, cmulf(fa[cf & 7], fb[cf >> 3]));
              }
            }
            sout = fmaf(y.x, y.x, fmaf(y.y, y.y, sout));
            sts2(curs + off[i], y);
          }
        }
        if (s == S - 1) nout += double(sout);
        // (TMA) the generic-proxy writes of the last stage become visible to the
        // tensor memory accelerator that writes the tile back
        if (tma && s == S - 1) asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        group_sync(g);  // the tile is complete before the next stage gathers
      }
      if (failed) break;
      if (P.permuted) {
        // the pass's exact SWAPs, taken as a relabeling: output u (the thread's row in
        // its low 7 bits, c above) takes the value at the tile position whose bit
        // rbit[k] is bit k of u; both offsets are XOR-linear in u
        auto perm = [&](uint32_t u) {
          uint32_t v = 0;
          for (int kb = 0; kb < m; ++kb) v |= ((u >> kb) & 1u) << srbit[kb];
          return v;
        };
        auto swz = [&](uint32_t u) { return tma ? tma_swz_bytes(u) : tile_swz(u) * 8u; };
        uint32_t pb[5];
#pragma unroll
        for (int b = 0; b < 5; ++b) pb[b] = swz(perm(1u << (7 + b)));
        uint32_t o = swz(perm(uint32_t(row)));
        float2 pv[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {  // Gray order: c = i ^ (i >> 1)
          if (i) o ^= pb[__ffs(i) - 1];
          pv[i ^ (i >> 1)] = lds2(curs + o);
        }
        group_sync(g);
        const uint32_t d0 = swz(uint32_t(row));
#pragma unroll
        for (int c = 0; c < 32; ++c) sts2(curs + (d0 ^ swz(uint32_t(c) << 7)), pv[c]);
        if (tma) asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        group_sync(g);
      }
      if (tma) {
        if (elect) {
          int32_t c[5];
          tma_coords(tile_base(t, tnt), tm, c);
          tma_store_tile(smem_u32(cur), &tmap, c, tm);
        }
        if (!loaded) tma_next();
        continue;
      }
      if (S == 0 && k > 0) {  // no stage windows: write back and load here
        store(other, t - G2);
        group_sync(g);
      }
      if (next && (S <= 1)) prefetch(other, t + G2, 0, 1);
      cp_async_commit();
    }
    if (tma) {
      // the write-backs are complete before the block leaves (and the loads, if a
      // failure cut the loop short)
      if (elect) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
      if (elect && nload > nwait) {
        // a failure cut the loop short with a load in flight (at most one: a load is
        // issued only after the previous one was waited for)
        const volatile int never = 0;
        mbar_wait_ab(tload, (nload - 1) & 1u, &never);
      }
    } else if (!failed && Kg > 0) {
      // the last tile's write-back
      store(buf0 + ((Kg - 1) & 1) * T, t0 + uint64_t(Kg - 1) * G2);
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (failed) *abort_word = 1;
    s_norm[0][tid] = nin;
    s_norm[1][tid] = nout;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (tid == 0 && *abort_word) atomicExch(status, 1);
  // this block's norm sums, added in thread order (the same on every run)
  if (tid == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < kTtGroups * kTtGroupThreads; ++i) {
      a += s_norm[0][i];
      b += s_norm[1][i];
    }
    if (nrm.first) nrm.in_part[blockIdx.x] = a;
    nrm.out_cur[blockIdx.x] = b;
  }
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------
using cd = std::complex<double>;

// the device tile swizzle (tile_swz) on the host: index bits 0..3 XOR-ed with a hash of
// the higher bits
static uint32_t tile_swz_host(uint32_t r) {
  const uint32_t x = r >> 4;
  return r ^ ((x ^ (x >> 4) ^ (x >> 8)) & 15u);
}

// nearest TF32 value (ties to even) of a finite fp32 value of modest size
static float tf32_rne_host(float v) {
  uint32_t u;
  memcpy(&u, &v, 4);
  u += 0xFFFu + ((u >> 13) & 1u);
  u &= 0xFFFFE000u;
  float r;
  memcpy(&r, &u, 4);
  return r;
}

// One stage's record and B image from its 32 x 32 block U (U[row * 32 + col], row and
// column bit k = slot k) and its layout rec.
static void tc_stage_record(const std::vector<cd>& U, const TileStage& rec, bool tma, std::vector<TcStage>& out,
                            std::vector<float>& imgs) {
  constexpr int D = 1 << kTtSB;
  // B image: Bt[n][k] (n = output column, k = input column) of the real form,
  // y_d = sum_c U[d][c] x_c; per K slice, the hi rows then the lo rows, each in the
  // swizzled layout
  TcStage ts{};
  ts.img = int32_t(imgs.size() / kTtImgFloats);
  const size_t o0 = imgs.size();
  imgs.resize(o0 + kTtImgFloats, 0.0f);
  float* img = imgs.data() + o0;
  for (int d = 0; d < D; ++d)
    for (int c = 0; c < D; ++c) {
      const double ur = U[d * D + c].real(), ui = U[d * D + c].imag();
      const double vals[4] = {ur, -ui, ui, ur};
      const int ns[4] = {2 * d, 2 * d, 2 * d + 1, 2 * d + 1};
      const int ks[4] = {2 * c, 2 * c + 1, 2 * c, 2 * c + 1};
      for (int e = 0; e < 4; ++e) {
        const float v = float(vals[e]), h = tf32_rne_host(v);
        const uint32_t off = ((ks[e] >> 5) * 2 * kTtBregion + sw128_offset(ns[e], ks[e] & 31, kTtCols)) / 4;
        img[off] = h;
        img[off + kTtBregion / 4] = tf32_rne_host(v - h);
      }
    }
  for (int k = 0; k < kTtSB; ++k)
    ts.swz[k] = tma ? tma_swz_bytes(1u << rec.slot_bit[k]) : tile_swz_host(1u << rec.slot_bit[k]) * 8u;
  for (int k = 0; k < kTtM - kTtSB; ++k) ts.lane_bit[k] = rec.lane_bit[k];
  if (tma) {
    // With the 128-byte swizzle, local bit p moves an 8-byte access to bank slot bit
    // (p = 0: 0; 1..3: p; 4..6: p - 3; 7 and up: none).  Rows are a warp's lanes, so
    // the first four row bits take one bit of each of these classes where the
    // stage's slots leave one (a half warp then reads 16 distinct slots).
    int8_t order[kTtM - kTtSB];
    bool used[kTtM - kTtSB] = {false};
    int no = 0;
    for (int cls = 0; cls < 4; ++cls)
      for (int k = 0; k < kTtM - kTtSB; ++k) {
        const int p = rec.lane_bit[k];
        const int c = p == 0 ? 0 : p <= 3 ? p : p <= 6 ? p - 3 : -1;
        if (!used[k] && c == cls) {
          used[k] = true;
          order[no++] = int8_t(p);
          break;
        }
      }
    for (int k = 0; k < kTtM - kTtSB; ++k)
      if (!used[k]) order[no++] = rec.lane_bit[k];
    for (int k = 0; k < kTtM - kTtSB; ++k) ts.lane_bit[k] = order[k];
  }
  out.push_back(ts);
}

// Deferred phase factors of a circuit plan, host side: per factor a row table (128
// complex values indexed by the stage's row number) and three tile-number chunk tables
// (3 x 256), products formed in FP64 and rounded to FP32.
struct TcDeferTabs {
  std::vector<float> row;   // 2 x 128 floats per factor
  std::vector<float> glob;  // 2 x 768 floats per factor
  int count = 0;
};

// The stages of one pass as 32 x 32 blocks and their B images.  mode 1: every control
// and phase bit of an op is a slot of its stage; false if an op depends on a bit outside
// them.  mode 2: the phase bits of a phase op conditioned on at most one slot need no
// slot; that part of the op is deferred to the end of the stage (its tables go into
// tabs); false if a later op of the stage acts densely on the condition's slot, or the
// factors exceed a stage's or a pass's share.  The pass's factors: global indices
// [*pass_def0, *pass_def0 + *pass_ndef).
static bool tc_pass_blocks(const BuiltPass& bp, const std::vector<PlanOp>& pops, int n, bool tma, int mode,
                           std::vector<TcStage>& out, std::vector<float>& imgs, TcDeferTabs& tabs, int* pass_def0,
                           int* pass_ndef, std::vector<std::vector<cd>>* blocks_out = nullptr,
                           std::vector<std::array<int8_t, 5>>* slots_out = nullptr) {
  int local_of[64];
  for (int b = 0; b < 64; ++b) local_of[b] = -1;
  for (int i = 0; i < kTtM; ++i) local_of[bp.B[i]] = i;
  std::vector<int> tnbits;  // bit i of a tile number sits at global bit tnbits[i]
  for (int b = 0; b < n; ++b)
    if (local_of[b] < 0) tnbits.push_back(b);
  if (mode == 2 && tnbits.size() > 24) return false;
  std::vector<std::vector<int>> takes, acts;
  split_stages_lookahead(bp, pops, local_of, kTtSB, takes, acts, mode, kTtStageLookahead);
  const std::vector<TileStage> recs = stage_layouts(acts, kTtM, kTtSB, 4);
  constexpr int D = 1 << kTtSB;
  *pass_def0 = tabs.count;
  *pass_ndef = 0;
  for (size_t si = 0; si < takes.size(); ++si) {
    int slot_of_local[16];
    for (int k = 0; k < 16; ++k) slot_of_local[k] = -1;
    for (int k = 0; k < kTtSB; ++k) slot_of_local[recs[si].slot_bit[k]] = k;
    auto slot_of = [&](int gbit) { return local_of[gbit] < 0 ? -1 : slot_of_local[local_of[gbit]]; };
    std::vector<cd> U(D * D, cd(0.0, 0.0));  // U[row * D + col]
    for (int d = 0; d < D; ++d) U[d * D + d] = 1.0;
    // deferred factors of the stage: key (-1, or 2 slot + value) and their angles on
    // the tile's local bits and on the global bits
    std::vector<int> dkeys;
    std::vector<std::vector<double>> dloc, dglob;
    const std::vector<int>& tk = takes[si];
    for (size_t oi = 0; oi < tk.size(); ++oi) {
      const PlanOp& p = pops[tk[oi]];
      uint32_t cm = 0, cv = 0;
      for (int b = 0; b < n; ++b) {
        if (!((p.cmask >> b) & 1)) continue;
        const int k = slot_of(b);
        if (k < 0) return false;
        cm |= 1u << k;
        if ((p.cval >> b) & 1) cv |= 1u << k;
      }
      if (p.phase) {
        std::vector<std::pair<int, double>> bs, rest;
        for (const auto& be : p.beta) {
          const int k = slot_of(be.first);
          if (k >= 0)
            bs.push_back({k, be.second});
          else if (mode == 2)
            rest.push_back(be);
          else
            return false;
        }
        if (!rest.empty()) {
          if (__builtin_popcount(cm) >= 2) return false;
          int key = -1;
          if (cm) {
            // the factor moves past the stage's later ops: none may act densely on its
            // slot, except an exact SWAP, which moves the factor to the other slot
            const int k0 = __builtin_ctz(cm);
            int k = k0;
            for (size_t oj = oi + 1; oj < tk.size(); ++oj) {
              const PlanOp& q = pops[tk[oj]];
              if (q.phase) continue;
              bool hit = false;
              for (int t = 0; t < q.nt; ++t) hit |= slot_of(q.tb[t]) == k;
              if (!hit) continue;
              if (!is_exact_swap(q)) return false;
              const int a = slot_of(q.tb[0]), b = slot_of(q.tb[1]);
              k = a == k ? b : a;
            }
            key = 2 * k + int((cv >> k0) & 1u);
          }
          int f = int(std::find(dkeys.begin(), dkeys.end(), key) - dkeys.begin());
          if (f == int(dkeys.size())) {
            dkeys.push_back(key);
            dloc.push_back(std::vector<double>(kTtM, 0.0));
            dglob.push_back(std::vector<double>(n, 0.0));
          }
          for (const auto& be : rest) {
            if (local_of[be.first] >= 0)
              dloc[f][local_of[be.first]] += be.second;
            else
              dglob[f][be.first] += be.second;
          }
        }
        for (int d = 0; d < D; ++d) {
          if ((uint32_t(d) & cm) != cv) continue;
          double ang = p.c;
          for (const auto& be : bs) ang += ((d >> be.first) & 1) ? be.second : 0.0;
          const cd f = std::polar(1.0, ang);
          for (int c = 0; c < D; ++c) U[d * D + c] *= f;
        }
      } else if (p.nt == 1) {
        const int a = slot_of(p.tb[0]);
        if (a < 0) return false;
        const cd m00(p.m[0], p.m[1]), m01(p.m[2], p.m[3]), m10(p.m[4], p.m[5]), m11(p.m[6], p.m[7]);
        for (int d = 0; d < D; ++d) {
          if ((d >> a) & 1 || (uint32_t(d) & cm) != cv) continue;
          const int d1 = d | (1 << a);
          for (int c = 0; c < D; ++c) {
            const cd u0 = U[d * D + c], u1 = U[d1 * D + c];
            U[d * D + c] = m00 * u0 + m01 * u1;
            U[d1 * D + c] = m10 * u0 + m11 * u1;
          }
        }
      } else {
        const int a = slot_of(p.tb[0]), b2 = slot_of(p.tb[1]);  // row index 2 b_a + b_b
        if (a < 0 || b2 < 0) return false;
        cd M[16];
        for (int e = 0; e < 16; ++e) M[e] = cd(p.m[2 * e], p.m[2 * e + 1]);
        for (int d = 0; d < D; ++d) {
          if ((d >> a) & 1 || (d >> b2) & 1 || (uint32_t(d) & cm) != cv) continue;
          const int ix[4] = {d, d | (1 << b2), d | (1 << a), d | (1 << a) | (1 << b2)};
          for (int c = 0; c < D; ++c) {
            cd x[4];
            for (int i = 0; i < 4; ++i) x[i] = U[ix[i] * D + c];
            for (int i = 0; i < 4; ++i)
              U[ix[i] * D + c] = M[4 * i] * x[0] + M[4 * i + 1] * x[1] + M[4 * i + 2] * x[2] + M[4 * i + 3] * x[3];
          }
        }
      }
    }
    tc_stage_record(U, recs[si], tma, out, imgs);
    if (blocks_out) blocks_out->push_back(U);
    if (slots_out) {
      std::array<int8_t, 5> sl;
      for (int k = 0; k < kTtSB; ++k) sl[k] = recs[si].slot_bit[k];
      slots_out->push_back(sl);
    }
    if (!dkeys.empty()) {
      const int nd = int(dkeys.size());
      if (nd > kTtMaxDefStage || *pass_ndef + nd > kTtMaxDefPass) return false;
      TcStage& ts = out.back();
      ts.ndef = int8_t(nd);
      ts.def0 = tabs.count;
      for (int f = 0; f < nd; ++f) {
        ts.dkey[f] = int8_t(dkeys[f]);
        for (int r = 0; r < kTtRows; ++r) {  // row bit b sits at local bit lane_bit[b]
          double ang = 0.0;
          for (int b = 0; b < kTtM - kTtSB; ++b)
            if ((r >> b) & 1) ang += dloc[f][ts.lane_bit[b]];
          tabs.row.push_back(float(std::cos(ang)));
          tabs.row.push_back(float(std::sin(ang)));
        }
        for (int c = 0; c < 3; ++c)
          for (int v = 0; v < 256; ++v) {
            double ang = 0.0;
            for (int i = 0; i < 8; ++i)
              if (((v >> i) & 1) && 8 * c + i < int(tnbits.size())) ang += dglob[f][tnbits[8 * c + i]];
            tabs.glob.push_back(float(std::cos(ang)));
            tabs.glob.push_back(float(std::sin(ang)));
          }
        ++tabs.count;
      }
      *pass_ndef += nd;
    }
  }
  return true;
}

// The box plan of a pass's tile (bit set B, index bits 0..3 among them): dimension 0 =
// bits 0..3; the runs of bits above (alternately in and out of the tile) grouped into
// at most 4 dimensions of consecutive bits so that as few tile bits as possible fall in
// dimensions that are not copied whole (those become box coordinates; at most
// kTtMaxCoordBits); tma = 0 if no grouping fits.  Bloc receives the
// tile's bits in the boxes' local order.
static TcTma tma_plan(const std::vector<int>& B, int n, std::vector<int>& Bloc) {
  bool in[64] = {false};
  for (int b : B) in[b] = true;
  for (int b = 0; b < kTtL; ++b)
    if (!in[b]) return TcTma{};
  std::vector<int> rs, rl;
  std::vector<char> rin;
  for (int b = kTtL; b < n;) {
    const int st = b;
    const bool t = in[b];
    while (b < n && in[b] == t) ++b;
    rs.push_back(st);
    rl.push_back(b - st);
    rin.push_back(t ? 1 : 0);
  }
  const int R = int(rs.size());
  constexpr int kGroups = 4, kInf = 1 << 20;
  // a group of runs [i, j): copied whole if it is one run, else its tile bits are
  // coordinates
  auto cost = [&](int i, int j) {
    if (j - i == 1) return 0;
    int c = 0;
    for (int x = i; x < j; ++x)
      if (rin[x]) c += rl[x];
    return c;
  };
  std::vector<std::vector<int>> best(kGroups + 1, std::vector<int>(R + 1, kInf)), from = best;
  best[0][0] = 0;
  for (int g = 1; g <= kGroups; ++g)
    for (int j = 1; j <= R; ++j)
      for (int i = g - 1; i < j; ++i)
        if (best[g - 1][i] < kInf && best[g - 1][i] + cost(i, j) < best[g][j]) {
          best[g][j] = best[g - 1][i] + cost(i, j);
          from[g][j] = i;
        }
  int G = 0;
  for (int g = 1; g <= kGroups; ++g)
    if (best[g][R] < (G ? best[G][R] : kInf)) G = g;
  if (G == 0 || best[G][R] > kTtMaxCoordBits) return TcTma{};
  std::vector<std::pair<int, int>> groups(G);  // runs [first, last)
  for (int g = G, j = R; g >= 1; --g) {
    groups[g - 1] = {from[g][j], j};
    j = from[g][j];
  }
  TcTma tm{};
  tm.start[0] = 0;
  tm.len[0] = int8_t(kTtL);
  tm.tile[0] = 1;
  Bloc.clear();
  for (int b = 0; b < kTtL; ++b) Bloc.push_back(b);
  std::vector<int> coords;
  for (int g = 0; g < G; ++g) {
    const int i = groups[g].first, j = groups[g].second, d = g + 1;
    tm.start[d] = int8_t(rs[i]);
    tm.len[d] = int8_t(rs[j - 1] + rl[j - 1] - rs[i]);
    tm.tile[d] = (j - i == 1 && rin[i]) ? 1 : 0;
    for (int x = i; x < j; ++x) {
      if (!rin[x]) continue;
      for (int b = rs[x]; b < rs[x] + rl[x]; ++b) {
        if (tm.tile[d]) {
          Bloc.push_back(b);
        } else {
          tm.cdim[coords.size()] = int8_t(d);
          tm.coff[coords.size()] = int8_t(b - rs[i]);
          coords.push_back(b);
        }
      }
    }
  }
  for (int d = G + 1; d < 5; ++d) {  // padding dimensions of size 1 above the state
    tm.start[d] = int8_t(n);
    tm.len[d] = 0;
    tm.tile[d] = 0;
  }
  tm.nc = int8_t(coords.size());
  for (int b : coords) Bloc.push_back(b);
  if (int(Bloc.size()) != kTtM) return TcTma{};
  tm.tma = 1;
  return tm;
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// the tensor map of a pass's box over the state at `amps` (complex64, n qubits)
static bool encode_tile_map(CUtensorMap* map, const TcTma& tm, void* amps, int n) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  cuuint64_t gdim[5], gstride[4];
  cuuint32_t box[5], estr[5] = {1, 1, 1, 1, 1};
  for (int d = 0; d < 5; ++d) {
    gdim[d] = cuuint64_t(1) << tm.len[d];
    box[d] = tm.tile[d] ? (cuuint32_t(1) << tm.len[d]) : 1u;
    if (d > 0) gstride[d - 1] = (cuuint64_t(1) << tm.start[d]) * 8u;
  }
  (void)n;
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, amps, gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The most recent tensor-core circuit plan of the process: the resolved ops it was built
// from (compared exactly on the next call), its passes, and on the device its stage
// records and B images.  A repeated circuit (the usual case: the same circuit on new
// inputs) skips planning, the host products of the stage blocks and the upload.
struct TcPlanCache {
  int device = -1;
  int n = 0;
  std::vector<ResolvedOp> rops;
  bool valid = false;
  bool tc = false;  // false: an op depends on a bit outside its stage (CUDA-core passes)
  std::vector<TilePass> passes;
  std::vector<TcTma> tmas;  // per pass: box copies or cp.async
  std::vector<char> defer;  // per pass: 1 stages with deferred phase factors, 2 a copy pass
  int nstages = 0;
  std::vector<char> host;  // staging of the upload (kept until the next rebuild)
  void* dev = nullptr;
  size_t dev_bytes = 0;
  size_t stage_bytes = 0;
  size_t row_off = 0, glob_off = 0;  // byte offsets of the factor tables in `dev`
  cudaEvent_t done = nullptr;  // recorded after the launches that read `dev`
  bool pending = false;
};
static TcPlanCache g_tc;
static std::mutex g_tc_mu;

static bool same_ops(const std::vector<ResolvedOp>& a, const std::vector<ResolvedOp>& b) {
  if (a.size() != b.size()) return false;
  for (size_t i = 0; i < a.size(); ++i) {
    const ResolvedOp &x = a[i], &y = b[i];
    if (x.form != y.form || x.nq != y.nq || x.cstate != y.cstate) return false;
    for (int k = 0; k < x.nq; ++k)
      if (x.bits[k] != y.bits[k]) return false;
    const int dim = x.form == FORM_2Q ? 4 : 2;
    if (memcmp(x.m, y.m, sizeof(double) * 2 * dim * dim) != 0) return false;
  }
  return true;
}

// plans `rops` into the cache (host stage blocks, B images, upload)
// A pass's exact SWAPs of two tile bits taken as a relabeling: the other ops renamed
// into rpops (br: the pass over them, the same tile bits), rbit[k] = the local bit (in
// the order of bp.B) where the data of local bit k sits when the pass ends; false (rbit
// the identity) if the pass has no such SWAP.
static bool relabel_swaps(const BuiltPass& bp, const std::vector<PlanOp>& pops, std::vector<PlanOp>& rpops,
                          BuiltPass& br, int8_t* rbit) {
  int ren[64], loc[64];
  for (int b = 0; b < 64; ++b) {
    ren[b] = b;
    loc[b] = -1;
  }
  for (int i = 0; i < kTtM; ++i) loc[bp.B[i]] = i;
  br.B = bp.B;
  br.ops.clear();
  rpops.clear();
  bool permuted = false;
  for (int idx : bp.ops) {
    const PlanOp& p = pops[idx];
    if (is_exact_swap(p) && loc[ren[p.tb[0]]] >= 0 && loc[ren[p.tb[1]]] >= 0) {
      std::swap(ren[p.tb[0]], ren[p.tb[1]]);
      permuted = true;
      continue;
    }
    br.ops.push_back(int(rpops.size()));
    rpops.push_back(renamed(p, ren));
  }
  for (int k = 0; k < 16; ++k) rbit[k] = int8_t(k < kTtM && permuted ? loc[ren[bp.B[k]]] : k);
  return permuted;
}

// The variant a pass's plan takes (every phase bit a slot or deferred factors; SWAPs as
// ops or relabeled) depends only on the pass's structure: op kinds, bits, conditions,
// phase bits and which ops are exact SWAPs, the tile's bits and its copy kind.  Recent
// choices are kept (-1: none fits; -2: not known).
static std::vector<int64_t> variant_key(const BuiltPass& bp, const std::vector<PlanOp>& pops, int n, bool tma) {
  std::vector<int64_t> key = {n, tma ? 1 : 0};
  for (int b : bp.B) key.push_back(b);
  for (int idx : bp.ops) {
    const PlanOp& p = pops[size_t(idx)];
    key.push_back(p.phase ? -1 : p.nt);
    key.push_back(p.phase ? 0 : int64_t(p.tb[0]) * 64 + (p.nt == 2 ? p.tb[1] : 0));
    key.push_back(int64_t(p.touched));
    key.push_back(int64_t(p.cmask));
    key.push_back(int64_t(p.cval));
    uint64_t bb = 0;
    for (const auto& be : p.beta) bb |= uint64_t(1) << be.first;
    key.push_back(int64_t(bb));
    key.push_back(is_exact_swap(p) ? 1 : 0);
  }
  return key;
}
static std::mutex g_variant_mu;
static std::vector<std::pair<std::vector<int64_t>, int>> g_variants;  // most recent last
static int cached_variant(const std::vector<int64_t>& key) {
  std::lock_guard<std::mutex> lock(g_variant_mu);
  for (const auto& e : g_variants)
    if (e.first == key) return e.second;
  return -2;
}
static void keep_variant(const std::vector<int64_t>& key, int pick) {
  std::lock_guard<std::mutex> lock(g_variant_mu);
  if (g_variants.size() >= 512) g_variants.erase(g_variants.begin());
  g_variants.push_back({key, pick});
}

// A circuit's tensor-core plan on the host: passes, their box plans and kinds (defer: 0
// plain, 1 with deferred phase factors, 2 a relabeling copied by the CUDA-core pass),
// stage records, B images and factor tables; optionally each stage's FP64 block and slot
// bits (for a host emulation).  amps: the state whose address the box plans are tried
// with (nullptr: no trial encoding).  False: the circuit does not fit the stages.
struct TcHostPlan {
  std::vector<TilePass> passes;
  std::vector<TcTma> tmas;
  std::vector<char> defer;
  std::vector<TcStage> stages;
  std::vector<float> imgs;
  TcDeferTabs tabs;
  std::vector<std::vector<cd>>* blocks = nullptr;
  std::vector<std::array<int8_t, 5>>* slots = nullptr;
};

// An empty host plan whose vectors keep their capacity from this thread's earlier plans:
// re-planning a circuit (new parameter values) then writes its 2-4 MB of stage images
// into memory already mapped instead of growing a new vector page by page.  Valid until
// the thread's next call.
static TcHostPlan& tc_scratch_plan() {
  thread_local TcHostPlan hp;
  hp.passes.clear();
  hp.tmas.clear();
  hp.defer.clear();
  hp.stages.clear();
  hp.imgs.clear();
  hp.tabs.row.clear();
  hp.tabs.glob.clear();
  hp.tabs.count = 0;
  hp.blocks = nullptr;
  hp.slots = nullptr;
  return hp;
}

static bool tc_build(int n, const std::vector<ResolvedOp>& rops, void* amps, TcHostPlan& hp) {
  std::vector<PlanOp> pops;
  to_plan_ops(rops, pops);
  const std::vector<BuiltPass> bps = build_passes(pops, n, kTtM, kTtL, /*cond_in_tile=*/true);
  std::vector<TilePass>& passes = hp.passes;
  std::vector<TcTma>& tmas = hp.tmas;
  std::vector<char>& defer = hp.defer;
  std::vector<TcStage>& stages = hp.stages;
  std::vector<float>& imgs = hp.imgs;
  TcDeferTabs& tabs = hp.tabs;
  for (const BuiltPass& bp : bps) {
    std::vector<int> Bloc;
    TcTma tm = tma_plan(bp.B, n, Bloc);
    if (tm.tma && amps) {  // a trial encoding with this state's address
      alignas(64) CUtensorMap probe;
      if (!encode_tile_map(&probe, tm, amps, n)) tm = TcTma{};
    }
    BuiltPass bl = bp;  // the tile's bits in the local order of its boxes
    if (tm.tma) bl.B = Bloc;
    TilePass P{};
    P.m = kTtM;
    P.L = kTtL;
    for (int i = 0; i < kTtM; ++i) P.bits[i] = int8_t(bl.B[i]);
    P.ntiles = uint64_t(1) << (n - kTtM);
    P.stage0 = int(stages.size());
    // The pass's exact SWAPs of two tile bits, either as ops of the stages or as a
    // relabeling (the later ops renamed, the tile permuted before its write-back)
    std::vector<PlanOp> rpops;
    BuiltPass br;
    int8_t rbit[16];
    const bool permuted = relabel_swaps(bl, pops, rpops, br, rbit);
    // every phase bit a slot (mode 1), or phase bits off the slots deferred (mode 2);
    // SWAPs as ops or relabeled: the fewest stages win (a relabeling counts half a
    // stage; the earlier variant on ties); none: the CUDA-core passes take the circuit
    int def0 = 0, ndef = 0;
    const size_t i0 = imgs.size(), r0 = tabs.row.size(), g0 = tabs.glob.size();
    const int c0 = tabs.count;
    auto reset = [&]() {
      stages.resize(size_t(P.stage0));
      imgs.resize(i0);
      tabs.row.resize(r0);
      tabs.glob.resize(g0);
      tabs.count = c0;
      if (hp.blocks) hp.blocks->resize(size_t(P.stage0));
      if (hp.slots) hp.slots->resize(size_t(P.stage0));
    };
    auto plan = [&](int v) {  // v: 2 relabel + (mode - 1)
      const bool rl = v >= 2;
      return tc_pass_blocks(rl ? br : bl, rl ? rpops : pops, n, tm.tma != 0, 1 + (v & 1), stages, imgs, tabs,
                            &def0, &ndef, hp.blocks, hp.slots);
    };
    // (the choice depends on the pass's structure only: kept and reused when the circuit
    // runs again with other values)
    const std::vector<int64_t> vkey = variant_key(bl, pops, n, tm.tma != 0);
    int pick = cached_variant(vkey);
    bool planned = false;
    if (pick >= 0) {  // should it no longer fit, every variant is tried
      reset();
      planned = plan(pick);
      if (!planned) pick = -2;
    }
    if (pick == -2) {
      pick = -1;
      double best = 1e30;
      for (int v = 0; v < (permuted ? 4 : 2); ++v) {
        reset();
        if (!plan(v)) continue;
        const double score = double(stages.size() - size_t(P.stage0)) + (v >= 2 ? 0.5 : 0.0);
        if (score < best) {
          best = score;
          pick = v;
        }
      }
      keep_variant(vkey, pick);
    }
    if (pick < 0) return false;
    if (!planned) {
      reset();
      if (!plan(pick)) return false;
    }
    bool copy = false;
    if (pick >= 2) {
      P.permuted = 1;
      for (int k = 0; k < 16; ++k) P.rbit[k] = rbit[k];
      if (int(stages.size()) == P.stage0) {
        // nothing but the relabeling: the CUDA-core pass copies the tiles (bits in
        // ascending order, the relabeling in that order)
        copy = true;
        std::vector<PlanOp> cpops;
        BuiltPass cb;
        relabel_swaps(bp, pops, cpops, cb, P.rbit);
        for (int k = 0; k < 16; ++k) P.bits[k] = int8_t(k < kTtM ? bp.B[k] : 0);
      }
    } else {
      for (int k = 0; k < 16; ++k) P.rbit[k] = int8_t(k);
    }
    P.pool0 = def0;  // the pass's deferred factors (global indices)
    P.npool = ndef;
    P.nstages = int(stages.size()) - P.stage0;
    if (P.nstages > kTtMaxStages) return false;
    passes.push_back(P);
    tmas.push_back(tm);
    defer.push_back(copy ? 2 : ndef > 0 ? 1 : 0);
  }
  return true;
}

static qc_status tc_plan(qc_state* s, const std::vector<ResolvedOp>& rops, int dev) {
  const int n = s->n;
  g_tc.valid = false;
  TcHostPlan& hp = tc_scratch_plan();
  const bool tc = tc_build(n, rops, s->amps, hp);
  std::vector<TilePass>& passes = hp.passes;
  std::vector<TcTma>& tmas = hp.tmas;
  std::vector<char>& defer = hp.defer;
  std::vector<TcStage>& stages = hp.stages;
  std::vector<float>& imgs = hp.imgs;
  TcDeferTabs& tabs = hp.tabs;
  g_tc.device = dev;
  g_tc.n = n;
  g_tc.rops = rops;
  g_tc.tc = tc;
  g_tc.valid = true;
  if (!tc) return QC_OK;
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t sb = al(stages.size() * sizeof(TcStage) + 1);
  const size_t ib = al(imgs.size() * sizeof(float));
  const size_t rb = al(tabs.row.size() * sizeof(float)), gb = tabs.glob.size() * sizeof(float);
  const size_t total = sb + ib + rb + gb;
  g_tc.host.assign(total, 0);
  if (!stages.empty()) memcpy(g_tc.host.data(), stages.data(), stages.size() * sizeof(TcStage));
  if (!imgs.empty()) memcpy(g_tc.host.data() + sb, imgs.data(), imgs.size() * sizeof(float));
  if (!tabs.row.empty()) memcpy(g_tc.host.data() + sb + ib, tabs.row.data(), tabs.row.size() * sizeof(float));
  if (gb) memcpy(g_tc.host.data() + sb + ib + rb, tabs.glob.data(), gb);
  // the previous plan's launches are done with the buffer before it is overwritten
  if (g_tc.pending) cudaEventSynchronize(g_tc.done);
  g_tc.pending = false;
  if (g_tc.dev_bytes < total) {
    if (g_tc.dev) cudaFree(g_tc.dev);
    g_tc.dev = nullptr;
    g_tc.dev_bytes = 0;
    if (qc_status st = check_cuda(cudaMalloc(&g_tc.dev, total), "tensor-core plan buffer")) {
      g_tc.valid = false;
      return st;
    }
    g_tc.dev_bytes = total;
  }
  if (qc_status st = check_cuda(cudaMemcpyAsync(g_tc.dev, g_tc.host.data(), total, cudaMemcpyHostToDevice,
                                                s->stream),
                                "tensor-core plan upload")) {
    g_tc.valid = false;
    return st;
  }
  g_tc.passes = passes;
  g_tc.tmas = tmas;
  g_tc.defer = defer;
  g_tc.nstages = int(stages.size());
  g_tc.stage_bytes = sb;
  g_tc.row_off = sb + ib;
  g_tc.glob_off = sb + ib + rb;
  return QC_OK;
}

// the shared-memory opt-in of both pass kernels
static qc_status tc_pass_smem() {
  for (auto kern : {k_tile_pass_tc<false, false>, k_tile_pass_tc<true, false>, k_tile_pass_tc<false, true>,
                    k_tile_pass_tc<true, true>})
    if (qc_status st = check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       int(kTtSmem)),
                                  "tensor-core tile pass shared memory"))
      return st;
  return QC_OK;
}

// one pass on s's stream: box copies with a tensor map of this state where tm.tma;
// defer: the pass's stages have deferred phase factors (tables rowtab, gtab)
static qc_status launch_tc_pass(qc_state* s, const TilePass& P, const TcTma& tm, bool defer, const TcStage* dst,
                                const float* dimg, int* status, const TcNorm& nm, unsigned grid,
                                const float2* rowtab = nullptr, const float2* gtab = nullptr) {
  alignas(64) CUtensorMap map;
  memset(&map, 0, sizeof(map));
  if (tm.tma && !encode_tile_map(&map, tm, s->amps, s->n)) {
    set_error("tensor-core tile pass: tensor map encoding failed");
    return QC_ERR_CUDA;
  }
  float* a = reinterpret_cast<float*>(s->amps);
  auto kern = tm.tma ? (defer ? k_tile_pass_tc<true, true> : k_tile_pass_tc<true, false>)
                     : (defer ? k_tile_pass_tc<false, true> : k_tile_pass_tc<false, false>);
  QC_COUNT(), kern<<<grid, kTtThreads, kTtSmem, s->stream>>>(a, P, dst, dimg, status, map, tm, nm, rowtab, gtab);
  return QC_OK;
}

qc_status run_tiles_tc(qc_state* s, const std::vector<ResolvedOp>& rops, bool* handled) {
  *handled = false;
  const int n = s->n;
  if (s->dtype != QC_C64 || n < kTtM) return QC_OK;
  int dev = 0;
  if (qc_status st = check_cuda(cudaGetDevice(&dev), "cudaGetDevice")) return st;
  std::lock_guard<std::mutex> lock(g_tc_mu);
  if (!g_tc.done)
    if (qc_status st = check_cuda(cudaEventCreateWithFlags(&g_tc.done, cudaEventDisableTiming), "plan event"))
      return st;
  if (!(g_tc.valid && g_tc.device == dev && g_tc.n == n && same_ops(g_tc.rops, rops)))
    if (qc_status st = tc_plan(s, rops, dev)) return st;
  if (!g_tc.tc) return QC_OK;
  const uint64_t ntiles0 = uint64_t(1) << (n - kTtM);
  const unsigned grid0 = unsigned(std::min<uint64_t>((ntiles0 + 1) / 2, uint64_t(device_sm_count())));
  void* scr = nullptr;
  if (qc_status st = state_scratch(s, 256 + 3 * sizeof(double) * grid0, &scr)) return st;
  int* status = static_cast<int*>(scr);
  double* norm_in = reinterpret_cast<double*>(static_cast<char*>(scr) + 256);
  double* norm_out[2] = {norm_in + grid0, norm_in + 2 * grid0};
  // norm restoration needs every pass to have a stage (stage 0 scales, the last sums)
  bool restore = true;
  for (const TilePass& P : g_tc.passes) restore &= P.nstages > 0;
  const TcStage* dst = static_cast<const TcStage*>(g_tc.dev);
  const float* dimg = reinterpret_cast<const float*>(static_cast<char*>(g_tc.dev) + g_tc.stage_bytes);
  const float2* drow = reinterpret_cast<const float2*>(static_cast<char*>(g_tc.dev) + g_tc.row_off);
  const float2* dglob = reinterpret_cast<const float2*>(static_cast<char*>(g_tc.dev) + g_tc.glob_off);
  if (qc_status st = check_cuda(cudaMemsetAsync(status, 0, sizeof(int), s->stream), "status reset")) return st;
  if (qc_status st = tc_pass_smem()) return st;
  const uint64_t ntiles = uint64_t(1) << (n - kTtM);
  // one CTA per SM, two tiles in flight per CTA
  const unsigned grid = unsigned(std::min<uint64_t>((ntiles + 1) / 2, uint64_t(device_sm_count())));
  for (size_t i = 0; i < g_tc.passes.size(); ++i) {
    TcNorm nm{};
    nm.first = i == 0 ? 1 : 0;
    nm.apply = restore && i > 0 ? 1 : 0;
    nm.nblocks = int(grid);
    nm.in_part = norm_in;
    nm.out_prev = norm_out[(i + 1) & 1];
    nm.out_cur = norm_out[i & 1];
    if (g_tc.defer[i] == 2) {
      if (qc_status st = launch_copy_pass(s, g_tc.passes[i])) return st;
      continue;
    }
    if (qc_status st = launch_tc_pass(s, g_tc.passes[i], g_tc.tmas[i], g_tc.defer[i] != 0, dst, dimg, status, nm,
                                      grid, drow, dglob))
      return st;
  }
  if (qc_status st = check_launch("tensor-core tile pass")) return st;
  if (qc_status st = check_cuda(cudaEventRecord(g_tc.done, s->stream), "plan event")) return st;
  g_tc.pending = true;
  int h = 0;
  if (qc_status st = check_cuda(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s->stream),
                                "status"))
    return st;
  if (qc_status st = check_cuda(cudaStreamSynchronize(s->stream), "tensor-core tile pass")) return st;
  if (qc_status st = device_status(h, "tensor-core tile pass")) return st;
  g_last_pass_count = int(g_tc.passes.size());
  g_last_fused_path = 2;
  g_last_stage_count = g_tc.nstages;
  *handled = true;
  return QC_OK;
}

// The tile of a one-block pass: index bits 0..3, the block's bits and fillers up to kTtM
// bits.  Every subset of the gaps between the tile's runs that the fillers can close is
// tried (at most 2^(k + 1)); the remaining fillers extend runs without splitting a gap
// (lowest bits first, or highest first); the tile whose box plan has the fewest
// coordinate bits, then the fewest dimensions, wins.  Bloc receives its bits in the
// boxes' local order; tma = 0 if no candidate has a box plan.
static TcTma block_tile_plan(const int* bits, int k, int n, std::vector<int>& Bloc) {
  bool base[64] = {false};
  for (int b = 0; b < kTtL; ++b) base[b] = true;
  for (int j = 0; j < k; ++j) base[bits[j]] = true;
  std::vector<std::pair<int, int>> gaps;  // [first, end) of each run of bits outside
  for (int b = kTtL; b < n;) {
    if (base[b]) {
      ++b;
      continue;
    }
    const int a = b;
    while (b < n && !base[b]) ++b;
    gaps.push_back({a, b});
  }
  TcTma best{};
  int best_nc = 1 << 20, best_nd = 1 << 20;
  const int ng = std::min(int(gaps.size()), 16);
  for (uint32_t sub = 0; sub < (1u << ng); ++sub)
    for (int dir = 0; dir < 2; ++dir) {
      bool in[64];
      memcpy(in, base, sizeof(in));
      for (int g = 0; g < ng; ++g)
        if ((sub >> g) & 1)
          for (int x = gaps[g].first; x < gaps[g].second; ++x) in[x] = true;
      int cnt = 0;
      for (int b = 0; b < n; ++b) cnt += in[b] ? 1 : 0;
      if (cnt > kTtM) continue;
      while (cnt < kTtM) {
        int pick = -1;
        for (int i = 0; i < n - kTtL && pick < 0; ++i) {
          const int b = dir ? n - 1 - i : kTtL + i;
          if (!in[b] && ((b + 1 < n && in[b + 1]) || (b - 1 >= kTtL && in[b - 1]))) pick = b;
        }
        for (int b = kTtL; b < n && pick < 0; ++b)
          if (!in[b]) pick = b;
        in[pick] = true;
        ++cnt;
      }
      std::vector<int> B, bl;
      for (int b = 0; b < n; ++b)
        if (in[b]) B.push_back(b);
      const TcTma tm = tma_plan(B, n, bl);
      if (!tm.tma) continue;
      int nd = 0;
      for (int d = 0; d < 5; ++d) nd += tm.len[d] > 0 ? 1 : 0;
      if (tm.nc < best_nc || (tm.nc == best_nc && nd < best_nd)) {
        best = tm;
        best_nc = tm.nc;
        best_nd = nd;
        Bloc = bl;
      }
    }
  return best;
}

qc_status apply_block_tile_tc(qc_state* s, const int* bits, int k, const double* U, bool* handled) {
  *handled = false;
  const int n = s->n;
  if (s->dtype != QC_C64 || n < kTtM || k < 1 || k > kTtSB) return QC_OK;
  std::vector<int> B;  // the tile's bits in the local order of its boxes
  const TcTma tm = block_tile_plan(bits, k, n, B);
  // only as box copies: with per-amplitude copies the gathering block kernel is faster
  // (1.08 against 1.22 ms for a spread 5-qubit block at 28 qubits)
  if (!tm.tma) return QC_OK;
  {
    alignas(64) CUtensorMap probe;
    if (!encode_tile_map(&probe, tm, s->amps, n)) return QC_OK;
  }
  int local_of[64];
  for (int b = 0; b < 64; ++b) local_of[b] = -1;
  for (int i = 0; i < kTtM; ++i) local_of[B[i]] = i;
  std::vector<std::vector<int>> acts(1);
  for (int j = 0; j < k; ++j) acts[0].push_back(local_of[bits[j]]);
  const TileStage rec = stage_layouts(acts, kTtM, kTtSB, 4)[0];  // slot j = bits[j] for j < k
  // the 32 x 32 block: U on slots 0..k-1 (bits[0] the most significant bit of U's
  // index), the identity on the padding slots
  constexpr int D = 1 << kTtSB;
  const int Dk = 1 << k;
  auto urow = [&](int d) {
    int r = 0;
    for (int j = 0; j < k; ++j) r |= ((d >> j) & 1) << (k - 1 - j);
    return r;
  };
  std::vector<cd> U32(D * D, cd(0.0, 0.0));
  for (int d = 0; d < D; ++d)
    for (int c = 0; c < D; ++c)
      if ((d >> k) == (c >> k)) {
        const int e = urow(d) * Dk + urow(c);
        U32[d * D + c] = cd(U[2 * e], U[2 * e + 1]);
      }
  std::vector<TcStage> recs;
  std::vector<float> img;
  tc_stage_record(U32, rec, true, recs, img);
  TilePass P{};
  P.m = kTtM;
  P.L = kTtL;
  for (int i = 0; i < kTtM; ++i) P.bits[i] = int8_t(B[i]);
  P.ntiles = uint64_t(1) << (n - kTtM);
  P.stage0 = 0;
  P.nstages = 1;
  const unsigned grid = unsigned(std::min<uint64_t>((P.ntiles + 1) / 2, uint64_t(device_sm_count())));
  // scratch: status word, norm sums (written, not used: one pass), stage record, B image
  const size_t o_norm = 256, o_rec = (o_norm + sizeof(double) * grid + 255) & ~size_t(255);
  const size_t o_img = o_rec + 256, total = o_img + img.size() * sizeof(float);
  void* scr = nullptr;
  if (qc_status st = state_scratch(s, total, &scr)) return st;
  char* base = static_cast<char*>(scr);
  int* status = reinterpret_cast<int*>(base);
  double* norms = reinterpret_cast<double*>(base + o_norm);
  std::vector<char> up(total - o_rec, 0);
  memcpy(up.data(), recs.data(), sizeof(TcStage));
  memcpy(up.data() + (o_img - o_rec), img.data(), img.size() * sizeof(float));
  if (qc_status st = check_cuda(cudaMemsetAsync(status, 0, sizeof(int), s->stream), "status reset")) return st;
  if (qc_status st = check_cuda(cudaMemcpyAsync(base + o_rec, up.data(), up.size(), cudaMemcpyHostToDevice, s->stream),
                                "block upload"))
    return st;
  if (qc_status st = tc_pass_smem()) return st;
  TcNorm nm{};
  nm.nblocks = int(grid);
  nm.in_part = norms;
  nm.out_prev = norms;
  nm.out_cur = norms;
  if (qc_status st = launch_tc_pass(s, P, tm, false, reinterpret_cast<const TcStage*>(base + o_rec),
                                    reinterpret_cast<const float*>(base + o_img), status, nm, grid))
    return st;
  if (qc_status st = check_launch("tensor-core block pass")) return st;
  int h = 0;
  if (qc_status st = check_cuda(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s->stream), "status"))
    return st;
  // the host staging buffer `up` is read by the copy above before the stream is done
  if (qc_status st = check_cuda(cudaStreamSynchronize(s->stream), "tensor-core block pass")) return st;
  *handled = true;
  return device_status(h, "tensor-core block pass");
}

// the box plan's fields as plain integers: dims[3 d + {0, 1, 2}] = first bit, bits, copied
// whole; coords[0] = coordinate bits, coords[1 + 2 q + {0, 1}] = dimension, bit in it
static void box_plan_out(const TcTma& tm, const std::vector<int>& Bloc, int* local_bits, int* dims, int* coords) {
  for (int i = 0; i < kTtM; ++i) local_bits[i] = Bloc[i];
  for (int d = 0; d < 5; ++d) {
    dims[3 * d] = tm.start[d];
    dims[3 * d + 1] = tm.len[d];
    dims[3 * d + 2] = tm.tile[d];
  }
  coords[0] = tm.nc;
  for (int q = 0; q < kTtMaxCoordBits; ++q) {
    coords[1 + 2 * q] = q < tm.nc ? tm.cdim[q] : -1;
    coords[2 + 2 * q] = q < tm.nc ? tm.coff[q] : -1;
  }
}

}  // namespace qcgb

using namespace qcgb;

extern "C" qc_status qc_tc_box_plan(int n, const int* tile_bits, int* local_bits, int* dims, int* coords) {
  clear_error();
  if (n < kTtM || n > 34 || !tile_bits || !local_bits || !dims || !coords) {
    set_error("qc_tc_box_plan: invalid arguments");
    return QC_ERR_INVALID_ARG;
  }
  std::vector<int> B;
  uint64_t seen = 0;
  for (int i = 0; i < kTtM; ++i) {
    const int b = tile_bits[i];
    if (b < 0 || b >= n || ((seen >> b) & 1)) {
      set_error("qc_tc_box_plan: tile bits must be %d distinct bits below n", kTtM);
      return QC_ERR_INVALID_ARG;
    }
    seen |= uint64_t(1) << b;
  }
  for (int b = 0; b < n; ++b)
    if ((seen >> b) & 1) B.push_back(b);
  std::vector<int> Bloc;
  const TcTma tm = tma_plan(B, n, Bloc);
  if (!tm.tma) {
    set_error("qc_tc_box_plan: no box plan with at most %d coordinate bits", kTtMaxCoordBits);
    return QC_ERR_UNSUPPORTED;
  }
  box_plan_out(tm, Bloc, local_bits, dims, coords);
  return QC_OK;
}

extern "C" qc_status qc_tc_block_plan(int n, const int* qubits, int k, int* local_bits, int* dims, int* coords) {
  clear_error();
  if (n < kTtM || n > 34 || !qubits || k < 1 || k > kTtSB || !local_bits || !dims || !coords) {
    set_error("qc_tc_block_plan: invalid arguments");
    return QC_ERR_INVALID_ARG;
  }
  int bits[kTtSB];
  for (int j = 0; j < k; ++j) {
    if (qubits[j] < 0 || qubits[j] >= n) {
      set_error("qc_tc_block_plan: qubit %d out of range", qubits[j]);
      return QC_ERR_INVALID_ARG;
    }
    bits[j] = n - 1 - qubits[j];
    for (int i = 0; i < j; ++i)
      if (bits[i] == bits[j]) {
        set_error("qc_tc_block_plan: repeated qubit %d", qubits[j]);
        return QC_ERR_INVALID_ARG;
      }
  }
  std::vector<int> Bloc;
  const TcTma tm = block_tile_plan(bits, k, n, Bloc);
  if (!tm.tma) {
    set_error("qc_tc_block_plan: no tile of the block has a box plan");
    return QC_ERR_UNSUPPORTED;
  }
  box_plan_out(tm, Bloc, local_bits, dims, coords);
  return QC_OK;
}

extern "C" qc_status qc_tc_emulate(const qc_circuit* c, const double* params, double* state) {
  clear_error();
  if (!c || !state || c->n < kTtM || c->n > 26 || (c->nops > 0 && !c->ops)) {
    set_error("qc_tc_emulate: invalid arguments (%d <= n <= 26)", kTtM);
    return QC_ERR_INVALID_ARG;
  }
  const int n = c->n;
  std::vector<ResolvedOp> rops(size_t(c->nops));
  for (int i = 0; i < c->nops; ++i)
    if (qc_status st = resolve_op(c, c->ops[i], params, &rops[size_t(i)])) return st;
  std::vector<std::vector<cd>> blocks;
  std::vector<std::array<int8_t, 5>> slots;
  TcHostPlan hp;
  hp.blocks = &blocks;
  hp.slots = &slots;
  if (!tc_build(n, rops, nullptr, hp)) {
    set_error("qc_tc_emulate: the circuit does not fit the tensor-core stages");
    return QC_ERR_UNSUPPORTED;
  }
  cd* a = reinterpret_cast<cd*>(state);
  constexpr uint32_t T = 1u << kTtM;
  const uint64_t ntiles = uint64_t(1) << (n - kTtM);
  std::vector<cd> tile(T), tmp(T);
  for (const TilePass& P : hp.passes) {
    bool in[64] = {false};
    for (int k = 0; k < kTtM; ++k) in[P.bits[k]] = true;
    std::vector<int> tnb;  // bit i of a tile number sits at global bit tnb[i]
    for (int b = 0; b < n; ++b)
      if (!in[b]) tnb.push_back(b);
    for (uint64_t t = 0; t < ntiles; ++t) {
      uint64_t base = 0;
      for (size_t i = 0; i < tnb.size(); ++i)
        if ((t >> i) & 1) base |= uint64_t(1) << tnb[i];
      auto addr = [&](uint32_t u) {
        uint64_t g = base;
        for (int k = 0; k < kTtM; ++k)
          if ((u >> k) & 1) g |= uint64_t(1) << P.bits[k];
        return g;
      };
      for (uint32_t u = 0; u < T; ++u) tile[u] = a[addr(u)];
      for (int si = P.stage0; si < P.stage0 + P.nstages; ++si) {
        const TcStage& ts = hp.stages[size_t(si)];
        const std::vector<cd>& U = blocks[size_t(si)];
        const std::array<int8_t, 5>& sl = slots[size_t(si)];
        for (int r = 0; r < kTtRows; ++r) {
          uint32_t rb = 0;
          for (int b = 0; b < kTtM - kTtSB; ++b)
            if ((r >> b) & 1) rb |= 1u << ts.lane_bit[b];
          uint32_t pos[32];
          cd x[32], y[32];
          for (int cc = 0; cc < 32; ++cc) {
            uint32_t u = rb;
            for (int k = 0; k < kTtSB; ++k)
              if ((cc >> k) & 1) u |= 1u << sl[size_t(k)];
            pos[cc] = u;
            x[cc] = tile[u];
          }
          for (int d = 0; d < 32; ++d) {
            cd acc = 0.0;
            for (int cc = 0; cc < 32; ++cc) acc += U[size_t(d * 32 + cc)] * x[cc];
            y[d] = acc;
          }
          for (int f = 0; f < ts.ndef; ++f) {  // deferred factors: row table times the tile's value
            const size_t src = size_t(ts.def0 + f);
            const float* rt = &hp.tabs.row[src * 256 + size_t(2 * r)];
            const float* gt = &hp.tabs.glob[src * 1536];
            cd fac(rt[0], rt[1]);
            for (int ch = 0; ch < 3; ++ch) {
              const size_t v = size_t((t >> (8 * ch)) & 255);
              fac *= cd(gt[2 * (ch * 256 + v)], gt[2 * (ch * 256 + v) + 1]);
            }
            const int key = ts.dkey[f];
            for (int d = 0; d < 32; ++d)
              if (key < 0 || ((d >> (key >> 1)) & 1) == (key & 1)) y[d] *= fac;
          }
          for (int d = 0; d < 32; ++d) tile[pos[d]] = y[d];
        }
      }
      if (P.permuted) {  // output u from the position whose bit rbit[k] is bit k of u
        for (uint32_t u = 0; u < T; ++u) {
          uint32_t v = 0;
          for (int k = 0; k < kTtM; ++k) v |= ((u >> k) & 1u) << P.rbit[k];
          tmp[u] = tile[v];
        }
        tile.swap(tmp);
      }
      for (uint32_t u = 0; u < T; ++u) a[addr(u)] = tile[u];
    }
  }
  return QC_OK;
}

extern "C" qc_status qc_tc_plan_info(const qc_circuit* c, const double* params, int* passes, int* stages,
                                     int* factors, int* copy_passes) {
  clear_error();
  if (!c || c->n < kTtM || c->n > 34 || (c->nops > 0 && !c->ops) || !passes || !stages || !factors ||
      !copy_passes) {
    set_error("qc_tc_plan_info: invalid arguments (%d <= n <= 34)", kTtM);
    return QC_ERR_INVALID_ARG;
  }
  std::vector<ResolvedOp> rops(size_t(c->nops));
  for (int i = 0; i < c->nops; ++i)
    if (qc_status st = resolve_op(c, c->ops[i], params, &rops[size_t(i)])) return st;
  TcHostPlan& hp = tc_scratch_plan();
  if (!tc_build(c->n, rops, nullptr, hp)) {
    set_error("qc_tc_plan_info: the circuit does not fit the tensor-core stages");
    return QC_ERR_UNSUPPORTED;
  }
  *passes = int(hp.passes.size());
  *stages = int(hp.stages.size());
  *factors = hp.tabs.count;
  int cp = 0;
  for (char d : hp.defer) cp += d == 2 ? 1 : 0;
  *copy_passes = cp;
  return QC_OK;
}
