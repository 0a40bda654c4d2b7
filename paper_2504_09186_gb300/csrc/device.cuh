// Device-side parameter blocks and storage helpers shared by the kernels.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tnc {

constexpr int kMaxTileBits = 16;  // per canonical tile set (M, N or K)
constexpr int kMaxOuter = 40;     // outer labels per set
constexpr int kThreads = 256;
constexpr int kStreamStages = 3;  // shared-memory ring depth of k_stream
// splits over K from which the partial sums are reduced by one warp per output
// (k_splitk_reduce_wide) instead of one thread per output
constexpr int kWideReduceSplit = 64;

// Storage conversion: FP32 arithmetic, fp32 / fp16 / bf16 storage (round to nearest even).
template <typename T>
struct Conv;
template <>
struct Conv<float> {
  static __device__ __forceinline__ float to_f(float x) { return x; }
  static __device__ __forceinline__ float from_f(float x) { return x; }
};
template <>
struct Conv<__half> {
  static __device__ __forceinline__ float to_f(__half x) { return __half2float(x); }
  static __device__ __forceinline__ __half from_f(float x) { return __float2half_rn(x); }
};
template <>
struct Conv<__nv_bfloat16> {
  static __device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }
  static __device__ __forceinline__ __nv_bfloat16 from_f(float x) { return __float2bfloat16_rn(x); }
};

// Tree-like reuse across slices (Sec. III-B).  Instances of a wave are row-major over
// (bitstring row, slice id) with s slice bits per row.  A step whose result depends only on
// the sliced indices in dep_c runs once per assignment of those indices: launch index z =
// row << popcount(dep_c) | assignment.  It writes the instance whose other slice bits are 0,
// and reads each operand at its own such instance (dep_a, dep_b are subsets of dep_c).
// s < 0: identity (every instance computed).
struct InstMap {
  int32_t s;
  uint32_t dep_c, dep_a, dep_b;
};
struct Inst3 {
  int64_t c, a, b;
};
__device__ __forceinline__ Inst3 map_inst(int64_t z, const InstMap& m) {
  if (m.s < 0) return Inst3{z, z, z};
  const int nd = __popc(m.dep_c);
  const int64_t row = z >> nd;
  uint32_t asg = (uint32_t)(z & ((int64_t(1) << nd) - 1));
  uint32_t slice = 0, msk = m.dep_c;
  while (msk) {
    const uint32_t low = msk & (~msk + 1u);
    if (asg & 1u) slice |= low;
    asg >>= 1;
    msk &= msk - 1;
  }
  const int64_t base = row << m.s;
  return Inst3{base | slice, base | (slice & m.dep_a), base | (slice & m.dep_b)};
}

// One pairwise contraction C = A * B with tiles over index sets (see compiler.cpp).
struct GenParams {
  const void* A;  // instance-0 base of A's real plane (imag plane at +planeA)
  const void* B;
  void* C;
  int64_t strideA, strideB, strideC;  // instance strides in scalars
  int64_t planeA, planeB, planeC;     // 2^rank
  int32_t mt, nt, kt;
  int32_t runA, runB, runC;           // low positions of each operand covered by the tile
  uint32_t maskA, maskB, maskC;       // tile positions in each operand
  int8_t pAm[kMaxTileBits], pAk[kMaxTileBits];  // tile-native bit of canonical bit j
  int8_t pBk[kMaxTileBits], pBn[kMaxTileBits];
  int8_t pCm[kMaxTileBits], pCn[kMaxTileBits];
  int32_t n_om, n_on, n_ok;
  int8_t om_A[kMaxOuter], om_C[kMaxOuter], on_B[kMaxOuter], on_C[kMaxOuter], ok_A[kMaxOuter], ok_B[kMaxOuter];
  int32_t splitk, kgroups;
  int32_t nK;                          // common labels (bound for the output scale)
  // scaling slots: value = stored * 2^exps[slot]; maxabs = max |re|,|im| of stored
  float* maxabs;
  int32_t* exps;
  int32_t n_slots, slotA, slotB, slotC;
  float2* partials;                    // split-K partial sums [inst][split][planeC]
  int32_t smem_tables;                 // byte offset of the index tables in shared memory
  int32_t stream;                      // 1: k_stream (raw tiles through a cp.async ring)
  int32_t kvb;                         // each K group takes chunks of 2^kvb consecutive k (0: one k)
  InstMap im;                          // launch index -> instances (tree-like reuse)
};

// One SIMT step of a wave inside the persistent steps kernel (k_steps): the contraction's
// units, then (split over K) the reduce's blocks after a grid barrier.
struct StepOp {
  GenParams p;
  int32_t rm, rn;   // register micro-tile
  int32_t reduce;   // 0: no split, 1: a thread per output, 2: a warp per output
  int32_t pad;
};

// Leaf gather: fix sliced legs and closed output legs, convert, scale.
struct LeafDesc {
  int64_t src;      // offset (complex entries) of the full leaf in the FP64 source array
  int64_t dst;      // scalar offset of the reduced leaf in the instance arena
  int32_t rank_full, rank, slot, nfix;
  int8_t fix_pos[8];
  int8_t fix_kind[8];   // 0 = slice bit, 1 = output bit of a qubit
  int16_t fix_idx[8];   // slice bit index or qubit
};

// Tensor-core complex GEMM step (tc_gemm.cu): 128 x 128 x 64 tiles.
struct TcParams {
  CUtensorMap tmA, tmB;      // TMA descriptors of A and B (tensor-memory-accelerator path only)
  const void* A;
  const void* B;
  void* C;
  int64_t strideA, strideB, strideC;
  int64_t planeA, planeB, planeC;
  int32_t bn, bk;            // tile width (64 / 128 / 256) and K tile (16 / 32)
  int32_t stages;            // 3 = short pipeline (two CTAs per SM), 0 = deepest
  int8_t pAm[7], pBn[8];     // operand positions of the canonical tile m / n bits
  int8_t pAk[3], pBk[3];     // operand positions of k bits 3..5 (bits 0..2 are positions 0..2)
  int8_t pCm[7], pCn[8];     // C-tile-native bit of canonical m / n bit
  uint32_t maskC;            // C positions of the tile (m and n labels)
  int32_t runC;
  int32_t n_om, n_on, n_ok;
  int8_t om_A[kMaxOuter], om_C[kMaxOuter], on_B[kMaxOuter], on_C[kMaxOuter], ok_A[kMaxOuter], ok_B[kMaxOuter];
  int32_t nK;
  int32_t splitk;            // CTAs along the outer K labels; > 1 writes FP32 partials
  float2* partials;          // [inst][split][planeC]
  int32_t bf16;              // operand format: 0 fp16, 1 bf16
  float* maxabs;
  int32_t* exps;
  int32_t n_slots, slotA, slotB, slotC;
  int32_t* status;           // TNC_E_TIMEOUT on a bounded wait that ran out
  int32_t persistent;        // 1 = persistent TMA kernel (short K loops, no split)
  int32_t direct;            // 1 = C's three lowest positions are tile columns 0..2: each
                             //     thread stores runs of 8 columns straight from registers
  int32_t n_inst;            // launch indices (persistent kernel: tiles span all)
  InstMap im;                // launch index -> instances (tree-like reuse)
};

// Fused chain of absorptions (Sec. IV): one tile of the big tensor stays on chip while
// every link contracts it with a small tensor.
constexpr int kChainMaxBits = 12;  // on-chip tile <= 2^12 complex entries per CTA
// Cluster-cooperative chains (Sec. IV: the core array's fused sections): a thread-block
// cluster of up to 2^3 CTAs holds a tile of up to 2^(12 + 3) entries in distributed shared
// memory, each CTA the 2^12 entries whose top tile bits equal its rank in the cluster.
constexpr int kChainClusterBits = 3;
struct ChainLink {
  int64_t g_off;     // arena offset (scalars, instance 0) of the small operand
  int64_t g_plane;   // 2^rank(small operand)
  int32_t slot_g, g_size, out_bits, k_bits, n_bits;
  uint16_t kin[64];  // tile offset of each common-label assignment in the previous tile
  uint8_t kg[64];    // ... and in the small operand
  uint8_t gn[64];    // small-operand offset of each free-label assignment (bound only)
  // output entry x -> (offset in the previous tile, offset in the small operand); both are
  // bit scatters of x, so they split over x's low and high six bits
  uint16_t ib_lo[64], ib_hi[64];
  uint8_t gb_lo[64], gb_hi[64];
  // ... and over the cluster rank (cluster-cooperative chain: x is the entry within the CTA,
  // the rank holds the tile's top cl_bits bits)
  uint16_t ib_top[8];
  uint8_t gb_top[8];
  int32_t in_ibits, out_ibits;  // per-CTA index bits of the link's input and output tiles
  int32_t remote;               // 1: some input entries sit in other CTAs of the cluster
};
struct ChainParams {
  const void* arena;
  int64_t stride;                     // instance stride (scalars)
  int64_t offA0, planeA0, offC, planeC;
  uint32_t maskA0, maskC;             // on-chip positions in the first operand / the result
  int32_t runA0, runC, bits0, bitsC;
  int32_t n_o;
  int8_t o_A[kMaxOuter], o_C[kMaxOuter];  // outer (grid) labels: positions in A0 and in C
  int32_t n_links;
  const ChainLink* links;
  float* maxabs;
  int32_t* exps;
  int32_t n_slots, slotA0, slotC;
  int32_t cl_bits;                    // log2 CTAs per cluster (0: one CTA holds the tile)
};

// Index permutation of a planar binary-index tensor (the transposes of TTGT, Sec. V-A,
// Sec. V-B): out[y] = in[x] where every label has the same bit in y (at its output
// position) as in x (at its input position).  Tiles are label sets holding the lowest
// positions of both layouts, so loads and stores are contiguous runs.
struct PermParams {
  const void* in;
  void* out;
  int64_t plane;              // 2^rank entries per plane (both tensors)
  int32_t bits;               // tile labels (<= 12)
  int32_t run_in, run_out;    // lowest positions of each layout inside the tile
  uint32_t mask_in, mask_out; // tile positions in each layout
  uint16_t plo[64], phi[64];  // output-tile index -> input-tile index (low / high 6 bits)
  int32_t n_o;                // outer labels (one CTA per assignment)
  int8_t o_in[kMaxOuter], o_out[kMaxOuter];
};

// A run of consecutive instances of one wave that belong to the same bitstring row.
struct RootSeg {
  int32_t row;
  int32_t begin, end;  // instances within the wave
};

// Raises a kernel's dynamic shared-memory limit once per (kernel, size) instead of on every
// launch (keeps attribute calls out of CUDA-graph captures after the first, eager launch).
cudaError_t set_smem_once(const void* kernel, size_t bytes);

}  // namespace tnc
