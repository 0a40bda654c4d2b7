// Tensor-core complex GEMM step for fp16 / bf16 storage (sm_103a, tcgen05 + TMEM).
//
// One pairwise contraction C = A * B (Sec. II-A: an M x K x N complex GEMM over the
// common indices) whose operands are large enough for 128 x 128 x 64 tiles.  Tiles are
// sets of indices, as in the SIMT kernel: the compiler places three common indices at
// the lowest positions of both operands, so every 8 consecutive entries of an operand
// are 8 consecutive k of one row and a row's 64-wide K tile is gathered with 16-byte
// cp.async copies straight into the 128B-swizzled K-major layout the tensor core reads;
// the other tile indices are scattered over the operands and handled by per-row address
// tables -- the permutation costs no extra pass (Sec. V-A: permutation inside the
// contraction kernel).
//
// Complex product with planar operands: per 16-wide k step, four MMAs into two FP32
// accumulators in TMEM,
//   Dr += Ar Br,  Dr += (-Ai) Bi  (negate-A bit),  Di += Ar Bi,  Di += Ai Br.
// Warp-specialized pipeline: warps 0..6 gather stages with cp.async, and after their own
// copies of a stage have landed (cp.async.wait_group) fence them to the async proxy and
// arrive on the stage's "full" mbarrier; one thread of warp 7 waits on "full", issues the
// MMAs and commits them to the stage's "empty" mbarrier, which the loaders wait on before
// reusing the buffer.  Every wait is bounded by the global timer; on timeout the kernel
// records TNC_E_TIMEOUT in a status word, stops issuing work and still releases its TMEM.  The epilogue reads TMEM (tcgen05.ld),
// applies the exact power-of-two scale, converts, stages the tile in shared memory in
// C's own order and writes contiguous runs.
#include "device.cuh"

namespace tnc {

constexpr int TC_BM = 128;                   // rows of A per tile (TMEM lanes)
constexpr int TC_THREADS = 256;
constexpr int TC_PIPE_BUDGET = 192 * 1024;   // shared memory for the operand pipeline
constexpr uint64_t TC_WAIT_NS = 2000000000ull;  // 2 s bound on any wait

// Compile-time shape of one tensor-core kernel instance: BN columns (64, 128 or 256), BK-wide
// K tiles (16 or 32 fp16 = 32 or 64-byte rows, swizzled 32B / 64B), NST pipeline stages.
template <int BN, int BK, int NST>
struct TcShape {
  static constexpr int ROWB = BK * 2;                         // bytes per tile row
  static constexpr int A_BYTES = TC_BM * ROWB;                // one plane of the A tile
  static constexpr int B_BYTES = BN * ROWB;                   // one plane of the B tile
  static constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;     // Ar, Ai, Br, Bi
  static constexpr int STAGES = NST;
  static constexpr int DIST = NST - 2;                        // loads in flight per loader
  static constexpr int PIPE = STAGES * STAGE;
  static constexpr int STG = TC_BM * BN * 2 * 2;              // staged C tile (2 planes, 16-bit)
  static constexpr int REGION = PIPE > STG ? PIPE : STG;
  static constexpr int SBO = 8 * ROWB;                        // bytes between 8-row groups
  static constexpr int LAYOUT = BK == 64 ? 2 : (BK == 32 ? 4 : 6);  // SW128 / SW64 / SW32
  static constexpr int CHUNKS = BK / 8;                        // 16-byte chunks per row
  static constexpr int TMEM_COLS = 2 * BN;                     // Dr, Di
  static constexpr int N_BITS = BN == 256 ? 8 : (BN == 128 ? 7 : (BN == 64 ? 6 : 5));
  static constexpr int C_BITS = 7 + N_BITS;                    // log2 entries of the C tile
  static_assert(STAGES >= 3 && PIPE <= TC_PIPE_BUDGET, "bad pipeline");
};
// deepest pipeline that fits the budget, at most 8 stages
template <int BN, int BK>
constexpr int tc_deep_stages() {
  return (TC_PIPE_BUDGET / (2 * TC_BM * BK * 2 + 2 * BN * BK * 2)) > 8 ? 8
                                                                       : (TC_PIPE_BUDGET / (2 * TC_BM * BK * 2 + 2 * BN * BK * 2));
}

// Byte offset of 16-byte chunk c of row r in a swizzled K-major tile with `rowb`-byte rows:
// the chunk index is XORed with address bits 7.. (the Swizzle<log2(rowb/16), 4, 3> pattern).
__device__ __forceinline__ uint32_t swz(uint32_t r, uint32_t c, uint32_t rowb) {
  const uint32_t off = r * rowb + c * 16;
  return off ^ (((off >> 7) & (rowb / 16 - 1)) << 4);
}

#ifndef TNC_TC_SELFCHECK
#define TNC_TC_SELFCHECK 0
#endif
// Self-check build (-DTNC_TC_SELFCHECK=1): every address is validated before use; the
// first violation is recorded in status[1..7] (code, block, thread, detail...) and the
// access is skipped instead of faulting.
__device__ __forceinline__ bool tc_check(bool good, int32_t* status, int code, int64_t d0, int64_t d1) {
#if TNC_TC_SELFCHECK
  if (!good) {
    if (atomicCAS(&status[1], 0, code) == 0) {
      status[2] = (int32_t)blockIdx.x;
      status[3] = (int32_t)threadIdx.x;
      status[4] = (int32_t)(d0 & 0xffffffff);
      status[5] = (int32_t)(d0 >> 32);
      status[6] = (int32_t)(d1 & 0xffffffff);
      status[7] = (int32_t)(d1 >> 32);
    }
    status[0] = 9;
  }
  return good;
#else
  (void)status; (void)code; (void)d0; (void)d1;
  return true;
#endif
}



__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
// 4-D tiled TMA load (coordinates innermost first) completing on an mbarrier.
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
// Bounded wait; returns false (and records a timeout) if the phase did not complete.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, int32_t* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > TC_WAIT_NS) {
      atomicExch(status, 4);  // TNC_E_TIMEOUT
      return false;
    }
  }
  return true;
}

// Shared-memory matrix descriptor: K-major, swizzled (layout 2 / 4 / 6 = 128B / 64B / 32B),
// 8-row groups `sbo` bytes apart.
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t saddr, uint32_t sbo, uint32_t layout) {
  uint64_t d = 0;
  d |= uint64_t((saddr >> 4) & 0x3FFFu);    // start address
  d |= uint64_t(1) << 16;                   // leading byte offset (unused for swizzled K-major)
  d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;  // stride byte offset: next 8-row group
  d |= uint64_t(1) << 46;                   // descriptor version (tcgen05)
  d |= uint64_t(layout) << 61;              // swizzle mode
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulate, K-major A and B, M = 128, N = n.
__device__ __forceinline__ uint32_t instr_desc(int bf16, int neg_a, int n) {
  uint32_t d = 0;
  d |= 1u << 4;                              // D format F32
  d |= uint32_t(bf16) << 7;                  // A format (0 F16, 1 BF16)
  d |= uint32_t(bf16) << 10;                 // B format
  d |= uint32_t(neg_a) << 13;                // negate A
  d |= uint32_t(n >> 3) << 17;               // N
  d |= uint32_t(TC_BM >> 4) << 24;           // M
  return d;
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// CH (32 or 16) consecutive TMEM columns of this warp's lanes.
template <int CH>
__device__ __forceinline__ void tmem_ldn(uint32_t taddr, float* v) {
  if constexpr (CH == 32) tmem_ld32(taddr, v);
  else tmem_ld16(taddr, v);
}

// Two values converted as Conv<T>::from_f does, packed low-first (the byte order of two
// consecutive entries in memory).
template <typename T>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
  const T x = Conv<T>::from_f(a), y = Conv<T>::from_f(b);
  uint16_t ux, uy;
  memcpy(&ux, &x, 2);
  memcpy(&uy, &y, 2);
  return uint32_t(ux) | (uint32_t(uy) << 16);
}

// Eight 16-bit values, one 16-byte store.
template <typename T>
struct alignas(16) Vec8 {
  T v[8];
};

// Staging-buffer swizzle: 16-byte chunks of each 128-byte group are permuted by higher index
// bits, so the threads of a warp (one tile row each) do not all hit one bank when rows are
// far apart in C's order; reads of whole 16-byte chunks stay contiguous.
__device__ __forceinline__ uint32_t stg_swz(uint32_t idx) {
  return idx ^ ((((idx >> 7) ^ (idx >> 10) ^ (idx >> 13)) & 7u) << 3);
}

// Epilogue shared by both tensor-core kernels: TMEM -> registers -> (split: FP32 partials)
// or (scale, convert, stage in C's own order, contiguous 16-byte stores); frees TMEM.
template <typename T, int BN, int TMEM_COLS>
__device__ __forceinline__ void tc_epilogue(const TcParams& p, uint32_t tmem, bool ok, unsigned char* smem,
                                            const uint16_t* TCm, const uint16_t* TCn, const uint32_t* hiC, float* red,
                                            int64_t oC, const Inst3 I) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t sa = I.a * p.n_slots, sbb = I.b * p.n_slots, sc = I.c * p.n_slots;
  const uint32_t lane_addr = uint32_t((warp & 3) * 32) << 16;
  const int row = (warp & 3) * 32 + lane;
  const int col0 = (warp >> 2) * (BN / 2);
  constexpr int CH = BN / 2 >= 32 ? 32 : 16;  // TMEM columns per load (16 for 32-wide tiles)
  if (p.splitk > 1) {
    // FP32 partial sums by C's flat index; k_splitk_reduce sums them in a fixed order
    if (ok) {
      float2* part = p.partials + (int64_t(blockIdx.z) * p.splitk + blockIdx.y) * p.planeC + oC;
      const uint32_t lowmask = (1u << p.runC) - 1u;
#pragma unroll 1
      for (int cc = 0; cc < BN / 2; cc += CH) {
        float vr[CH], vi[CH];
        tmem_ldn<CH>(tmem + lane_addr + col0 + cc, vr);
        tmem_ldn<CH>(tmem + lane_addr + BN + col0 + cc, vi);
        const uint32_t rm = TCm[row];
#pragma unroll
        for (int j = 0; j < CH; ++j) {
          const uint32_t t = stg_swz(rm ^ TCn[col0 + cc + j]);  // the tables hold swizzled offsets
          part[hiC[t >> p.runC] + (t & lowmask)] = make_float2(vr[j], vi[j]);
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    return;
  }
  // epilogue: TMEM -> registers -> scaled, converted, staged in C-native order -> global
  int sh = 0;
  {
    const float a = p.maxabs[sa + p.slotA], b = p.maxabs[sbb + p.slotB];
    if (a > 0.f && b > 0.f) {
      int ea, eb;
      frexpf(a, &ea);
      frexpf(b, &eb);
      sh = ea + eb + p.nK + 1 - 15;
    }
  }
  const float scale = ldexpf(1.f, -sh);
  constexpr int CT = TC_BM * BN;  // entries of the C tile
  T* stg = reinterpret_cast<T*>(smem);  // [2][CT] re plane then im plane
  float mx = 0.f;
  if (ok && p.direct) {
    // columns 8g..8g+7 of a row are 8 consecutive entries of C: 16-byte stores from registers
    T* Cre = reinterpret_cast<T*>(p.C) + I.c * p.strideC + oC;
    const uint32_t lowmask = (1u << p.runC) - 1u;
    const uint32_t rm = TCm[row];
#pragma unroll 1
    for (int cc = 0; cc < BN / 2; cc += CH) {
      float vr[CH], vi[CH];
      tmem_ldn<CH>(tmem + lane_addr + col0 + cc, vr);
      tmem_ldn<CH>(tmem + lane_addr + BN + col0 + cc, vi);
#pragma unroll
      for (int g = 0; g < CH / 8; ++g) {
        const uint32_t t = stg_swz(rm ^ TCn[col0 + cc + 8 * g]);  // C-tile index, low 3 bits 0
        const uint32_t off = hiC[t >> p.runC] + (t & lowmask);
        Vec8<T> r8, i8;
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          r8.v[v] = Conv<T>::from_f(vr[8 * g + v] * scale);
          i8.v[v] = Conv<T>::from_f(vi[8 * g + v] * scale);
          mx = fmaxf(mx, fmaxf(fabsf(vr[8 * g + v]), fabsf(vi[8 * g + v])));
        }
        *reinterpret_cast<Vec8<T>*>(Cre + off) = r8;
        *reinterpret_cast<Vec8<T>*>(Cre + p.planeC + off) = i8;
      }
    }
    mx *= scale * (1.f + 0x1p-8f);
  } else if (ok) {
#pragma unroll 1
    for (int cc = 0; cc < BN / 2; cc += CH) {
      float vr[CH], vi[CH];
      tmem_ldn<CH>(tmem + lane_addr + col0 + cc, vr);
      tmem_ldn<CH>(tmem + lane_addr + BN + col0 + cc, vi);
      const uint32_t rm = TCm[row];
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        const uint32_t idx = rm ^ TCn[col0 + cc + j];  // swizzled staging index
#if TNC_TC_SELFCHECK
        if (!tc_check(idx < uint32_t(CT), p.status, 16, idx, row)) continue;
#endif
        stg[idx] = Conv<T>::from_f(vr[j] * scale);
        stg[CT + idx] = Conv<T>::from_f(vi[j] * scale);
        mx = fmaxf(mx, fmaxf(fabsf(vr[j]), fabsf(vi[j])));
      }
    }
    // max of the stored values: from the FP32 values, scaled, widened by the largest
    // rounding step of either 16-bit format so it never falls below the stored maximum
    mx *= scale * (1.f + 0x1p-8f);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
  if (!ok) return;
  // contiguous runs of C: 16-byte vectors (the compiler guarantees runC >= 3)
  T* Cre = reinterpret_cast<T*>(p.C) + I.c * p.strideC + oC;
  const uint32_t lowmask = (1u << p.runC) - 1u;
  for (int t = tid * 8; t < (p.direct ? 0 : CT); t += TC_THREADS * 8) {
    const uint32_t off = hiC[t >> p.runC] + (uint32_t(t) & lowmask);
#if TNC_TC_SELFCHECK
    {
      const int64_t ec = (Cre + off - reinterpret_cast<T*>(p.C)) - I.c * p.strideC;
      if (!tc_check(((reinterpret_cast<uintptr_t>(Cre + off) & 15u) == 0) && ec >= 0 && ec + 8 <= p.planeC, p.status, 17, ec, t))
        continue;
    }
#endif
    // 8 entries: one 16-byte vector of 16-bit values, two of FP32 values
    constexpr int VE = 16 / int(sizeof(T));
#pragma unroll
    for (int v = 0; v < 8 / VE; ++v) {
      *reinterpret_cast<uint4*>(Cre + off + v * VE) = *reinterpret_cast<const uint4*>(stg + stg_swz(t) + v * VE);
      *reinterpret_cast<uint4*>(Cre + p.planeC + off + v * VE) =
          *reinterpret_cast<const uint4*>(stg + CT + stg_swz(t) + v * VE);
    }
  }
  // block max -> tensor max
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) red[warp] = mx;
  __syncthreads();
  if (tid == 0) {
    float m = 0.f;
    for (int w = 0; w < TC_THREADS / 32; ++w) m = fmaxf(m, red[w]);
    atomicMax(reinterpret_cast<unsigned int*>(&p.maxabs[sc + p.slotC]), __float_as_uint(m));
    if (blockIdx.x == 0) p.exps[sc + p.slotC] = p.exps[sa + p.slotA] + p.exps[sbb + p.slotB] + sh;
  }
}

template <typename T, int BN, int BK, int NST>
__global__ void __launch_bounds__(TC_THREADS, (NST == 3 ? 2 : 1)) k_tc_gemm(const TcParams p) {
  using S = TcShape<BN, BK, NST>;
  constexpr int LOADERS = TC_THREADS - 32;  // warps 0..6 load, warp 7 issues the MMAs
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // 1024-byte aligned pipeline buffers (the swizzle pattern is address based)
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint32_t* depA = reinterpret_cast<uint32_t*>(smem + S::REGION);        // [128] row offsets in A
  uint32_t* depB = depA + TC_BM;                                         // [BN] row offsets in B
  uint32_t* hiC = depB + BN;                                             // [2^(C_BITS - runC)]
  const int nhC = 1 << (S::C_BITS - p.runC);
  uint16_t* TCm = reinterpret_cast<uint16_t*>(hiC + nhC);               // [128]
  uint16_t* TCn = TCm + TC_BM;                                           // [BN]
  uint64_t* bars = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(TCn + BN) + 15) & ~uintptr_t(7));
  uint64_t* full = bars;                    // [NST] loads of a stage have landed
  uint64_t* empty = bars + NST;             // [NST] MMAs reading a stage have completed
  uint64_t* done = bars + 2 * NST;          // all MMAs have completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NST + 1);
  float* red = reinterpret_cast<float*>(tmem_slot + 4);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const Inst3 I = map_inst(blockIdx.z, p.im);
  // grid.x enumerates (on fastest, om): CTAs sharing an A row tile run together
  const uint32_t on = blockIdx.x & ((1u << p.n_on) - 1u);
  const uint32_t om = p.n_on >= 31 ? 0u : (blockIdx.x >> p.n_on);
  int64_t oA = 0, oB = 0, oC = 0;
  for (int j = 0; j < p.n_om; ++j)
    if ((om >> j) & 1u) oA += int64_t(1) << p.om_A[j], oC += int64_t(1) << p.om_C[j];
  for (int j = 0; j < p.n_on; ++j)
    if ((on >> j) & 1u) oB += int64_t(1) << p.on_B[j], oC += int64_t(1) << p.on_C[j];
  const int nb = BN == 128 ? 7 : 6;

  // tables
  for (int r = tid; r < TC_BM; r += TC_THREADS) {
    uint32_t a = 0, cm = 0;
    for (int j = 0; j < 7; ++j)
      if ((r >> j) & 1) a |= 1u << p.pAm[j], cm |= 1u << p.pCm[j];
    depA[r] = a;
    TCm[r] = (uint16_t)stg_swz(cm);  // staging offsets, stored swizzled (stg_swz is linear)
  }
  for (int r = tid; r < BN; r += TC_THREADS) {
    uint32_t b = 0, cn = 0;
    for (int j = 0; j < nb; ++j)
      if ((r >> j) & 1) b |= 1u << p.pBn[j], cn |= 1u << p.pCn[j];
    depB[r] = b;
    TCn[r] = (uint16_t)stg_swz(cn);
  }
  for (int h = tid; h < nhC; h += TC_THREADS) {
    uint32_t m = p.maskC;
    for (int i = 0; i < p.runC; ++i) m &= m - 1;
    uint32_t r = 0, x = (uint32_t)h;
    while (m) {
      const uint32_t low = m & (~m + 1u);
      if (x & 1u) r |= low;
      x >>= 1;
      m &= m - 1;
    }
    hiC[h] = r;
  }
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(smem_u32(&full[s]), LOADERS);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(S::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;
#if TNC_TC_SELFCHECK
  tc_check((smem_u32(smem) & 1023u) == 0, p.status, 11, smem_u32(smem), 0);
  tc_check((tmem >> 16) == 0 && (tmem & 0xFFFFu) + S::TMEM_COLS <= 512, p.status, 12, tmem, 0);
  tc_check((smem_u32(bars) & 7u) == 0, p.status, 18, smem_u32(bars), 0);
#endif

  const T* Ab = reinterpret_cast<const T*>(p.A) + I.a * p.strideA + oA;
  const T* Bb = reinterpret_cast<const T*>(p.B) + I.b * p.strideB + oB;
  const int n_total = 1 << p.n_ok;
  const int per = n_total / p.splitk;
  const int it0 = blockIdx.y * per;
  const int n_iter = per;
  const uint32_t sbase = smem_u32(smem);

  // per stage: (128 + BN) rows x CHUNKS chunks of 16 B per plane; each (row, chunk) pair is
  // copied for the real and the imaginary plane
  constexpr int PAIRS = (TC_BM + BN) * S::CHUNKS;
  auto load_stage = [&](int it, int buf) {
    const int g = it0 + it;
    int64_t okA = 0, okB = 0;
    for (int j = 0; j < p.n_ok; ++j)
      if ((g >> j) & 1) okA += int64_t(1) << p.ok_A[j], okB += int64_t(1) << p.ok_B[j];
    const uint32_t st = sbase + buf * S::STAGE;
    for (int idx = tid; idx < PAIRS; idx += LOADERS) {
      const bool isA = idx < TC_BM * S::CHUNKS;
      const int li = isA ? idx : idx - TC_BM * S::CHUNKS;
      const int row = li / S::CHUNKS, c = li % S::CHUNKS;
      uint32_t kk = 0;
#pragma unroll
      for (int j = 0; j < 3; ++j)
        if ((c >> j) & 1) kk |= 1u << (isA ? p.pAk[j] : p.pBk[j]);
      const uint32_t so = swz(row, c, S::ROWB);
      const T* g0 = isA ? (Ab + okA + depA[row] + kk) : (Bb + okB + depB[row] + kk);
      const int64_t plane = isA ? p.planeA : p.planeB;
      const uint32_t d0 = st + (isA ? 0u : uint32_t(2 * S::A_BYTES)) + so;
      const uint32_t d1 = d0 + (isA ? uint32_t(S::A_BYTES) : uint32_t(S::B_BYTES));
#if TNC_TC_SELFCHECK
      {
        const int64_t e = isA ? (g0 - reinterpret_cast<const T*>(p.A)) - I.a * p.strideA
                              : (g0 - reinterpret_cast<const T*>(p.B)) - I.b * p.strideB;
        const bool good = ((reinterpret_cast<uintptr_t>(g0) & 15u) == 0) && e >= 0 && e + 8 <= plane &&
                          (d0 & 15u) == 0 && d1 + 16 <= sbase + S::PIPE;
        if (!tc_check(good, p.status, 13, e, isA)) continue;
      }
#endif
      cp_async16(d0, g0);
      cp_async16(d1, g0 + plane);
    }
  };

  bool ok = true;
  if (warp < 7) {
    // loaders
    for (int it = 0; it < n_iter && ok; ++it) {
      const int buf = it % NST;
      // the buffer was last read by the MMAs of iteration it - NST
      if (it >= NST) ok = mbar_wait_bounded(smem_u32(&empty[buf]), (uint32_t)((it / NST - 1) & 1), p.status);
      if (!ok) break;
      load_stage(it, buf);
      cp_async_commit();
      if (it >= S::DIST) {
        cp_async_wait<S::DIST>();  // own copies of iteration it - DIST have landed
        fence_async_shared();
        mbar_arrive(smem_u32(&full[(it - S::DIST) % NST]));
      }
    }
    cp_async_wait<0>();
    fence_async_shared();
    if (ok)
      for (int it = n_iter - S::DIST > 0 ? n_iter - S::DIST : 0; it < n_iter; ++it) mbar_arrive(smem_u32(&full[it % NST]));
  } else if (lane == 0) {
    // MMA issuer
    const uint32_t id_pos = instr_desc(p.bf16, 0, BN), id_neg = instr_desc(p.bf16, 1, BN);
    for (int it = 0; it < n_iter; ++it) {
      const int buf = it % NST;
      if (!mbar_wait_bounded(smem_u32(&full[buf]), (uint32_t)((it / NST) & 1), p.status)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t st = sbase + buf * S::STAGE;
#pragma unroll
      for (int j = 0; j < BK / 16; ++j) {
        const uint64_t ar = kmajor_desc(st + j * 32, S::SBO, S::LAYOUT);
        const uint64_t ai = kmajor_desc(st + S::A_BYTES + j * 32, S::SBO, S::LAYOUT);
        const uint64_t br = kmajor_desc(st + 2 * S::A_BYTES + j * 32, S::SBO, S::LAYOUT);
        const uint64_t bi = kmajor_desc(st + 2 * S::A_BYTES + S::B_BYTES + j * 32, S::SBO, S::LAYOUT);
        const uint32_t first = (it == 0 && j == 0) ? 0u : 1u;
        mma_f16(tmem, ar, br, id_pos, first);        // Dr  = Ar Br
        mma_f16(tmem, ai, bi, id_neg, 1u);           // Dr -= Ai Bi
        mma_f16(tmem + BN, ar, bi, id_pos, first);   // Di  = Ar Bi
        mma_f16(tmem + BN, ai, br, id_pos, 1u);      // Di += Ai Br
      }
      mma_commit(smem_u32(&empty[buf]));
    }
    mma_commit(smem_u32(done));  // arrives once every MMA issued above has completed
  }
  // all MMAs done (waited for even after a timeout, so TMEM is never freed under them)
  const bool fin = mbar_wait_bounded(smem_u32(done), 0u, p.status);
  ok = ok && fin;
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  ok = __syncthreads_and(ok);

  tc_epilogue<T, BN, S::TMEM_COLS>(p, tmem, ok, smem, TCm, TCn, hiC, red, oC, I);
}

// Tensor-memory-accelerator variant: the compiler laid the operands out as [Kt | Mt | ...]
// and [Kt | Nt | ...], so a stage's A (B) tile is 128 (BN) consecutive rows of 2^kt
// entries, one 4-D box (k, row, plane, instance) per plane.  One thread issues the four
// TMA loads of a stage against the "full" mbarrier (expect_tx), one thread issues the
// MMAs and commits them to "empty"; the TMA swizzle (32B / 64B) writes exactly the K-major
// layout the MMA descriptors read.
template <typename T, int BN, int BK, int NST>
__global__ void __launch_bounds__(TC_THREADS, (NST == 3 ? 2 : 1)) k_tc_tma(const __grid_constant__ TcParams p) {
  using S = TcShape<BN, BK, NST>;
  constexpr int KT = BK == 32 ? 5 : 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint32_t* hiC = reinterpret_cast<uint32_t*>(smem + S::REGION);        // [2^(C_BITS - runC)]
  const int nhC = 1 << (S::C_BITS - p.runC);
  uint16_t* TCm = reinterpret_cast<uint16_t*>(hiC + nhC);               // [128]
  uint16_t* TCn = TCm + TC_BM;                                           // [BN]
  uint64_t* bars = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(TCn + BN) + 15) & ~uintptr_t(7));
  uint64_t* full = bars;
  uint64_t* empty = bars + NST;
  uint64_t* done = bars + 2 * NST;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NST + 1);
  float* red = reinterpret_cast<float*>(tmem_slot + 4);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const Inst3 I = map_inst(blockIdx.z, p.im);
  const uint32_t on = blockIdx.x & ((1u << p.n_on) - 1u);
  const uint32_t om = p.n_on >= 31 ? 0u : (blockIdx.x >> p.n_on);
  int64_t oA = 0, oB = 0, oC = 0;
  for (int j = 0; j < p.n_om; ++j)
    if ((om >> j) & 1u) oA += int64_t(1) << p.om_A[j], oC += int64_t(1) << p.om_C[j];
  for (int j = 0; j < p.n_on; ++j)
    if ((on >> j) & 1u) oB += int64_t(1) << p.on_B[j], oC += int64_t(1) << p.on_C[j];
  constexpr int nb = S::N_BITS;
  for (int r = tid; r < TC_BM; r += TC_THREADS) {
    uint32_t cm = 0;
    for (int j = 0; j < 7; ++j)
      if ((r >> j) & 1) cm |= 1u << p.pCm[j];
    TCm[r] = (uint16_t)stg_swz(cm);  // staging offsets, stored swizzled (stg_swz is linear)
  }
  for (int r = tid; r < BN; r += TC_THREADS) {
    uint32_t cn = 0;
    for (int j = 0; j < nb; ++j)
      if ((r >> j) & 1) cn |= 1u << p.pCn[j];
    TCn[r] = (uint16_t)stg_swz(cn);
  }
  for (int h = tid; h < nhC; h += TC_THREADS) {
    uint32_t m = p.maskC;
    for (int i = 0; i < p.runC; ++i) m &= m - 1;
    uint32_t r = 0, x = (uint32_t)h;
    while (m) {
      const uint32_t low = m & (~m + 1u);
      if (x & 1u) r |= low;
      x >>= 1;
      m &= m - 1;
    }
    hiC[h] = r;
  }
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(S::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  const int n_total = 1 << p.n_ok;
  const int per = n_total / p.splitk;
  const int it0 = blockIdx.y * per;
  const int n_iter = per;
  const uint32_t sbase = smem_u32(smem);
  bool ok = true;
  if (warp == 0 && lane == 0) {
    // TMA producer
    int issued = 0;
    for (int it = 0; it < n_iter; ++it) {
      const int buf = it % NST;
      if (it >= NST && !mbar_wait_bounded(smem_u32(&empty[buf]), (uint32_t)((it / NST - 1) & 1), p.status)) {
        ok = false;
        break;
      }
      const int g = it0 + it;
      int64_t okA = 0, okB = 0;
      for (int j = 0; j < p.n_ok; ++j)
        if ((g >> j) & 1) okA += int64_t(1) << p.ok_A[j], okB += int64_t(1) << p.ok_B[j];
      const int rowA = (int)((oA + okA) >> KT), rowB = (int)((oB + okB) >> KT);
      const uint32_t st = sbase + buf * S::STAGE;
      const uint32_t fb = smem_u32(&full[buf]);
      mbar_arrive_expect_tx(fb, S::STAGE);
      tma_load_4d(st, &p.tmA, 0, rowA, 0, (int)I.a, fb);
      tma_load_4d(st + S::A_BYTES, &p.tmA, 0, rowA, 1, (int)I.a, fb);
      tma_load_4d(st + 2 * S::A_BYTES, &p.tmB, 0, rowB, 0, (int)I.b, fb);
      tma_load_4d(st + 2 * S::A_BYTES + S::B_BYTES, &p.tmB, 0, rowB, 1, (int)I.b, fb);
      issued = it + 1;
    }
    // copies still in flight land before the CTA may exit (all complete on the normal path)
    for (int it = issued - NST > 0 ? issued - NST : 0; it < issued; ++it)
      if (!mbar_wait_bounded(smem_u32(&full[it % NST]), (uint32_t)((it / NST) & 1), p.status)) ok = false;
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t id_pos = instr_desc(p.bf16, 0, BN), id_neg = instr_desc(p.bf16, 1, BN);
    for (int it = 0; it < n_iter; ++it) {
      const int buf = it % NST;
      if (!mbar_wait_bounded(smem_u32(&full[buf]), (uint32_t)((it / NST) & 1), p.status)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t st = sbase + buf * S::STAGE;
#pragma unroll
      for (int j = 0; j < BK / 16; ++j) {
        const uint64_t ar = kmajor_desc(st + j * 32, S::SBO, S::LAYOUT);
        const uint64_t ai = kmajor_desc(st + S::A_BYTES + j * 32, S::SBO, S::LAYOUT);
        const uint64_t br = kmajor_desc(st + 2 * S::A_BYTES + j * 32, S::SBO, S::LAYOUT);
        const uint64_t bi = kmajor_desc(st + 2 * S::A_BYTES + S::B_BYTES + j * 32, S::SBO, S::LAYOUT);
        const uint32_t first = (it == 0 && j == 0) ? 0u : 1u;
        mma_f16(tmem, ar, br, id_pos, first);
        mma_f16(tmem, ai, bi, id_neg, 1u);
        mma_f16(tmem + BN, ar, bi, id_pos, first);
        mma_f16(tmem + BN, ai, br, id_pos, 1u);
      }
      mma_commit(smem_u32(&empty[buf]));
    }
    mma_commit(smem_u32(done));
  }
  const bool fin = mbar_wait_bounded(smem_u32(done), 0u, p.status);
  ok = ok && fin;
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  ok = __syncthreads_and(ok);
  tc_epilogue<T, BN, S::TMEM_COLS>(p, tmem, ok, smem, TCm, TCn, hiC, red, oC, I);
}

// Complex64 on the tensor cores (3xTF32).  kind::tf32 MMAs read 32-bit operands with a
// 10-bit stored mantissa, so each FP32 operand entry x is split in shared memory into
// hi = x rounded to TF32 and lo = (x - hi) rounded to TF32 (x - hi is exact in FP32), and
// every real product is taken as hi_a hi_b + hi_a lo_b + lo_a hi_b: the dropped lo_a lo_b
// and the rounding of lo are each about 2^-22 of |a b|.  Per 8-wide k step twelve MMAs
// (six per accumulator) form
//   Dr = Ar Br - Ai Bi,  Di = Ar Bi + Ai Br   (each product in three parts).
// The tensor core adds into its FP32 accumulator without rounding to nearest (the sums are
// cut toward zero), a bias that grows with the length of the accumulation: over a K loop
// of 2^12 it shrank results by about 2e-4.  So each 8-wide k step accumulates from zero
// into one of two TMEM buffers, and the drain warps add that chunk to FP32 sums held in
// registers with ordinary round-to-nearest adds while the MMAs fill the other buffer; the
// biased chain is six MMAs long.
// The operand layouts are those of k_tc_tma ([Kt | Mt | ...], [Kt | Nt | ...]) with FP32
// entries: a K tile of 16 entries is one 64-byte row (SW64); a compiled 32-wide K tile is
// loaded as two halves through a 5-D tensor map (k low 16, k high bit, row, plane, instance).
// Warp roles (12 warps):
//   warp 0 lane 0   TMA loads of a stage's hi half, on "full";
//   warp 1 lane 0   waits on "conv", issues the MMAs of each k step into TMEM buffer
//                   (step & 1) after "acc empty", commits them to "acc full" and each stage
//                   to "empty";
//   warps 2..3      split the landed stage (hi in place, lo into the stage's second half),
//                   fence their writes to the async proxy and arrive on "conv";
//   warps 4..11     drain: lane quadrant (warp & 3), column half ((warp - 4) >> 2); add each
//                   chunk to the register sums, release the buffer on "acc empty"; then
//                   the epilogue (scale, FP32 stores, straight from registers or staged).
// Every wait is bounded as in the other kernels.
constexpr int TF32_THREADS = 384;
template <int BN>
struct Tf32Shape {
  static constexpr int ROWB = 64;                             // 16 FP32 entries per tile row
  static constexpr int A_BYTES = TC_BM * ROWB;                // one plane of the A tile
  static constexpr int B_BYTES = BN * ROWB;
  static constexpr int HALF = 2 * A_BYTES + 2 * B_BYTES;      // Ar, Ai, Br, Bi (hi parts)
  static constexpr int STAGE = 2 * HALF;                      // + their lo parts
  static constexpr int NST_FIT = TC_PIPE_BUDGET / STAGE;
  static constexpr int NST = NST_FIT > 4 ? 4 : NST_FIT;
  static constexpr int PIPE = NST * STAGE;
  static constexpr int STG = TC_BM * BN * 2 * 4;              // staged C tile (2 planes, FP32)
  static constexpr int REGION = PIPE > STG ? PIPE : STG;
  static constexpr int SBO = 8 * ROWB;
  static constexpr int LAYOUT = 4;                            // SW64
  static constexpr int TMEM_COLS = 4 * BN;                    // two buffers of (Dr, Di)
  static constexpr int N_BITS = BN == 128 ? 7 : (BN == 64 ? 6 : 5);
  static constexpr int C_BITS = 7 + N_BITS;
  static constexpr int CONV_THREADS = 64;                     // warps 2..3
  static constexpr int DRAIN_WARPS = 8;                       // warps 4..11
  static constexpr int HC = BN / 2;                           // columns per drain thread and plane
  static_assert(NST >= 3, "pipeline");
};

// Instruction descriptor, kind::tf32: FP32 accumulate, TF32 A and B (format 2), K-major.
__device__ __forceinline__ uint32_t instr_desc_tf32(int neg_a, int n) {
  uint32_t d = 0;
  d |= 1u << 4;                     // D format F32
  d |= 2u << 7;                     // A format TF32
  d |= 2u << 10;                    // B format TF32
  d |= uint32_t(neg_a) << 13;       // negate A
  d |= uint32_t(n >> 3) << 17;      // N
  d |= uint32_t(TC_BM >> 4) << 24;  // M
  return d;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// 5-D tiled TMA load (coordinates innermost first) completing on an mbarrier.
__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            int c4, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
      "%6}], [%7];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
      : "memory");
}

// Round an FP32 bit pattern to the nearest TF32 value (ties away from zero; finite inputs).
__device__ __forceinline__ uint32_t tf32_round_bits(uint32_t x) { return (x + 0x1000u) & 0xFFFFE000u; }

// Sixteen or thirty-two consecutive TMEM columns of this warp's lanes, added to acc.
template <int CH>
__device__ __forceinline__ void tmem_add(uint32_t taddr, float* acc) {
  float v[CH];
  tmem_ldn<CH>(taddr, v);
#pragma unroll
  for (int i = 0; i < CH; ++i) acc[i] += v[i];
}

template <int BN>
__global__ void __launch_bounds__(TF32_THREADS, 1) k_tc_tma_tf32(const __grid_constant__ TcParams p) {
  using S = Tf32Shape<BN>;
  constexpr int NST = S::NST;
  constexpr int HC = S::HC;
  constexpr int CH = HC >= 32 ? 32 : 16;
  constexpr int CT = TC_BM * BN;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint32_t* hiC = reinterpret_cast<uint32_t*>(smem + S::REGION);        // [2^(C_BITS - runC)]
  const int nhC = 1 << (S::C_BITS - p.runC);
  uint16_t* TCm = reinterpret_cast<uint16_t*>(hiC + nhC);               // [128]
  uint16_t* TCn = TCm + TC_BM;                                           // [BN]
  uint64_t* bars = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(TCn + BN) + 15) & ~uintptr_t(7));
  uint64_t* full = bars;                 // [NST] TMA loads of a stage have landed
  uint64_t* conv = bars + NST;           // [NST] the stage is split into hi and lo parts
  uint64_t* empty = bars + 2 * NST;      // [NST] the MMAs reading the stage have completed
  uint64_t* accf = bars + 3 * NST;       // [2] a k step's MMAs into TMEM buffer b completed
  uint64_t* acce = accf + 2;             // [2] TMEM buffer b drained
  uint64_t* done = acce + 2;             // all MMAs have completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  float* red = reinterpret_cast<float*>(tmem_slot + 4);                  // [12]

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const Inst3 I = map_inst(blockIdx.z, p.im);
  const uint32_t on = blockIdx.x & ((1u << p.n_on) - 1u);
  const uint32_t om = p.n_on >= 31 ? 0u : (blockIdx.x >> p.n_on);
  int64_t oA = 0, oB = 0, oC = 0;
  for (int j = 0; j < p.n_om; ++j)
    if ((om >> j) & 1u) oA += int64_t(1) << p.om_A[j], oC += int64_t(1) << p.om_C[j];
  for (int j = 0; j < p.n_on; ++j)
    if ((on >> j) & 1u) oB += int64_t(1) << p.on_B[j], oC += int64_t(1) << p.on_C[j];
  constexpr int nb = S::N_BITS;
  for (int r = tid; r < TC_BM; r += TF32_THREADS) {
    uint32_t cm = 0;
    for (int j = 0; j < 7; ++j)
      if ((r >> j) & 1) cm |= 1u << p.pCm[j];
    TCm[r] = (uint16_t)stg_swz(cm);
  }
  for (int r = tid; r < BN; r += TF32_THREADS) {
    uint32_t cn = 0;
    for (int j = 0; j < nb; ++j)
      if ((r >> j) & 1) cn |= 1u << p.pCn[j];
    TCn[r] = (uint16_t)stg_swz(cn);
  }
  for (int h = tid; h < nhC; h += TF32_THREADS) {
    uint32_t m = p.maskC;
    for (int i = 0; i < p.runC; ++i) m &= m - 1;
    uint32_t r = 0, x = (uint32_t)h;
    while (m) {
      const uint32_t low = m & (~m + 1u);
      if (x & 1u) r |= low;
      x >>= 1;
      m &= m - 1;
    }
    hiC[h] = r;
  }
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&conv[s]), S::CONV_THREADS);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&accf[b]), 1);
      mbar_init(smem_u32(&acce[b]), S::DRAIN_WARPS);
    }
    mbar_init(smem_u32(done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(S::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // a compiled 32-wide K tile (kt = 5) is loaded as two 16-wide halves
  const int kt = p.bk == 32 ? 5 : 4;
  const int halves = kt == 5 ? 2 : 1;
  const int n_total = 1 << p.n_ok;
  const int per = n_total / p.splitk;
  const int it0 = blockIdx.y * per;
  const int n_iter = per * halves;   // stages
  const int n_steps = 2 * n_iter;    // 8-wide k steps (TMEM chunks)
  const uint32_t sbase = smem_u32(smem);
  bool ok = true;
  float accR[HC], accI[HC];
#pragma unroll
  for (int i = 0; i < HC; ++i) accR[i] = accI[i] = 0.f;
  const int q = warp & 3, hcol = ((warp - 4) >> 2) * HC;  // drain warps: lane quadrant, first column
  if (warp == 0) {
    if (lane == 0) {
      // TMA producer: the hi half of each stage (Ar, Ai, Br, Bi as FP32)
      int issued = 0;
      for (int it = 0; it < n_iter; ++it) {
        const int buf = it % NST;
        if (it >= NST && !mbar_wait_bounded(smem_u32(&empty[buf]), (uint32_t)((it / NST - 1) & 1), p.status)) {
          ok = false;
          break;
        }
        const int g = it0 + it / halves, kh = it % halves;
        int64_t okA = 0, okB = 0;
        for (int j = 0; j < p.n_ok; ++j)
          if ((g >> j) & 1) okA += int64_t(1) << p.ok_A[j], okB += int64_t(1) << p.ok_B[j];
        const int rowA = (int)((oA + okA) >> kt), rowB = (int)((oB + okB) >> kt);
        const uint32_t st = sbase + buf * S::STAGE;
        const uint32_t fb = smem_u32(&full[buf]);
        mbar_arrive_expect_tx(fb, S::HALF);
        if (kt == 4) {
          tma_load_4d(st, &p.tmA, 0, rowA, 0, (int)I.a, fb);
          tma_load_4d(st + S::A_BYTES, &p.tmA, 0, rowA, 1, (int)I.a, fb);
          tma_load_4d(st + 2 * S::A_BYTES, &p.tmB, 0, rowB, 0, (int)I.b, fb);
          tma_load_4d(st + 2 * S::A_BYTES + S::B_BYTES, &p.tmB, 0, rowB, 1, (int)I.b, fb);
        } else {
          tma_load_5d(st, &p.tmA, 0, kh, rowA, 0, (int)I.a, fb);
          tma_load_5d(st + S::A_BYTES, &p.tmA, 0, kh, rowA, 1, (int)I.a, fb);
          tma_load_5d(st + 2 * S::A_BYTES, &p.tmB, 0, kh, rowB, 0, (int)I.b, fb);
          tma_load_5d(st + 2 * S::A_BYTES + S::B_BYTES, &p.tmB, 0, kh, rowB, 1, (int)I.b, fb);
        }
        issued = it + 1;
      }
      for (int it = issued - NST > 0 ? issued - NST : 0; it < issued; ++it)
        if (!mbar_wait_bounded(smem_u32(&full[it % NST]), (uint32_t)((it / NST) & 1), p.status)) ok = false;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer: k step u accumulates from zero into TMEM buffer u & 1
      const uint32_t id_pos = instr_desc_tf32(0, BN), id_neg = instr_desc_tf32(1, BN);
      for (int it = 0; it < n_iter && ok; ++it) {
        const int buf = it % NST;
        if (!mbar_wait_bounded(smem_u32(&conv[buf]), (uint32_t)((it / NST) & 1), p.status)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t st = sbase + buf * S::STAGE;
        for (int j = 0; j < 2; ++j) {
          const int u = 2 * it + j, b = u & 1;
          if (u >= 2 && !mbar_wait_bounded(smem_u32(&acce[b]), (uint32_t)((u / 2 - 1) & 1), p.status)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const uint32_t dr = tmem + b * 2 * BN, di = dr + BN;
          // 8 TF32 entries = 32 bytes of each row per MMA
          const uint32_t o = j * 32;
          const uint64_t arh = kmajor_desc(st + o, S::SBO, S::LAYOUT);
          const uint64_t aih = kmajor_desc(st + S::A_BYTES + o, S::SBO, S::LAYOUT);
          const uint64_t brh = kmajor_desc(st + 2 * S::A_BYTES + o, S::SBO, S::LAYOUT);
          const uint64_t bih = kmajor_desc(st + 2 * S::A_BYTES + S::B_BYTES + o, S::SBO, S::LAYOUT);
          const uint64_t arl = kmajor_desc(st + S::HALF + o, S::SBO, S::LAYOUT);
          const uint64_t ail = kmajor_desc(st + S::HALF + S::A_BYTES + o, S::SBO, S::LAYOUT);
          const uint64_t brl = kmajor_desc(st + S::HALF + 2 * S::A_BYTES + o, S::SBO, S::LAYOUT);
          const uint64_t bil = kmajor_desc(st + S::HALF + 2 * S::A_BYTES + S::B_BYTES + o, S::SBO, S::LAYOUT);
          // Dr = Ar Br - Ai Bi; the small cross terms first
          mma_tf32(dr, arh, brl, id_pos, 0u);
          mma_tf32(dr, arl, brh, id_pos, 1u);
          mma_tf32(dr, aih, bil, id_neg, 1u);
          mma_tf32(dr, ail, bih, id_neg, 1u);
          mma_tf32(dr, arh, brh, id_pos, 1u);
          mma_tf32(dr, aih, bih, id_neg, 1u);
          // Di = Ar Bi + Ai Br
          mma_tf32(di, arh, bil, id_pos, 0u);
          mma_tf32(di, arl, bih, id_pos, 1u);
          mma_tf32(di, aih, brl, id_pos, 1u);
          mma_tf32(di, ail, brh, id_pos, 1u);
          mma_tf32(di, arh, bih, id_pos, 1u);
          mma_tf32(di, aih, brh, id_pos, 1u);
          mma_commit(smem_u32(&accf[b]));
        }
        mma_commit(smem_u32(&empty[buf]));
      }
      mma_commit(smem_u32(done));
    }
  } else if (warp < 4) {
    // converters: hi = tf32(x) in place, lo = tf32(x - hi) in the stage's second half
    const int ct = tid - 64;
    for (int it = 0; it < n_iter; ++it) {
      const int buf = it % NST;
      if (!mbar_wait_bounded(smem_u32(&full[buf]), (uint32_t)((it / NST) & 1), p.status)) {
        ok = false;
        break;
      }
      uint4* hi = reinterpret_cast<uint4*>(smem + buf * S::STAGE);
      uint4* lo = reinterpret_cast<uint4*>(smem + buf * S::STAGE + S::HALF);
#pragma unroll 4
      for (int v = ct; v < S::HALF / 16; v += S::CONV_THREADS) {
        const uint4 x = hi[v];
        uint4 h, l;
        h.x = tf32_round_bits(x.x);
        h.y = tf32_round_bits(x.y);
        h.z = tf32_round_bits(x.z);
        h.w = tf32_round_bits(x.w);
        l.x = tf32_round_bits(__float_as_uint(__uint_as_float(x.x) - __uint_as_float(h.x)));
        l.y = tf32_round_bits(__float_as_uint(__uint_as_float(x.y) - __uint_as_float(h.y)));
        l.z = tf32_round_bits(__float_as_uint(__uint_as_float(x.z) - __uint_as_float(h.z)));
        l.w = tf32_round_bits(__float_as_uint(__uint_as_float(x.w) - __uint_as_float(h.w)));
        hi[v] = h;
        lo[v] = l;
      }
      fence_async_shared();  // the tensor core reads these writes through the async proxy
      mbar_arrive(smem_u32(&conv[buf]));
    }
  } else {
    // drain: add every k step's chunk to the register sums (round to nearest)
    const uint32_t lane_addr = uint32_t(q * 32) << 16;
    for (int u = 0; u < n_steps; ++u) {
      const int b = u & 1;
      bool got = true;
      if (lane == 0) got = mbar_wait_bounded(smem_u32(&accf[b]), (uint32_t)((u / 2) & 1), p.status);
      got = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
      if (!got) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t dr = tmem + lane_addr + b * 2 * BN + hcol;
#pragma unroll
      for (int c = 0; c < HC; c += CH) {
        tmem_add<CH>(dr + c, accR + c);
        tmem_add<CH>(dr + BN + c, accI + c);
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&acce[b]));
    }
  }
  // all MMAs done (waited for even after a timeout, so TMEM is never freed under them)
  const bool fin = mbar_wait_bounded(smem_u32(done), 0u, p.status);
  ok = ok && fin;
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  ok = __syncthreads_and(ok);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(S::TMEM_COLS) : "memory");
  if (!ok) return;
  // epilogue from the drain warps' registers (FP32 storage)
  const bool drain = warp >= 4;
  const int row = q * 32 + lane;
  const int64_t sa = I.a * p.n_slots, sbb = I.b * p.n_slots, sc = I.c * p.n_slots;
  const uint32_t lowmask = (1u << p.runC) - 1u;
  if (p.splitk > 1) {
    if (drain) {
      float2* part = p.partials + (int64_t(blockIdx.z) * p.splitk + blockIdx.y) * p.planeC + oC;
      const uint32_t rm = TCm[row];
#pragma unroll
      for (int j = 0; j < HC; ++j) {
        const uint32_t t = stg_swz(rm ^ TCn[hcol + j]);
        part[hiC[t >> p.runC] + (t & lowmask)] = make_float2(accR[j], accI[j]);
      }
    }
    return;
  }
  int sh = 0;
  {
    const float a = p.maxabs[sa + p.slotA], b = p.maxabs[sbb + p.slotB];
    if (a > 0.f && b > 0.f) {
      int ea, eb;
      frexpf(a, &ea);
      frexpf(b, &eb);
      sh = ea + eb + p.nK + 1 - 15;
    }
  }
  const float scale = ldexpf(1.f, -sh);
  float* stg = reinterpret_cast<float*>(smem);  // [2][CT]: the pipeline's buffers are free now
  float* Cre = reinterpret_cast<float*>(p.C) + I.c * p.strideC + oC;
  float mx = 0.f;
  if (drain) {
    const uint32_t rm = TCm[row];
#pragma unroll
    for (int j = 0; j < HC; ++j) mx = fmaxf(mx, fmaxf(fabsf(accR[j]), fabsf(accI[j])));
    if (p.direct) {
      // columns 8g..8g+7 of a row are 8 consecutive entries of C
#pragma unroll
      for (int g = 0; g < HC / 8; ++g) {
        const uint32_t t = stg_swz(rm ^ TCn[hcol + 8 * g]);
        const uint32_t off = hiC[t >> p.runC] + (t & lowmask);
        float4 r0, r1, i0, i1;
        r0 = make_float4(accR[8 * g] * scale, accR[8 * g + 1] * scale, accR[8 * g + 2] * scale, accR[8 * g + 3] * scale);
        r1 = make_float4(accR[8 * g + 4] * scale, accR[8 * g + 5] * scale, accR[8 * g + 6] * scale, accR[8 * g + 7] * scale);
        i0 = make_float4(accI[8 * g] * scale, accI[8 * g + 1] * scale, accI[8 * g + 2] * scale, accI[8 * g + 3] * scale);
        i1 = make_float4(accI[8 * g + 4] * scale, accI[8 * g + 5] * scale, accI[8 * g + 6] * scale, accI[8 * g + 7] * scale);
        *reinterpret_cast<float4*>(Cre + off) = r0;
        *reinterpret_cast<float4*>(Cre + off + 4) = r1;
        *reinterpret_cast<float4*>(Cre + p.planeC + off) = i0;
        *reinterpret_cast<float4*>(Cre + p.planeC + off + 4) = i1;
      }
    } else {
#pragma unroll
      for (int j = 0; j < HC; ++j) {
        const uint32_t idx = rm ^ TCn[hcol + j];  // swizzled staging index
        stg[idx] = accR[j] * scale;
        stg[CT + idx] = accI[j] * scale;
      }
    }
  }
  mx *= scale;
  __syncthreads();
  if (!p.direct) {
    for (int t = tid * 8; t < CT; t += TF32_THREADS * 8) {
      const uint32_t off = hiC[t >> p.runC] + (uint32_t(t) & lowmask);
      const uint32_t so = stg_swz(t);
      *reinterpret_cast<uint4*>(Cre + off) = *reinterpret_cast<const uint4*>(stg + so);
      *reinterpret_cast<uint4*>(Cre + off + 4) = *reinterpret_cast<const uint4*>(stg + so + 4);
      *reinterpret_cast<uint4*>(Cre + p.planeC + off) = *reinterpret_cast<const uint4*>(stg + CT + so);
      *reinterpret_cast<uint4*>(Cre + p.planeC + off + 4) = *reinterpret_cast<const uint4*>(stg + CT + so + 4);
    }
  }
  // block max -> tensor max
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) red[warp] = mx;
  __syncthreads();
  if (tid == 0) {
    float m = 0.f;
    for (int w = 0; w < TF32_THREADS / 32; ++w) m = fmaxf(m, red[w]);
    atomicMax(reinterpret_cast<unsigned int*>(&p.maxabs[sc + p.slotC]), __float_as_uint(m));
    if (blockIdx.x == 0) p.exps[sc + p.slotC] = p.exps[sa + p.slotA] + p.exps[sbb + p.slotB] + sh;
  }
}

// Persistent variant of k_tc_tma for short K loops (at most eight K tiles per output tile)
// over many output tiles.  One CTA per SM walks the tiles of all instances (instance-major,
// then the tile order of the one-CTA-per-tile launch) with a stride of gridDim.x; its j-th
// tile uses TMEM accumulator buffer j & 1:
//   NG epilogue groups (each GW warps: four TMEM lane quadrants x BN/CPW column slices):
//                    group g drains the CTA's tiles j = g (mod NG) -- scale, convert, stage in
//                    C's order in its own staging buffer, store -- and releases the buffer
//                    on "tmem empty".  With two groups (K loops of at most two K tiles) they
//                    work on consecutive tiles at once, so one group's stores overlap the
//                    other's staging; longer K loops keep one group and a deeper pipeline;
//   producer warp, lane 0   issues the TMA loads of every K tile through an NST-stage ring
//                    ("full" / "empty" mbarriers), running ahead across tiles;
//   MMA warp, lane 0        issues the MMAs of tile j into buffer j & 1 and commits them to
//                    "tmem full" of that buffer,
// so the epilogue of one tile also overlaps the loads and MMAs of the next.  Each group
// synchronises on its own named barrier; one thread per group waits on each mbarrier and
// shares the outcome, so a timeout ends the group's loop for all of its threads together.
template <int BN, int BK, int NG, bool DIRECT = false>
struct TcpShape {
  static constexpr int ROWB = BK * 2;
  static constexpr int A_BYTES = TC_BM * ROWB;
  static constexpr int B_BYTES = BN * ROWB;
  static constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
  // one staged C tile (2 planes, 16-bit); none when every tile stores straight from registers
  static constexpr int STG = DIRECT ? 0 : TC_BM * BN * 2 * 2;
  static constexpr int NST_FIT = (204 * 1024 - NG * STG) / STAGE;
  static constexpr int NST = NST_FIT > 6 ? 6 : NST_FIT;
  static constexpr int PIPE = NST * STAGE;
  static constexpr int SBO = 8 * ROWB;
  static constexpr int LAYOUT = BK == 32 ? 4 : 6;             // SW64 / SW32
  static constexpr int N_BITS = BN == 128 ? 7 : 6;
  static constexpr int C_BITS = 7 + N_BITS;
  static constexpr int TMEM_COLS = 4 * BN;                    // two buffers of (Dr, Di)
  static constexpr int CPW = NG == 2 ? 64 : 32;               // TMEM columns per epilogue warp
  static constexpr int GW = 4 * BN / CPW;                     // warps per epilogue group
  static constexpr int GT = GW * 32;                          // threads per epilogue group
  static constexpr int THREADS = NG * GT + 64;                // + producer warp + MMA warp
  static_assert(NG == 1 || NG == 2, "one or two epilogue groups");
  static_assert(BN == 64 || BN == 128, "two accumulator buffers need BN <= 128");
  static_assert(NST >= 2, "pipeline");
};

template <int N>
__device__ __forceinline__ void group_bar(int id) {
  __syncwarp();
  asm volatile("barrier.sync %0, %1;\n" ::"r"(id), "n"(N) : "memory");
}

template <typename T, int BN, int BK, int NG, bool DIRECT>
__global__ void __launch_bounds__(TcpShape<BN, BK, NG, DIRECT>::THREADS, 1)
    k_tc_tma_persist(const __grid_constant__ TcParams p) {
  using S = TcpShape<BN, BK, NG, DIRECT>;
  constexpr int KT = BK == 32 ? 5 : 4;
  constexpr int NST = S::NST;
  constexpr int CT = TC_BM * BN;  // entries of the C tile
  constexpr int NT = S::THREADS, GW = S::GW, GT = S::GT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  int64_t* oCt = reinterpret_cast<int64_t*>(smem + S::PIPE + NG * S::STG);   // [2][1024] C offsets of tile bits
  uint32_t* hiC = reinterpret_cast<uint32_t*>(oCt + 2048);                     // [2^(C_BITS - runC)]
  const int nhC = 1 << (S::C_BITS - p.runC);
  uint16_t* TCm = reinterpret_cast<uint16_t*>(hiC + nhC);                     // [128]
  uint16_t* TCn = TCm + TC_BM;                                                 // [BN]
  uint64_t* bars = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(TCn + BN) + 15) & ~uintptr_t(7));
  uint64_t* full = bars;
  uint64_t* empty = bars + NST;
  uint64_t* tfull = bars + 2 * NST;
  uint64_t* tempty = tfull + 2;
  uint64_t* done = tempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  float* red = reinterpret_cast<float*>(tmem_slot + 4);                       // [NG][2][GW]
  volatile int32_t* flag = reinterpret_cast<volatile int32_t*>(red + NG * 2 * GW);  // [NG]
  int32_t* cnt = const_cast<int32_t*>(flag) + NG;                               // [NG][2]

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int prod_warp = NG * GW, mma_warp = NG * GW + 1;
  constexpr int nb = S::N_BITS;
  for (int r = tid; r < TC_BM; r += NT) {
    uint32_t cm = 0;
    for (int j = 0; j < 7; ++j)
      if ((r >> j) & 1) cm |= 1u << p.pCm[j];
    TCm[r] = (uint16_t)stg_swz(cm);  // staging offsets, stored swizzled (stg_swz is linear)
  }
  for (int r = tid; r < BN; r += NT) {
    uint32_t cn = 0;
    for (int j = 0; j < nb; ++j)
      if ((r >> j) & 1) cn |= 1u << p.pCn[j];
    TCn[r] = (uint16_t)stg_swz(cn);
  }
  for (int h = tid; h < nhC; h += NT) {
    uint32_t m = p.maskC;
    for (int i = 0; i < p.runC; ++i) m &= m - 1;
    uint32_t r = 0, x = (uint32_t)h;
    while (m) {
      const uint32_t low = m & (~m + 1u);
      if (x & 1u) r |= low;
      x >>= 1;
      m &= m - 1;
    }
    hiC[h] = r;
  }
  // C offset of a tile index (within an instance) = oCt[0][bits 0..9] + oCt[1][bits 10..19]
  // (+ the bits from 20 up, summed in the epilogue): the deposit is additive over disjoint bits
  for (int x = tid; x < 2048; x += NT) {
    int64_t o = 0;
    for (int j = 0; j < 10; ++j) {
      const int b = (x >> 10) * 10 + j;  // tile-index bit
      if (!((x >> j) & 1)) continue;
      if (b < p.n_on) o += int64_t(1) << p.on_C[b];
      else if (b < p.n_on + p.n_om) o += int64_t(1) << p.om_C[b - p.n_on];
    }
    oCt[x] = o;
  }
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&tfull[b]), 1);
      // the direct epilogue's warps hand TMEM back one by one
      mbar_init(smem_u32(&tempty[b]), (DIRECT || p.direct) ? GW : 1);
    }
    mbar_init(smem_u32(done), 1);
    for (int q = 0; q < 2 * NG; ++q) cnt[q] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(S::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  const int tile_bits = p.n_om + p.n_on;
  const int64_t n_tiles = (int64_t(p.n_inst)) << tile_bits;
  const uint32_t tile_mask = (1u << tile_bits) - 1u;
  const int k_iters = 1 << p.n_ok;
  const uint32_t sbase = smem_u32(smem);
  bool ok = true;

  if (warp == prod_warp) {
    if (lane == 0) {
      // TMA producer
      int64_t g = 0, issued = 0;
      for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        const Inst3 It = map_inst(t >> tile_bits, p.im);
        const uint32_t r = (uint32_t)t & tile_mask;
        const uint32_t on = r & ((1u << p.n_on) - 1u);
        const uint32_t om = p.n_on >= 31 ? 0u : (r >> p.n_on);
        int64_t oA = 0, oB = 0;
        for (int j = 0; j < p.n_om; ++j)
          if ((om >> j) & 1u) oA += int64_t(1) << p.om_A[j];
        for (int j = 0; j < p.n_on; ++j)
          if ((on >> j) & 1u) oB += int64_t(1) << p.on_B[j];
        for (int it = 0; it < k_iters; ++it, ++g) {
          const int buf = (int)(g % NST);
          if (g >= NST && !mbar_wait_bounded(smem_u32(&empty[buf]), (uint32_t)(((g / NST) - 1) & 1), p.status)) {
            ok = false;
            break;
          }
          int64_t okA = 0, okB = 0;
          for (int j = 0; j < p.n_ok; ++j)
            if ((it >> j) & 1) okA += int64_t(1) << p.ok_A[j], okB += int64_t(1) << p.ok_B[j];
          const int rowA = (int)((oA + okA) >> KT), rowB = (int)((oB + okB) >> KT);
          const uint32_t st = sbase + buf * S::STAGE;
          const uint32_t fb = smem_u32(&full[buf]);
          mbar_arrive_expect_tx(fb, S::STAGE);
          tma_load_4d(st, &p.tmA, 0, rowA, 0, (int)It.a, fb);
          tma_load_4d(st + S::A_BYTES, &p.tmA, 0, rowA, 1, (int)It.a, fb);
          tma_load_4d(st + 2 * S::A_BYTES, &p.tmB, 0, rowB, 0, (int)It.b, fb);
          tma_load_4d(st + 2 * S::A_BYTES + S::B_BYTES, &p.tmB, 0, rowB, 1, (int)It.b, fb);
          issued = g + 1;
        }
      }
      // copies still in flight land before the CTA may exit
      for (int64_t x = issued - NST > 0 ? issued - NST : 0; x < issued; ++x)
        if (!mbar_wait_bounded(smem_u32(&full[x % NST]), (uint32_t)((x / NST) & 1), p.status)) ok = false;
    }
  } else if (warp == mma_warp) {
    if (lane == 0) {
      // MMA issuer
      const uint32_t id_pos = instr_desc(p.bf16, 0, BN), id_neg = instr_desc(p.bf16, 1, BN);
      int64_t g = 0;
      int j = 0;
      for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++j) {
        const int b = j & 1;
        if (j >= 2 && !mbar_wait_bounded(smem_u32(&tempty[b]), (uint32_t)(((j >> 1) - 1) & 1), p.status)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t acc = tmem + uint32_t(b * 2 * BN);
        for (int it = 0; it < k_iters; ++it, ++g) {
          const int buf = (int)(g % NST);
          if (!mbar_wait_bounded(smem_u32(&full[buf]), (uint32_t)((g / NST) & 1), p.status)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const uint32_t st = sbase + buf * S::STAGE;
#pragma unroll
          for (int jj = 0; jj < BK / 16; ++jj) {
            const uint64_t ar = kmajor_desc(st + jj * 32, S::SBO, S::LAYOUT);
            const uint64_t ai = kmajor_desc(st + S::A_BYTES + jj * 32, S::SBO, S::LAYOUT);
            const uint64_t br = kmajor_desc(st + 2 * S::A_BYTES + jj * 32, S::SBO, S::LAYOUT);
            const uint64_t bi = kmajor_desc(st + 2 * S::A_BYTES + S::B_BYTES + jj * 32, S::SBO, S::LAYOUT);
            const uint32_t first = (it == 0 && jj == 0) ? 0u : 1u;
            mma_f16(acc, ar, br, id_pos, first);
            mma_f16(acc, ai, bi, id_neg, 1u);
            mma_f16(acc + BN, ar, bi, id_pos, first);
            mma_f16(acc + BN, ai, br, id_pos, 1u);
          }
          mma_commit(smem_u32(&empty[buf]));
        }
        if (!ok) break;
        mma_commit(smem_u32(&tfull[b]));
      }
      // every MMA issued above completes before the CTA may free its TMEM
      mma_commit(smem_u32(done));
      if (!mbar_wait_bounded(smem_u32(done), 0u, p.status)) ok = false;
    }
  } else {
    // epilogue group gq: thread = one TMEM lane (row) of its warp's quadrant, CPW columns
    constexpr int CPW = S::CPW;
    const int gq = warp / GW, lw = warp % GW, gtid = tid - gq * GT;
    T* stg = reinterpret_cast<T*>(smem + S::PIPE + gq * S::STG);  // [2][CT]
    float* gred = red + gq * 2 * GW;
    const uint32_t lane_addr = uint32_t((warp & 3) * 32) << 16;
    const int row = (warp & 3) * 32 + lane;
    const int col0 = (lw >> 2) * CPW;
    const uint32_t lowmask = (1u << p.runC) - 1u;
    if (DIRECT || p.direct) {
      // Direct epilogue, warps independent: each waits for its tile, drains its TMEM columns
      // into 16-bit registers (scaled, converted), hands TMEM back (tempty counts the GW warps
      // of the group), then stores runs of 8 columns as 16-byte vectors (C's lowest positions
      // are tile columns 0..2, then row 0).  The group's maximum goes through a per-tile-parity
      // slot of red; the last warp of the group to finish (cnt) publishes it.  A warp reaches
      // tile j + 4 of its group only after every warp has handed back tile j + 2, i.e. has
      // finished tile j, so two parity slots suffice.
      const uint32_t rm = TCm[row];
      int64_t inst_cached = -1;
      int sh = 0;
      float scale = 1.f;
      int64_t sa = 0, sbb = 0, sc = 0;
      T* Cbase = nullptr;
      for (int64_t t = blockIdx.x + int64_t(gq) * gridDim.x, j = gq; t < n_tiles; t += NG * int64_t(gridDim.x), j += NG) {
        const int b = (int)(j & 1);
        const int par = (int)((j / NG) & 1);
        const uint32_t acc = tmem + uint32_t(b * 2 * BN);
        int wok = 1;
        if (lane == 0) wok = mbar_wait_bounded(smem_u32(&tfull[b]), (uint32_t)((j >> 1) & 1), p.status) ? 1 : 0;
        wok = __shfl_sync(0xffffffffu, wok, 0);
        if (!wok) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const int64_t inst = t >> tile_bits;
        if (inst != inst_cached) {
          inst_cached = inst;
          const Inst3 It = map_inst(inst, p.im);
          sa = It.a * p.n_slots;
          sbb = It.b * p.n_slots;
          sc = It.c * p.n_slots;
          sh = 0;
          const float a = p.maxabs[sa + p.slotA], bb = p.maxabs[sbb + p.slotB];
          if (a > 0.f && bb > 0.f) {
            int ea, eb;
            frexpf(a, &ea);
            frexpf(bb, &eb);
            sh = ea + eb + p.nK + 1 - 15;
          }
          scale = ldexpf(1.f, -sh);
          Cbase = reinterpret_cast<T*>(p.C) + It.c * p.strideC;
        }
        const uint32_t r = (uint32_t)t & tile_mask;
        int64_t oC = oCt[r & 1023u] + oCt[1024 + ((r >> 10) & 1023u)];
        for (int b = 20; b < tile_bits; ++b)
          if ((r >> b) & 1u) oC += int64_t(1) << (b < p.n_on ? p.on_C[b] : p.om_C[b - p.n_on]);
        T* Cre = Cbase + oC;
        float mx = 0.f;
        // columns 8g..8g+7 of the row are 8 consecutive entries of C: one 16-byte store per plane
        auto store8 = [&](int col, const uint32_t* r4, const uint32_t* i4) {
          const uint32_t x = stg_swz(rm ^ TCn[col]);  // C-tile index, low 3 bits 0
          const uint32_t off = hiC[x >> p.runC] + (x & lowmask);
          *reinterpret_cast<uint4*>(Cre + off) = make_uint4(r4[0], r4[1], r4[2], r4[3]);
          *reinterpret_cast<uint4*>(Cre + p.planeC + off) = make_uint4(i4[0], i4[1], i4[2], i4[3]);
        };
        // the first CPW - HOLD columns are stored as they are drained, the last HOLD are held
        // in registers while TMEM goes back to the MMA warp
        constexpr int HOLD = CPW / 2;
#pragma unroll 1
        for (int c = 0; c < CPW - HOLD; c += 16) {
          float vr[16], vi[16];
          tmem_ld16(acc + lane_addr + col0 + c, vr);
          tmem_ld16(acc + lane_addr + BN + col0 + c, vi);
#pragma unroll
          for (int g = 0; g < 2; ++g) {
            uint32_t r4[4], i4[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int v = 8 * g + 2 * q;
              r4[q] = pack2<T>(vr[v] * scale, vr[v + 1] * scale);
              i4[q] = pack2<T>(vi[v] * scale, vi[v + 1] * scale);
              mx = fmaxf(mx, fmaxf(fmaxf(fabsf(vr[v]), fabsf(vr[v + 1])), fmaxf(fabsf(vi[v]), fabsf(vi[v + 1]))));
            }
            store8(col0 + c + 8 * g, r4, i4);
          }
        }
        uint32_t pr[HOLD / 2], pi[HOLD / 2];
#pragma unroll
        for (int c = 0; c < HOLD; c += 16) {
          float vr[16], vi[16];
          tmem_ld16(acc + lane_addr + col0 + CPW - HOLD + c, vr);
          tmem_ld16(acc + lane_addr + BN + col0 + CPW - HOLD + c, vi);
#pragma unroll
          for (int q = 0; q < 16; q += 2) {
            pr[(c + q) >> 1] = pack2<T>(vr[q] * scale, vr[q + 1] * scale);
            pi[(c + q) >> 1] = pack2<T>(vi[q] * scale, vi[q + 1] * scale);
            mx = fmaxf(mx, fmaxf(fmaxf(fabsf(vr[q]), fabsf(vr[q + 1])), fmaxf(fabsf(vi[q]), fabsf(vi[q + 1]))));
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&tempty[b]));
#pragma unroll
        for (int g = 0; g < HOLD / 8; ++g) store8(col0 + CPW - HOLD + 8 * g, pr + 4 * g, pi + 4 * g);
        mx *= scale * (1.f + 0x1p-8f);  // bound on the stored maximum (see tc_epilogue)
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) {
          float* slot = red + (gq * 2 + par) * GW;
          slot[lw] = mx;
          __threadfence_block();
          if (atomicAdd(&cnt[gq * 2 + par], 1) == GW - 1) {
            __threadfence_block();
            float m = 0.f;
            for (int w = 0; w < GW; ++w) m = fmaxf(m, *reinterpret_cast<volatile float*>(&slot[w]));
            cnt[gq * 2 + par] = 0;
            atomicMax(reinterpret_cast<unsigned int*>(&p.maxabs[sc + p.slotC]), __float_as_uint(m));
            if (r == 0) p.exps[sc + p.slotC] = p.exps[sa + p.slotA] + p.exps[sbb + p.slotB] + sh;
          }
        }
      }
    }
    for (int64_t t = blockIdx.x + int64_t(gq) * gridDim.x, j = gq; t < n_tiles && !(DIRECT || p.direct);
         t += NG * int64_t(gridDim.x), j += NG) {
      const int b = (int)(j & 1);
      const uint32_t acc = tmem + uint32_t(b * 2 * BN);
      if (gtid == 0) flag[gq] = mbar_wait_bounded(smem_u32(&tfull[b]), (uint32_t)((j >> 1) & 1), p.status) ? 1 : 0;
      group_bar<GT>(1 + gq);
      if (flag[gq] == 0) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const Inst3 It = map_inst(t >> tile_bits, p.im);
      const uint32_t r = (uint32_t)t & tile_mask;
      const uint32_t on = r & ((1u << p.n_on) - 1u);
      const uint32_t om = p.n_on >= 31 ? 0u : (r >> p.n_on);
      int64_t oC = 0;
      for (int q = 0; q < p.n_om; ++q)
        if ((om >> q) & 1u) oC += int64_t(1) << p.om_C[q];
      for (int q = 0; q < p.n_on; ++q)
        if ((on >> q) & 1u) oC += int64_t(1) << p.on_C[q];
      const int64_t sa = It.a * p.n_slots, sbb = It.b * p.n_slots, sc = It.c * p.n_slots;
      int sh = 0;
      {
        const float a = p.maxabs[sa + p.slotA], bb = p.maxabs[sbb + p.slotB];
        if (a > 0.f && bb > 0.f) {
          int ea, eb;
          frexpf(a, &ea);
          frexpf(bb, &eb);
          sh = ea + eb + p.nK + 1 - 15;
        }
      }
      const float scale = ldexpf(1.f, -sh);
      float mx = 0.f;
      const uint32_t rm = TCm[row];
      T* Cre = reinterpret_cast<T*>(p.C) + It.c * p.strideC + oC;
      if constexpr (!DIRECT) {
#pragma unroll 1
      for (int cc = 0; cc < CPW; cc += 32) {
        float vr[32], vi[32];
        tmem_ld32(acc + lane_addr + col0 + cc, vr);
        tmem_ld32(acc + lane_addr + BN + col0 + cc, vi);
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const uint32_t idx = rm ^ TCn[col0 + cc + q];  // swizzled staging index
          stg[idx] = Conv<T>::from_f(vr[q] * scale);
          stg[CT + idx] = Conv<T>::from_f(vi[q] * scale);
          mx = fmaxf(mx, fmaxf(fabsf(vr[q]), fabsf(vi[q])));
        }
      }
      mx *= scale * (1.f + 0x1p-8f);  // bound on the stored maximum (see tc_epilogue)
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      group_bar<GT>(1 + gq);
      if (gtid == 0) mbar_arrive(smem_u32(&tempty[b]));
      // contiguous runs of C: 16-byte vectors (the compiler guarantees runC >= 3)
      for (int x = gtid * 8; x < CT; x += GT * 8) {
        const uint32_t off = hiC[x >> p.runC] + (uint32_t(x) & lowmask);
        *reinterpret_cast<uint4*>(Cre + off) = *reinterpret_cast<const uint4*>(stg + stg_swz(x));
        *reinterpret_cast<uint4*>(Cre + p.planeC + off) = *reinterpret_cast<const uint4*>(stg + CT + stg_swz(x));
      }
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0) gred[lw] = mx;
      group_bar<GT>(1 + gq);
      if (gtid == 0) {
        float m = 0.f;
        for (int w = 0; w < GW; ++w) m = fmaxf(m, gred[w]);
        atomicMax(reinterpret_cast<unsigned int*>(&p.maxabs[sc + p.slotC]), __float_as_uint(m));
        if (r == 0) p.exps[sc + p.slotC] = p.exps[sa + p.slotA] + p.exps[sbb + p.slotB] + sh;
      }
      }  // !DIRECT
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(S::TMEM_COLS) : "memory");
}

// Persistent variant for 256-wide tiles with the direct epilogue (tile columns 0..2 at C
// positions 0..2, row 0 at position 3).  The two accumulators of a 128 x 256 tile take all
// 512 TMEM columns, so there is one buffer.  The epilogue drains it into registers (each
// thread: one row, 128 columns of Dr and of Di, scaled and converted to 16-bit pairs, 128
// registers), hands TMEM back to the MMA warp at once, and stores from registers while the
// next tile's MMAs run.  The producer runs ahead through the ring, so the next tile's loads
// are in flight during the drain.  Warps 0..7: epilogue (TMEM lane quadrant warp & 3,
// column half warp >> 2); warp 8: TMA producer; warp 9: MMA issuer.
template <int BK>
struct TcwShape {
  static constexpr int BN = 256;
  static constexpr int ROWB = BK * 2;
  static constexpr int A_BYTES = TC_BM * ROWB;
  static constexpr int B_BYTES = BN * ROWB;
  static constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr int NST = (192 * 1024) / STAGE > 8 ? 8 : (192 * 1024) / STAGE;
  static constexpr int PIPE = NST * STAGE;
  static constexpr int SBO = 8 * ROWB;
  static constexpr int LAYOUT = BK == 32 ? 4 : 6;  // SW64 / SW32
  static constexpr int C_BITS = 15;
  static constexpr int TMEM_COLS = 512;
  static constexpr int EW = 8;                     // epilogue warps
  static constexpr int THREADS = EW * 32 + 64;     // + producer warp + MMA warp
  static constexpr int HOLD = 64;                  // columns per thread held in registers
  static_assert(NST >= 3, "pipeline");
};

template <typename T, int BK>
__global__ void __launch_bounds__(TcwShape<BK>::THREADS, 1) k_tc_tma_wide(const __grid_constant__ TcParams p) {
  using S = TcwShape<BK>;
  constexpr int BN = 256, KT = BK == 32 ? 5 : 4, NST = S::NST, NT = S::THREADS, ET = S::EW * 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint32_t* hiC = reinterpret_cast<uint32_t*>(smem + S::PIPE);  // [2^(C_BITS - runC)]
  const int nhC = 1 << (S::C_BITS - p.runC);
  uint16_t* TCm = reinterpret_cast<uint16_t*>(hiC + nhC);       // [128]
  uint16_t* TCn = TCm + TC_BM;                                   // [256]
  uint64_t* bars = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(TCn + BN) + 15) & ~uintptr_t(7));
  uint64_t* full = bars;
  uint64_t* empty = bars + NST;
  uint64_t* tfull = bars + 2 * NST;
  uint64_t* tempty = tfull + 1;
  uint64_t* done = tempty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  float* red = reinterpret_cast<float*>(tmem_slot + 4);                   // [EW]
  volatile int32_t* flag = reinterpret_cast<volatile int32_t*>(red + S::EW);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int prod_warp = S::EW, mma_warp = S::EW + 1;
  for (int r = tid; r < TC_BM; r += NT) {
    uint32_t cm = 0;
    for (int j = 0; j < 7; ++j)
      if ((r >> j) & 1) cm |= 1u << p.pCm[j];
    TCm[r] = (uint16_t)stg_swz(cm);
  }
  for (int r = tid; r < BN; r += NT) {
    uint32_t cn = 0;
    for (int j = 0; j < 8; ++j)
      if ((r >> j) & 1) cn |= 1u << p.pCn[j];
    TCn[r] = (uint16_t)stg_swz(cn);
  }
  for (int h = tid; h < nhC; h += NT) {
    uint32_t m = p.maskC;
    for (int i = 0; i < p.runC; ++i) m &= m - 1;
    uint32_t r = 0, x = (uint32_t)h;
    while (m) {
      const uint32_t low = m & (~m + 1u);
      if (x & 1u) r |= low;
      x >>= 1;
      m &= m - 1;
    }
    hiC[h] = r;
  }
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(tfull), 1);
    mbar_init(smem_u32(tempty), 1);
    mbar_init(smem_u32(done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"(S::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  const int tile_bits = p.n_om + p.n_on;
  const int64_t n_tiles = (int64_t(p.n_inst)) << tile_bits;
  const uint32_t tile_mask = (1u << tile_bits) - 1u;
  const int k_iters = 1 << p.n_ok;
  const uint32_t sbase = smem_u32(smem);
  bool ok = true;

  if (warp == prod_warp) {
    if (lane == 0) {
      // TMA producer (as in k_tc_tma_persist)
      int64_t g = 0, issued = 0;
      for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        const Inst3 It = map_inst(t >> tile_bits, p.im);
        const uint32_t r = (uint32_t)t & tile_mask;
        const uint32_t on = r & ((1u << p.n_on) - 1u);
        const uint32_t om = p.n_on >= 31 ? 0u : (r >> p.n_on);
        int64_t oA = 0, oB = 0;
        for (int j = 0; j < p.n_om; ++j)
          if ((om >> j) & 1u) oA += int64_t(1) << p.om_A[j];
        for (int j = 0; j < p.n_on; ++j)
          if ((on >> j) & 1u) oB += int64_t(1) << p.on_B[j];
        for (int it = 0; it < k_iters; ++it, ++g) {
          const int buf = (int)(g % NST);
          if (g >= NST && !mbar_wait_bounded(smem_u32(&empty[buf]), (uint32_t)(((g / NST) - 1) & 1), p.status)) {
            ok = false;
            break;
          }
          int64_t okA = 0, okB = 0;
          for (int j = 0; j < p.n_ok; ++j)
            if ((it >> j) & 1) okA += int64_t(1) << p.ok_A[j], okB += int64_t(1) << p.ok_B[j];
          const int rowA = (int)((oA + okA) >> KT), rowB = (int)((oB + okB) >> KT);
          const uint32_t st = sbase + buf * S::STAGE;
          const uint32_t fb = smem_u32(&full[buf]);
          mbar_arrive_expect_tx(fb, S::STAGE);
          tma_load_4d(st, &p.tmA, 0, rowA, 0, (int)It.a, fb);
          tma_load_4d(st + S::A_BYTES, &p.tmA, 0, rowA, 1, (int)It.a, fb);
          tma_load_4d(st + 2 * S::A_BYTES, &p.tmB, 0, rowB, 0, (int)It.b, fb);
          tma_load_4d(st + 2 * S::A_BYTES + S::B_BYTES, &p.tmB, 0, rowB, 1, (int)It.b, fb);
          issued = g + 1;
        }
      }
      for (int64_t x = issued - NST > 0 ? issued - NST : 0; x < issued; ++x)
        if (!mbar_wait_bounded(smem_u32(&full[x % NST]), (uint32_t)((x / NST) & 1), p.status)) ok = false;
    }
  } else if (warp == mma_warp) {
    if (lane == 0) {
      // MMA issuer: tile j waits until the epilogue has drained tile j - 1
      const uint32_t id_pos = instr_desc(p.bf16, 0, BN), id_neg = instr_desc(p.bf16, 1, BN);
      int64_t g = 0;
      int64_t j = 0;
      for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++j) {
        if (j >= 1 && !mbar_wait_bounded(smem_u32(tempty), (uint32_t)((j - 1) & 1), p.status)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        for (int it = 0; it < k_iters; ++it, ++g) {
          const int buf = (int)(g % NST);
          if (!mbar_wait_bounded(smem_u32(&full[buf]), (uint32_t)((g / NST) & 1), p.status)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const uint32_t st = sbase + buf * S::STAGE;
#pragma unroll
          for (int jj = 0; jj < BK / 16; ++jj) {
            const uint64_t ar = kmajor_desc(st + jj * 32, S::SBO, S::LAYOUT);
            const uint64_t ai = kmajor_desc(st + S::A_BYTES + jj * 32, S::SBO, S::LAYOUT);
            const uint64_t br = kmajor_desc(st + 2 * S::A_BYTES + jj * 32, S::SBO, S::LAYOUT);
            const uint64_t bi = kmajor_desc(st + 2 * S::A_BYTES + S::B_BYTES + jj * 32, S::SBO, S::LAYOUT);
            const uint32_t first = (it == 0 && jj == 0) ? 0u : 1u;
            mma_f16(tmem, ar, br, id_pos, first);
            mma_f16(tmem, ai, bi, id_neg, 1u);
            mma_f16(tmem + BN, ar, bi, id_pos, first);
            mma_f16(tmem + BN, ai, br, id_pos, 1u);
          }
          mma_commit(smem_u32(&empty[buf]));
        }
        if (!ok) break;
        mma_commit(smem_u32(tfull));
      }
      mma_commit(smem_u32(done));
      if (!mbar_wait_bounded(smem_u32(done), 0u, p.status)) ok = false;
    }
  } else {
    // epilogue: thread = one TMEM lane (row), 128 columns of Dr and of Di
    const uint32_t lane_addr = uint32_t((warp & 3) * 32) << 16;
    const int row = (warp & 3) * 32 + lane;
    const int col0 = (warp >> 2) * 128;
    const uint32_t lowmask = (1u << p.runC) - 1u;
    int64_t j = 0;
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x, ++j) {
      if (tid == 0) flag[0] = mbar_wait_bounded(smem_u32(tfull), (uint32_t)(j & 1), p.status) ? 1 : 0;
      group_bar<ET>(1);
      if (flag[0] == 0) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const Inst3 It = map_inst(t >> tile_bits, p.im);
      const uint32_t r = (uint32_t)t & tile_mask;
      const uint32_t on = r & ((1u << p.n_on) - 1u);
      const uint32_t om = p.n_on >= 31 ? 0u : (r >> p.n_on);
      int64_t oC = 0;
      for (int q = 0; q < p.n_om; ++q)
        if ((om >> q) & 1u) oC += int64_t(1) << p.om_C[q];
      for (int q = 0; q < p.n_on; ++q)
        if ((on >> q) & 1u) oC += int64_t(1) << p.on_C[q];
      const int64_t sa = It.a * p.n_slots, sbb = It.b * p.n_slots, sc = It.c * p.n_slots;
      int sh = 0;
      {
        const float a = p.maxabs[sa + p.slotA], bb = p.maxabs[sbb + p.slotB];
        if (a > 0.f && bb > 0.f) {
          int ea, eb;
          frexpf(a, &ea);
          frexpf(bb, &eb);
          sh = ea + eb + p.nK + 1 - 15;
        }
      }
      const float scale = ldexpf(1.f, -sh);
      float mx = 0.f;
      const uint32_t rm = TCm[row];
      T* Cre = reinterpret_cast<T*>(p.C) + It.c * p.strideC + oC;
      // columns 8g..8g+7 of the row are 8 consecutive entries of C: one 16-byte store each
      auto store8 = [&](int col, uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3, uint32_t i0, uint32_t i1,
                        uint32_t i2, uint32_t i3) {
        const uint32_t x = stg_swz(rm ^ TCn[col]);  // C-tile index, low 3 bits 0
        const uint32_t off = hiC[x >> p.runC] + (x & lowmask);
        *reinterpret_cast<uint4*>(Cre + off) = make_uint4(r0, r1, r2, r3);
        *reinterpret_cast<uint4*>(Cre + p.planeC + off) = make_uint4(i0, i1, i2, i3);
      };
      // drain the first 128 - HOLD columns storing as it goes, then the last HOLD columns
      // into registers; TMEM is handed back before those are stored
      constexpr int HOLD = TcwShape<BK>::HOLD;
#pragma unroll 1
      for (int c = 0; c < 128 - HOLD; c += 16) {
        float vr[16], vi[16];
        tmem_ld16(tmem + lane_addr + col0 + c, vr);
        tmem_ld16(tmem + lane_addr + BN + col0 + c, vi);
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          uint32_t a[4], b[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int v = 8 * g + 2 * q;
            a[q] = pack2<T>(vr[v] * scale, vr[v + 1] * scale);
            b[q] = pack2<T>(vi[v] * scale, vi[v + 1] * scale);
            mx = fmaxf(mx, fmaxf(fmaxf(fabsf(vr[v]), fabsf(vr[v + 1])), fmaxf(fabsf(vi[v]), fabsf(vi[v + 1]))));
          }
          store8(col0 + c + 8 * g, a[0], a[1], a[2], a[3], b[0], b[1], b[2], b[3]);
        }
      }
      uint32_t pr[HOLD / 2 + 1], pi[HOLD / 2 + 1];
#pragma unroll
      for (int c = 0; c < HOLD; c += 16) {
        float vr[16], vi[16];
        tmem_ld16(tmem + lane_addr + col0 + 128 - HOLD + c, vr);
        tmem_ld16(tmem + lane_addr + BN + col0 + 128 - HOLD + c, vi);
#pragma unroll
        for (int q = 0; q < 16; q += 2) {
          pr[(c + q) >> 1] = pack2<T>(vr[q] * scale, vr[q + 1] * scale);
          pi[(c + q) >> 1] = pack2<T>(vi[q] * scale, vi[q + 1] * scale);
          mx = fmaxf(mx, fmaxf(fmaxf(fabsf(vr[q]), fabsf(vr[q + 1])), fmaxf(fabsf(vi[q]), fabsf(vi[q + 1]))));
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      group_bar<ET>(1);
      if (tid == 0) mbar_arrive(smem_u32(tempty));
#pragma unroll
      for (int g = 0; g < HOLD / 8; ++g)
        store8(col0 + 128 - HOLD + 8 * g, pr[4 * g], pr[4 * g + 1], pr[4 * g + 2], pr[4 * g + 3], pi[4 * g],
               pi[4 * g + 1], pi[4 * g + 2], pi[4 * g + 3]);
      mx *= scale * (1.f + 0x1p-8f);  // bound on the stored maximum (see tc_epilogue)
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0) red[warp] = mx;
      group_bar<ET>(1);
      if (tid == 0) {
        float m = 0.f;
        for (int w = 0; w < S::EW; ++w) m = fmaxf(m, red[w]);
        atomicMax(reinterpret_cast<unsigned int*>(&p.maxabs[sc + p.slotC]), __float_as_uint(m));
        if (r == 0) p.exps[sc + p.slotC] = p.exps[sa + p.slotA] + p.exps[sbb + p.slotB] + sh;
      }
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(S::TMEM_COLS) : "memory");
}

template <int BK>
size_t tma_wide_smem_bytes_t(int runC) {
  using S = TcwShape<BK>;
  return 1024 + S::PIPE + (size_t(1) << (S::C_BITS - runC)) * 4 + (TC_BM + 256) * 2 + 16 + (2 * S::NST + 3) * 8 + 16 +
         S::EW * 4 + 16 + 64;
}

template <int BN, int BK, int NG, bool DIRECT>
size_t tma_persist_smem_bytes_t(int runC) {
  using S = TcpShape<BN, BK, NG, DIRECT>;
  return 1024 + S::PIPE + NG * S::STG + 2048 * 8 + (size_t(1) << (S::C_BITS - runC)) * 4 + (TC_BM + BN) * 2 + 16 +
         (2 * S::NST + 5) * 8 + 16 + NG * 2 * S::GW * 4 + 16 + 16 + 64;
}

static int sm_count_cached() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
      n = 152;
  }
  return n;
}

template <typename T, int BN, int BK, int NG, bool DIRECT>
cudaError_t launch_tma_persist_ng(const TcParams& p, cudaStream_t s) {
  const size_t smem = tma_persist_smem_bytes_t<BN, BK, NG, DIRECT>(p.runC);
  cudaError_t e = set_smem_once(reinterpret_cast<const void*>(k_tc_tma_persist<T, BN, BK, NG, DIRECT>), smem);
  if (e != cudaSuccess) return e;
  const int64_t tiles = int64_t(p.n_inst) << (p.n_om + p.n_on);
  const unsigned grid = (unsigned)std::min<int64_t>(tiles, sm_count_cached());
  k_tc_tma_persist<T, BN, BK, NG, DIRECT><<<grid, TcpShape<BN, BK, NG, DIRECT>::THREADS, smem, s>>>(p);
  return cudaGetLastError();
}

template <typename T, int BK>
cudaError_t launch_tma_wide(const TcParams& p, cudaStream_t s) {
  const size_t smem = tma_wide_smem_bytes_t<BK>(p.runC);
  cudaError_t e = set_smem_once(reinterpret_cast<const void*>(k_tc_tma_wide<T, BK>), smem);
  if (e != cudaSuccess) return e;
  const int64_t tiles = int64_t(p.n_inst) << (p.n_om + p.n_on);
  const unsigned grid = (unsigned)std::min<int64_t>(tiles, sm_count_cached());
  k_tc_tma_wide<T, BK><<<grid, TcwShape<BK>::THREADS, smem, s>>>(p);
  return cudaGetLastError();
}

// Two epilogue groups for short K loops (output-bound tiles): up to four K tiles with the
// direct epilogue, up to two when staged (the staging buffers shorten the ring); one group
// otherwise.  Direct variants reserve no staging buffer.
template <typename T, int BN, int BK>
cudaError_t launch_tma_persist_t(const TcParams& p, cudaStream_t s) {
  if (p.direct) {
    if (p.n_ok <= 2) return launch_tma_persist_ng<T, BN, BK, 2, true>(p, s);
    return launch_tma_persist_ng<T, BN, BK, 1, true>(p, s);
  }
  if (p.n_ok <= 1) return launch_tma_persist_ng<T, BN, BK, 2, false>(p, s);
  return launch_tma_persist_ng<T, BN, BK, 1, false>(p, s);
}

template <int BN, int BK, int NST>
size_t tma_smem_bytes_t(int runC) {
  using S = TcShape<BN, BK, NST>;
  return 1024 + S::REGION + (size_t(1) << (S::C_BITS - runC)) * 4 + (TC_BM + BN) * 2 + 16 + (2 * NST + 1) * 8 + 16 +
         32 * 4 + 64;
}

template <typename T, int BN, int BK, int NST>
cudaError_t launch_tma_t(const TcParams& p, dim3 grid, cudaStream_t s) {
  const size_t smem = tma_smem_bytes_t<BN, BK, NST>(p.runC);
  cudaError_t e = set_smem_once(reinterpret_cast<const void*>(k_tc_tma<T, BN, BK, NST>), smem);
  if (e != cudaSuccess) return e;
  k_tc_tma<T, BN, BK, NST><<<grid, TC_THREADS, smem, s>>>(p);
  return cudaGetLastError();
}

template <typename T, int BN, int BK>
cudaError_t launch_tma_st(const TcParams& p, dim3 grid, cudaStream_t s) {
  // 256-wide tiles take all 512 TMEM columns: one CTA per SM, always the deep pipeline
  if (p.stages == 3 && BN < 256) return launch_tma_t<T, BN, BK, 3>(p, grid, s);
  return launch_tma_t<T, BN, BK, tc_deep_stages<BN, BK>()>(p, grid, s);
}

template <typename T>
cudaError_t launch_tma_bn_bk(const TcParams& p, dim3 grid, cudaStream_t s) {
  if (p.persistent && p.splitk == 1 && p.n_inst >= 1) {
    // 256-wide tiles: only with the direct epilogue (no room for a staging buffer)
    if (p.bn == 256 && p.direct && p.runC >= 3 && p.bk == 32) return launch_tma_wide<T, 32>(p, s);
    if (p.bn == 256 && p.direct && p.runC >= 3 && p.bk == 16) return launch_tma_wide<T, 16>(p, s);
    if (p.bn == 128 && p.bk == 32) return launch_tma_persist_t<T, 128, 32>(p, s);
    if (p.bn == 128 && p.bk == 16) return launch_tma_persist_t<T, 128, 16>(p, s);
    if (p.bn == 64 && p.bk == 32) return launch_tma_persist_t<T, 64, 32>(p, s);
    if (p.bn == 64 && p.bk == 16) return launch_tma_persist_t<T, 64, 16>(p, s);
  }
  if (p.bn == 32) {
    if (p.bk == 32) return launch_tma_st<T, 32, 32>(p, grid, s);
    if (p.bk == 16) return launch_tma_st<T, 32, 16>(p, grid, s);
  } else if (p.bn == 256) {
    if (p.bk == 32) return launch_tma_st<T, 256, 32>(p, grid, s);
    if (p.bk == 16) return launch_tma_st<T, 256, 16>(p, grid, s);
  } else if (p.bn == 128) {
    if (p.bk == 32) return launch_tma_st<T, 128, 32>(p, grid, s);
    if (p.bk == 16) return launch_tma_st<T, 128, 16>(p, grid, s);
  } else if (p.bn == 64) {
    if (p.bk == 32) return launch_tma_st<T, 64, 32>(p, grid, s);
    if (p.bk == 16) return launch_tma_st<T, 64, 16>(p, grid, s);
  }
  return cudaErrorInvalidValue;
}

template <int BN>
size_t tf32_smem_bytes(int runC) {
  using S = Tf32Shape<BN>;
  return 1024 + S::REGION + (size_t(1) << (S::C_BITS - runC)) * 4 + (TC_BM + BN) * 2 + 16 + (3 * S::NST + 5) * 8 + 16 +
         16 * 4 + 64;
}

template <int BN>
cudaError_t launch_tf32_bn(const TcParams& p, dim3 grid, cudaStream_t s) {
  const size_t smem = tf32_smem_bytes<BN>(p.runC);
  cudaError_t e = set_smem_once(reinterpret_cast<const void*>(k_tc_tma_tf32<BN>), smem);
  if (e != cudaSuccess) return e;
  k_tc_tma_tf32<BN><<<grid, TF32_THREADS, smem, s>>>(p);
  return cudaGetLastError();
}

// complex64: the 3xTF32 kernel (one CTA per tile; widths 32, 64 and 128)
cudaError_t launch_tc_tma_tf32(const TcParams& p, dim3 grid, cudaStream_t s) {
  if (p.persistent) return cudaErrorInvalidValue;
  if (p.bn == 128) return launch_tf32_bn<128>(p, grid, s);
  if (p.bn == 64) return launch_tf32_bn<64>(p, grid, s);
  if (p.bn == 32) return launch_tf32_bn<32>(p, grid, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_tc_tma(int precision, const TcParams& p, dim3 grid, cudaStream_t s) {
  if (precision == 0) return launch_tc_tma_tf32(p, grid, s);
  if (precision == 1) return launch_tma_bn_bk<__half>(p, grid, s);
  if (precision == 2) return launch_tma_bn_bk<__nv_bfloat16>(p, grid, s);
  return cudaErrorInvalidValue;
}

template <int BN, int BK, int NST>
size_t tc_smem_bytes_t(int runC) {
  using S = TcShape<BN, BK, NST>;
  return 1024 + S::REGION + (TC_BM + BN) * 4 + (size_t(1) << (S::C_BITS - runC)) * 4 + (TC_BM + BN) * 2 + 16 +
         (2 * NST + 1) * 8 + 16 + 32 * 4 + 64;
}

template <typename T, int BN, int BK, int NST>
cudaError_t launch_tc_t(const TcParams& p, dim3 grid, cudaStream_t s) {
  const size_t smem = tc_smem_bytes_t<BN, BK, NST>(p.runC);
  cudaError_t e = set_smem_once(reinterpret_cast<const void*>(k_tc_gemm<T, BN, BK, NST>), smem);
  if (e != cudaSuccess) return e;
  k_tc_gemm<T, BN, BK, NST><<<grid, TC_THREADS, smem, s>>>(p);
  return cudaGetLastError();
}

// p.stages: 3 (short K loops: two CTAs share an SM) or 0 (deepest pipeline)
template <typename T, int BN, int BK>
cudaError_t launch_tc_st(const TcParams& p, dim3 grid, cudaStream_t s) {
  if (p.stages == 3) return launch_tc_t<T, BN, BK, 3>(p, grid, s);
  return launch_tc_t<T, BN, BK, tc_deep_stages<BN, BK>()>(p, grid, s);
}

template <typename T>
cudaError_t launch_tc_bn_bk(const TcParams& p, dim3 grid, cudaStream_t s) {
  if (p.bn == 128) {
    if (p.bk == 32) return launch_tc_st<T, 128, 32>(p, grid, s);
    if (p.bk == 16) return launch_tc_st<T, 128, 16>(p, grid, s);
  } else if (p.bn == 64) {
    if (p.bk == 32) return launch_tc_st<T, 64, 32>(p, grid, s);
    if (p.bk == 16) return launch_tc_st<T, 64, 16>(p, grid, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_tc_gemm(int precision, const TcParams& p, dim3 grid, cudaStream_t s) {
  if (precision == 1) return launch_tc_bn_bk<__half>(p, grid, s);
  if (precision == 2) return launch_tc_bn_bk<__nv_bfloat16>(p, grid, s);
  return cudaErrorInvalidValue;
}

}  // namespace tnc
