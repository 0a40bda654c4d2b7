// CUDA kernels of the contraction path (sm_103a).
//
//  k_generic      -- one pairwise contraction C = A * B (Sec. II-A: an M x K x N complex
//                    GEMM over the common indices).  Each CTA owns a tile that is a set of
//                    indices of each operand; because indices are binary, a tile is a
//                    sub-tensor whose lowest positions are contiguous in memory, so tiles
//                    are loaded in the operand's own order with vector loads and the
//                    permutation happens in the shared-memory indexing (the permutation
//                    folded into the kernel, Sec. V-A).  FP32 complex multiply-adds.
//                    With splitk > 1 the CTAs split the outer common indices and write
//                    FP32 partial sums (split-common TTGT for GEPDOT shapes, Sec. V-B).
//  k_splitk_reduce -- sums the partials of a split step in a fixed order (blocked
//                    summation, Eq. 3), scales and stores.
//  k_leaf_gather  -- per instance (bitstring, slice): fixes sliced and closed-output legs
//                    of every leaf (Sec. III-A slicing), converts and scales.
//  k_root_accum   -- adds the root tensors of a wave into the FP64 amplitude accumulator
//                    (sum over subtasks, Sec. III-A).
//  k_maxabs       -- max |re|,|im| of a planar tensor (scale of tnc_contract's inputs).
//
// Scaling: every tensor carries an int32 exponent E (value = stored * 2^E) and the max
// |re|,|im| of its stored values.  A producer scales its FP32 results by the exact power
// of two that brings the bound 2^(nK+1) * max|A| * max|B| below 2^15, so fp16 storage
// can neither overflow nor flush ordinary values to zero.
#include <map>
#include <mutex>

#include <cooperative_groups.h>

#include "device.cuh"

namespace tnc {

// The attribute belongs to the kernel on one device, so the cache is keyed by both: a
// call on another device sets it there too.
cudaError_t set_smem_once(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> done;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_pair(dev, kernel);
  auto it = done.find(key);
  if (it != done.end() && it->second >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done[key] = bytes;
  return e;
}

template <typename T, int V>
struct alignas(sizeof(T) * V) Vec {
  T v[V];
};

__device__ __forceinline__ uint32_t deposit_hi(uint32_t h, uint32_t mask, int run) {
  uint32_t m = mask;
  for (int i = 0; i < run; ++i) m &= m - 1;
  uint32_t r = 0;
  while (m) {
    uint32_t low = m & (~m + 1u);
    if (h & 1u) r |= low;
    h >>= 1;
    m &= m - 1;
  }
  return r;
}

__device__ __forceinline__ uint32_t scatter_bits(uint32_t x, const int8_t* pos, int n) {
  uint32_t r = 0;
  for (int j = 0; j < n; ++j) r |= ((x >> j) & 1u) << pos[j];
  return r;
}

__device__ __forceinline__ void atomic_max_nonneg(float* addr, float v) {
  atomicMax(reinterpret_cast<unsigned int*>(addr), __float_as_uint(v));
}

// Exponent shift for a product of tensors with stored max a, b over 2^nK terms.
__device__ __forceinline__ int product_shift(float a, float b, int nK) {
  if (!(a > 0.f) || !(b > 0.f)) return 0;
  int ea, eb;
  frexpf(a, &ea);  // a < 2^ea
  frexpf(b, &eb);
  return ea + eb + nK + 1 - 15;
}

// Shared-memory swizzle of a float2 operand tile: the low four index bits (one 128-byte
// line holds 16 float2) are XORed with index bits 4..7 and 8..11.  A warp reading one
// entry per tile row hits distinct lines' banks even when the rows are a power of two
// apart (contiguous K, strided M).  The map is linear over GF(2): the swizzled index of
// a sum of disjoint bit sets is the XOR of their swizzled parts, so offset tables can be
// stored swizzled and combined with XOR.
__device__ __forceinline__ uint32_t sw16(uint32_t i) { return i ^ (((i >> 4) ^ (i >> 8)) & 15u); }

// Complex multiply-adds of a micro-tile in FP32: re += a.re b.re then re += (-a.im) b.im,
// im += a.re b.im then im += a.im b.re (the order every SIMT kernel here keeps).
template <int RM, int RN>
__device__ __forceinline__ void cmac_tile(float2 (&acc)[RM][RN], const float2 (&a)[RM], const float2 (&b)[RN]) {
#pragma unroll
  for (int i = 0; i < RM; ++i)
#pragma unroll
    for (int j = 0; j < RN; ++j) {
      acc[i][j].x = fmaf(a[i].x, b[j].x, acc[i][j].x);
      acc[i][j].x = fmaf(-a[i].y, b[j].y, acc[i][j].x);
      acc[i][j].y = fmaf(a[i].x, b[j].y, acc[i][j].y);
      acc[i][j].y = fmaf(a[i].y, b[j].x, acc[i][j].y);
    }
}

template <typename T>
struct MixFma;
template <>
struct MixFma<__half> {
  static __device__ __forceinline__ float fma(uint16_t a, uint16_t b, float c) {
    asm("fma.rn.f32.f16 %0, %1, %2, %0;" : "+f"(c) : "h"(a), "h"(b));
    return c;
  }
};
template <>
struct MixFma<__nv_bfloat16> {
  static __device__ __forceinline__ float fma(uint16_t a, uint16_t b, float c) {
    asm("fma.rn.f32.bf16 %0, %1, %2, %0;" : "+f"(c) : "h"(a), "h"(b));
    return c;
  }
};
__device__ __forceinline__ uint16_t word16(const uint2& w, int v) {
  const uint32_t x = v < 2 ? w.x : w.y;
  return (uint16_t)((v & 1) ? (x >> 16) : (x & 0xFFFFu));
}
template <typename T, int RM, int RN>
__device__ __forceinline__ void cmac_tile16(float2 (&acc)[RM][RN], const uint2 (&ar)[RM], const uint2 (&ai)[RM],
                                            const uint2 (&br)[RN], const uint2 (&bi)[RN], int v) {
#pragma unroll
  for (int i = 0; i < RM; ++i) {
    const uint16_t xr = word16(ar[i], v), xi = word16(ai[i], v), nxi = xi ^ 0x8000u;
#pragma unroll
    for (int j = 0; j < RN; ++j) {
      const uint16_t yr = word16(br[j], v), yi = word16(bi[j], v);
      acc[i][j].x = MixFma<T>::fma(xr, yr, acc[i][j].x);
      acc[i][j].x = MixFma<T>::fma(nxi, yi, acc[i][j].x);
      acc[i][j].y = MixFma<T>::fma(xr, yi, acc[i][j].y);
      acc[i][j].y = MixFma<T>::fma(xi, yr, acc[i][j].y);
    }
  }
}

// A vector of V entries read at L2 (ld.global.cg): data written by other CTAs earlier in the
// same launch (the persistent steps kernel, after a grid barrier) is never served stale from
// the non-coherent or L1 paths.
template <typename T, int V>
__device__ __forceinline__ Vec<T, V> ld_cg(const T* p) {
  constexpr int B = int(sizeof(T)) * V;
  Vec<T, V> r;
  if constexpr (B == 16) {
    const uint4 x = __ldcg(reinterpret_cast<const uint4*>(p));
    memcpy(&r, &x, 16);
  } else if constexpr (B == 8) {
    const uint2 x = __ldcg(reinterpret_cast<const uint2*>(p));
    memcpy(&r, &x, 8);
  } else if constexpr (B == 4) {
    const unsigned int x = __ldcg(reinterpret_cast<const unsigned int*>(p));
    memcpy(&r, &x, 4);
  } else {
    const unsigned short x = __ldcg(reinterpret_cast<const unsigned short*>(p));
    memcpy(&r, &x, 2);
  }
  return r;
}

template <typename T, int V, bool SW, bool COH = false>
__device__ __forceinline__ void load_tile_v(const T* __restrict__ re, const T* __restrict__ im, int bits, int run,
                                            const uint32_t* __restrict__ hi, float2* __restrict__ dst) {
  const int n = 1 << bits;
  const uint32_t lowmask = (1u << run) - 1u;
  for (int t = threadIdx.x * V; t < n; t += kThreads * V) {
    const uint32_t off = hi[t >> run] + (uint32_t(t) & lowmask);
    Vec<T, V> r, i;
    if constexpr (COH) {
      r = ld_cg<T, V>(re + off);
      i = ld_cg<T, V>(im + off);
    } else {
      r = *reinterpret_cast<const Vec<T, V>*>(re + off);
      i = *reinterpret_cast<const Vec<T, V>*>(im + off);
    }
#pragma unroll
    for (int v = 0; v < V; ++v)
      dst[SW ? sw16(uint32_t(t + v)) : uint32_t(t + v)] = make_float2(Conv<T>::to_f(r.v[v]), Conv<T>::to_f(i.v[v]));
  }
}

template <typename T, bool SW = false, bool COH = false>
__device__ __forceinline__ void load_tile(const T* re, const T* im, int bits, int run, const uint32_t* hi, float2* dst) {
  constexpr int VMAX = 16 / sizeof(T);
  const int v = min(1 << run, VMAX);
  if (v >= 8) load_tile_v<T, (VMAX >= 8 ? 8 : 1), SW, COH>(re, im, bits, run, hi, dst);
  else if (v == 4) load_tile_v<T, 4, SW, COH>(re, im, bits, run, hi, dst);
  else if (v == 2) load_tile_v<T, 2, SW, COH>(re, im, bits, run, hi, dst);
  else load_tile_v<T, 1, SW, COH>(re, im, bits, run, hi, dst);
}

template <typename T, int V>
__device__ __forceinline__ float store_tile_v(T* __restrict__ re, T* __restrict__ im, int bits, int run,
                                              const uint32_t* __restrict__ hi, const float2* __restrict__ src, float scale) {
  const int n = 1 << bits;
  const uint32_t lowmask = (1u << run) - 1u;
  float mx = 0.f;
  for (int t = threadIdx.x * V; t < n; t += kThreads * V) {
    const uint32_t off = hi[t >> run] + (uint32_t(t) & lowmask);
    Vec<T, V> r, i;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const float2 x = src[t + v];
      r.v[v] = Conv<T>::from_f(x.x * scale);
      i.v[v] = Conv<T>::from_f(x.y * scale);
      mx = fmaxf(mx, fmaxf(fabsf(Conv<T>::to_f(r.v[v])), fabsf(Conv<T>::to_f(i.v[v]))));
    }
    *reinterpret_cast<Vec<T, V>*>(re + off) = r;
    *reinterpret_cast<Vec<T, V>*>(im + off) = i;
  }
  return mx;
}

template <typename T>
__device__ __forceinline__ float store_tile(T* re, T* im, int bits, int run, const uint32_t* hi, const float2* src, float scale) {
  constexpr int VMAX = 16 / sizeof(T);
  const int v = min(1 << run, VMAX);
  if (v >= 8) return store_tile_v<T, (VMAX >= 8 ? 8 : 1)>(re, im, bits, run, hi, src, scale);
  if (v == 4) return store_tile_v<T, 4>(re, im, bits, run, hi, src, scale);
  if (v == 2) return store_tile_v<T, 2>(re, im, bits, run, hi, src, scale);
  return store_tile_v<T, 1>(re, im, bits, run, hi, src, scale);
}

__device__ __forceinline__ float block_max(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = l < (int)(blockDim.x >> 5) ? red[l] : 0.f;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  return v;  // valid in thread 0
}

// After the K loop of k_generic / k_stream: the K groups' sums in a fixed order into the
// C-native staging tile R, then either FP32 split-K partials or the scaled, converted tile.
// Returns this thread's largest stored magnitude (0 for partials); generic_publish takes the
// CTA's maximum once, after all of its tiles.
template <typename T, int RM, int RN>
__device__ __forceinline__ float generic_finish(const GenParams& p, const Inst3 I, const float2 (&acc)[RM][RN],
                                                bool active, int grp, int mi, int ni, int TM, int TN,
                                                const uint16_t* TCm, const uint16_t* TCn, const uint32_t* hiC,
                                                float2* R, int64_t oC, float scale, uint32_t by, uint32_t bz) {
  const int tid = threadIdx.x;
  // K groups in a fixed order
  const int O = 1 << (p.mt + p.nt);
  if (active) {
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
      for (int j = 0; j < RN; ++j) R[grp * O + TCm[mi + i * TM] + TCn[ni + j * TN]] = acc[i][j];
  }
  __syncthreads();
  if (p.kgroups >= 8) {
    // pairwise tree over the groups (group g adds group g + h, h = G/2, G/4, ..., 1): the
    // same order on every run, log2(G) barriers instead of G dependent adds per output
    for (int h = p.kgroups >> 1; h > 0; h >>= 1) {
      for (int x = tid; x < h * O; x += kThreads) {
        const float2 v = R[h * O + x];
        R[x].x += v.x;
        R[x].y += v.y;
      }
      __syncthreads();
    }
  } else if (p.kgroups > 1) {
    for (int o = tid; o < O; o += kThreads) {
      float2 s = R[o];
      for (int g = 1; g < p.kgroups; ++g) {
        const float2 v = R[g * O + o];
        s.x += v.x;
        s.y += v.y;
      }
      R[o] = s;
    }
    __syncthreads();
  }
  if (p.splitk > 1) {
    // FP32 partial sums, indexed by C's flat index
    float2* part = p.partials + (int64_t(bz) * p.splitk + by) * p.planeC + oC;
    const uint32_t lowmask = (1u << p.runC) - 1u;
    for (int t = tid; t < O; t += kThreads) part[hiC[t >> p.runC] + (uint32_t(t) & lowmask)] = R[t];
    return 0.f;
  }
  // scale, convert, store
  T* Cre = reinterpret_cast<T*>(p.C) + I.c * p.strideC + oC;
  return store_tile<T>(Cre, Cre + p.planeC, p.mt + p.nt, p.runC, hiC, R, scale);
}

// The output scale of a launch's instance: 2^-sh with sh from the operands' stored maxima.
__device__ __forceinline__ int generic_shift(const GenParams& p, const Inst3 I) {
  return product_shift(p.maxabs[I.a * p.n_slots + p.slotA], p.maxabs[I.b * p.n_slots + p.slotB], p.nK);
}

// The CTA's largest stored magnitude into C's maximum, and (the CTA of tile 0) C's exponent.
__device__ __forceinline__ void generic_publish(const GenParams& p, const Inst3 I, float mx, float* red, int sh,
                                                bool first) {
  const float bm = block_max(mx, red);
  if (threadIdx.x == 0) {
    const int64_t sa = I.a * p.n_slots, sbb = I.b * p.n_slots, sc = I.c * p.n_slots;
    atomic_max_nonneg(&p.maxabs[sc + p.slotC], bm);
    if (first) p.exps[sc + p.slotC] = p.exps[sa + p.slotA] + p.exps[sbb + p.slotB] + sh;
  }
}

// One CTA of the tiled SIMT contraction: split column by, instance column bz, tiles bx,
// bx + gx, ... of the outer tile grid (k_generic, and each unit of k_steps).
template <typename T, int RM, int RN, bool COH = false>
__device__ __forceinline__ void generic_cta(const GenParams& p, unsigned char* smem, uint32_t bx, uint32_t gx,
                                            uint32_t by, uint32_t bz) {
  float2* As = reinterpret_cast<float2*>(smem);
  float2* Bs = As + (1 << (p.mt + p.kt));
  float2* R = As;  // reduction / staging after the K loop
  uint32_t* hiA = reinterpret_cast<uint32_t*>(smem + p.smem_tables);
  uint32_t* hiB = hiA + (1 << (p.mt + p.kt - p.runA));
  uint32_t* hiC = hiB + (1 << (p.kt + p.nt - p.runB));
  uint16_t* TAm = reinterpret_cast<uint16_t*>(hiC + (1 << (p.mt + p.nt - p.runC)));
  uint16_t* TAk = TAm + (1 << p.mt);
  uint16_t* TBk = TAk + (1 << p.kt);
  uint16_t* TBn = TBk + (1 << p.kt);
  uint16_t* TCm = TBn + (1 << p.nt);
  uint16_t* TCn = TCm + (1 << p.mt);
  float* red = reinterpret_cast<float*>(TCn + (1 << p.nt) + 2);  // 4-byte aligned (+2 pads)

  const int tid = threadIdx.x;
  const Inst3 I = map_inst(bz, p.im);
  // index tables (built once; the CTA then strides over the outer tiles)
  {
    const int nhA = 1 << (p.mt + p.kt - p.runA), nhB = 1 << (p.kt + p.nt - p.runB), nhC = 1 << (p.mt + p.nt - p.runC);
    for (int h = tid; h < nhA; h += kThreads) hiA[h] = deposit_hi(h, p.maskA, p.runA);
    for (int h = tid; h < nhB; h += kThreads) hiB[h] = deposit_hi(h, p.maskB, p.runB);
    for (int h = tid; h < nhC; h += kThreads) hiC[h] = deposit_hi(h, p.maskC, p.runC);
    // operand tables are stored swizzled (sw16), the C staging tables plain
    for (int x = tid; x < (1 << p.mt); x += kThreads) {
      TAm[x] = (uint16_t)sw16(scatter_bits(x, p.pAm, p.mt));
      TCm[x] = (uint16_t)scatter_bits(x, p.pCm, p.mt);
    }
    for (int x = tid; x < (1 << p.kt); x += kThreads) {
      TAk[x] = (uint16_t)sw16(scatter_bits(x, p.pAk, p.kt));
      TBk[x] = (uint16_t)sw16(scatter_bits(x, p.pBk, p.kt));
    }
    for (int x = tid; x < (1 << p.nt); x += kThreads) {
      TBn[x] = (uint16_t)sw16(scatter_bits(x, p.pBn, p.nt));
      TCn[x] = (uint16_t)scatter_bits(x, p.pCn, p.nt);
    }
  }
  __syncthreads();

  // thread -> micro-tile
  const int TM = (1 << p.mt) / RM, TN = (1 << p.nt) / RN;
  const int TPO = TM * TN;
  const int grp = tid / TPO, r = tid % TPO;
  const bool active = grp < p.kgroups;
  const int mi = r % TM, ni = r / TM;
  int am[RM], bn[RN];
#pragma unroll
  for (int i = 0; i < RM; ++i) am[i] = active ? TAm[mi + i * TM] : 0;
#pragma unroll
  for (int j = 0; j < RN; ++j) bn[j] = active ? TBn[ni + j * TN] : 0;
  const int64_t KO = int64_t(1) << p.n_ok;
  // CTA y of the split takes the outer K steps [y KO / splitk, (y + 1) KO / splitk)
  const int64_t k0 = int64_t(by) * KO / p.splitk;
  const int64_t per = (int64_t(by) + 1) * KO / p.splitk - k0;
  const int nk = 1 << p.kt;
  const uint32_t n_tiles = 1u << (p.n_om + p.n_on);
  // one output scale per instance; the maximum is published once per CTA
  const int sh = p.splitk == 1 ? generic_shift(p, I) : 0;
  const float scale = ldexpf(1.f, -sh);
  float mx = 0.f;
  for (uint32_t tile = bx; tile < n_tiles; tile += gx) {
    // outer coordinates of this tile
    const uint32_t om = tile & ((1u << p.n_om) - 1u);
    const uint32_t on = p.n_om >= 32 ? 0u : (tile >> p.n_om);
    int64_t oA = 0, oB = 0, oC = 0;
    for (uint32_t m = om; m; m &= m - 1u) {  // the set bits only
      const int j = __ffs(m) - 1;
      oA += int64_t(1) << p.om_A[j];
      oC += int64_t(1) << p.om_C[j];
    }
    for (uint32_t m = on; m; m &= m - 1u) {
      const int j = __ffs(m) - 1;
      oB += int64_t(1) << p.on_B[j];
      oC += int64_t(1) << p.on_C[j];
    }
    float2 acc[RM][RN];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
      for (int j = 0; j < RN; ++j) acc[i][j] = make_float2(0.f, 0.f);

    const T* Abase = reinterpret_cast<const T*>(p.A) + I.a * p.strideA + oA;
    const T* Bbase = reinterpret_cast<const T*>(p.B) + I.b * p.strideB + oB;
    for (int64_t ok = k0; ok < k0 + per; ++ok) {
      int64_t okA = 0, okB = 0;
      for (int j = 0; j < p.n_ok; ++j)
        if ((ok >> j) & 1) {
          okA += int64_t(1) << p.ok_A[j];
          okB += int64_t(1) << p.ok_B[j];
        }
      load_tile<T, true, COH>(Abase + okA, Abase + okA + p.planeA, p.mt + p.kt, p.runA, hiA, As);
      load_tile<T, true, COH>(Bbase + okB, Bbase + okB + p.planeB, p.kt + p.nt, p.runB, hiB, Bs);
      __syncthreads();
      if (active) {
        // K group grp takes k = grp, grp + kgroups, ..., or (kvb > 0) chunks c = grp,
        // grp + kgroups, ... of 2^kvb consecutive k
        auto mac = [&](int k) {
          const int ka = TAk[k], kb = TBk[k];
          float2 a[RM], b[RN];
#pragma unroll
          for (int i = 0; i < RM; ++i) a[i] = As[am[i] ^ ka];
#pragma unroll
          for (int j = 0; j < RN; ++j) b[j] = Bs[kb ^ bn[j]];
          cmac_tile<RM, RN>(acc, a, b);
        };
        if (p.kvb == 0) {
          for (int k = grp; k < nk; k += p.kgroups) mac(k);
        } else {
          for (int c = grp; c < (nk >> p.kvb); c += p.kgroups)
            for (int v = 0; v < (1 << p.kvb); ++v) mac((c << p.kvb) | v);
        }
      }
      __syncthreads();
    }
    mx = fmaxf(mx, generic_finish<T, RM, RN>(p, I, acc, active, grp, mi, ni, TM, TN, TCm, TCn, hiC, R, oC, scale, by, bz));
    __syncthreads();  // R (the staging tile) is the next tile's A tile
  }
  if (p.splitk == 1) generic_publish(p, I, mx, red, sh, bx == 0);
}

template <typename T, int RM, int RN>
__global__ void __launch_bounds__(kThreads) k_generic(const GenParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  generic_cta<T, RM, RN>(p, smem, blockIdx.x, gridDim.x, blockIdx.y, blockIdx.z);
}

// Streaming variant of k_generic for GEPDOT-shaped steps (few outputs, a long K loop;
// Sec. V-B).  Each K step's operand tiles are copied raw (16-bit or FP32 planes, in 16-byte
// cp.async chunks) into a kStreamStages-deep shared-memory ring, so the next steps' loads are
// in flight while one is multiplied; entries are converted to FP32 as they are read.  Every
// thread visits the same k values in the same order as in k_generic, so the two kernels give
// identical results.  Needs runs of at least 16 bytes at the low positions of A and B (every
// chunk is contiguous in memory).  Tiles are swizzled by sw_chunk, which moves whole chunks.
__device__ __forceinline__ void cpa16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Entry-index swizzle of a raw tile: the chunk-within-128-byte-line bits are XORed with the
// two groups of line-index bits above them, so the rows a warp reads at once (a power of
// two apart) fall on different banks.  Linear over GF(2) and leaves the low (within-chunk)
// bits alone: offset tables are stored swizzled and combined with XOR, and a 16-byte chunk
// stays one contiguous chunk.
template <typename T>
__device__ __forceinline__ uint32_t sw_chunk(uint32_t i) {
  constexpr int C = sizeof(T) == 2 ? 3 : 2;  // log2 entries per 16-byte chunk
  constexpr int L = C + 3;                   // log2 entries per 128-byte line
  return i ^ ((((i >> L) ^ (i >> (L + 3))) & 7u) << C);
}

// Issue the cp.async copies of one raw planar tile (2^bits entries, runs of 2^run).
template <typename T>
__device__ __forceinline__ void stream_copy(const T* re, const T* im, int bits, int run, const uint32_t* hi,
                                            uint32_t dst_re, uint32_t dst_im) {
  constexpr int VE = 16 / sizeof(T);
  const int n = 1 << bits;
  const uint32_t lowmask = (1u << run) - 1u;
  for (int t = threadIdx.x * VE; t < n; t += kThreads * VE) {
    const uint32_t off = hi[t >> run] + (uint32_t(t) & lowmask);
    const uint32_t d = sw_chunk<T>(uint32_t(t)) * uint32_t(sizeof(T));
    cpa16(dst_re + d, re + off);
    cpa16(dst_im + d, im + off);
  }
}

template <typename T, int RM, int RN>
__global__ void __launch_bounds__(kThreads, 2) k_stream(const GenParams p) {
  constexpr int NS = kStreamStages;
  extern __shared__ __align__(16) unsigned char smem[];
  const int nA = 1 << (p.mt + p.kt), nB = 1 << (p.kt + p.nt);
  const uint32_t stage_bytes = uint32_t(2 * (nA + nB)) * uint32_t(sizeof(T));
  float2* R = reinterpret_cast<float2*>(smem);  // reduction / staging after the K loop
  uint32_t* hiA = reinterpret_cast<uint32_t*>(smem + p.smem_tables);
  uint32_t* hiB = hiA + (1 << (p.mt + p.kt - p.runA));
  uint32_t* hiC = hiB + (1 << (p.kt + p.nt - p.runB));
  uint16_t* TAm = reinterpret_cast<uint16_t*>(hiC + (1 << (p.mt + p.nt - p.runC)));
  uint16_t* TAk = TAm + (1 << p.mt);
  uint16_t* TBk = TAk + (1 << p.kt);
  uint16_t* TBn = TBk + (1 << p.kt);
  uint16_t* TCm = TBn + (1 << p.nt);
  uint16_t* TCn = TCm + (1 << p.mt);
  float* red = reinterpret_cast<float*>(TCn + (1 << p.nt) + 2);

  const int tid = threadIdx.x;
  const Inst3 I = map_inst(blockIdx.z, p.im);
  const uint32_t om = blockIdx.x & ((1u << p.n_om) - 1u);
  const uint32_t on = p.n_om >= 32 ? 0u : (blockIdx.x >> p.n_om);
  int64_t oA = 0, oB = 0, oC = 0;
  for (int j = 0; j < p.n_om; ++j)
    if ((om >> j) & 1u) {
      oA += int64_t(1) << p.om_A[j];
      oC += int64_t(1) << p.om_C[j];
    }
  for (int j = 0; j < p.n_on; ++j)
    if ((on >> j) & 1u) {
      oB += int64_t(1) << p.on_B[j];
      oC += int64_t(1) << p.on_C[j];
    }
  {
    const int nhA = 1 << (p.mt + p.kt - p.runA), nhB = 1 << (p.kt + p.nt - p.runB), nhC = 1 << (p.mt + p.nt - p.runC);
    for (int h = tid; h < nhA; h += kThreads) hiA[h] = deposit_hi(h, p.maskA, p.runA);
    for (int h = tid; h < nhB; h += kThreads) hiB[h] = deposit_hi(h, p.maskB, p.runB);
    for (int h = tid; h < nhC; h += kThreads) hiC[h] = deposit_hi(h, p.maskC, p.runC);
    // operand tables are stored swizzled (sw_chunk), the C staging tables plain
    for (int x = tid; x < (1 << p.mt); x += kThreads) {
      TAm[x] = (uint16_t)sw_chunk<T>(scatter_bits(x, p.pAm, p.mt));
      TCm[x] = (uint16_t)scatter_bits(x, p.pCm, p.mt);
    }
    for (int x = tid; x < (1 << p.kt); x += kThreads) {
      TAk[x] = (uint16_t)sw_chunk<T>(scatter_bits(x, p.pAk, p.kt));
      TBk[x] = (uint16_t)sw_chunk<T>(scatter_bits(x, p.pBk, p.kt));
    }
    for (int x = tid; x < (1 << p.nt); x += kThreads) {
      TBn[x] = (uint16_t)sw_chunk<T>(scatter_bits(x, p.pBn, p.nt));
      TCn[x] = (uint16_t)scatter_bits(x, p.pCn, p.nt);
    }
  }
  __syncthreads();

  const int TM = (1 << p.mt) / RM, TN = (1 << p.nt) / RN;
  const int TPO = TM * TN;
  const int grp = tid / TPO, r = tid % TPO;
  const bool active = grp < p.kgroups;
  const int mi = r % TM, ni = r / TM;
  int am[RM], bn[RN];
#pragma unroll
  for (int i = 0; i < RM; ++i) am[i] = active ? TAm[mi + i * TM] : 0;
#pragma unroll
  for (int j = 0; j < RN; ++j) bn[j] = active ? TBn[ni + j * TN] : 0;
  float2 acc[RM][RN];
#pragma unroll
  for (int i = 0; i < RM; ++i)
#pragma unroll
    for (int j = 0; j < RN; ++j) acc[i][j] = make_float2(0.f, 0.f);

  const T* Abase = reinterpret_cast<const T*>(p.A) + I.a * p.strideA + oA;
  const T* Bbase = reinterpret_cast<const T*>(p.B) + I.b * p.strideB + oB;
  const int64_t KO = int64_t(1) << p.n_ok;
  // CTA y of the split takes the outer K steps [y KO / splitk, (y + 1) KO / splitk)
  const int64_t k0 = int64_t(blockIdx.y) * KO / p.splitk;
  const int64_t per = (int64_t(blockIdx.y) + 1) * KO / p.splitk - k0;
  const int nk = 1 << p.kt;
  const uint32_t sbase = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  // operand offsets of outer K step `nok` (the next one to copy), advanced one step at a time
  // by the bits that flip: the trailing ones of nok clear, the next bit sets
  int64_t nok = k0, okA = 0, okB = 0;
  for (int j = 0; j < p.n_ok; ++j)
    if ((nok >> j) & 1) {
      okA += int64_t(1) << p.ok_A[j];
      okB += int64_t(1) << p.ok_B[j];
    }
  // copies of K step `it` (= nok - k0) into stage it % NS; one commit group per call (empty
  // past the end)
  auto issue = [&](int64_t it) {
    if (it < per) {
      const uint32_t st = sbase + uint32_t(it % NS) * stage_bytes;
      const uint32_t esz = uint32_t(sizeof(T));
      stream_copy<T>(Abase + okA, Abase + okA + p.planeA, p.mt + p.kt, p.runA, hiA, st, st + uint32_t(nA) * esz);
      stream_copy<T>(Bbase + okB, Bbase + okB + p.planeB, p.kt + p.nt, p.runB, hiB, st + uint32_t(2 * nA) * esz,
                     st + uint32_t(2 * nA + nB) * esz);
      int j = 0;
      for (; j < p.n_ok && ((nok >> j) & 1); ++j) {
        okA -= int64_t(1) << p.ok_A[j];
        okB -= int64_t(1) << p.ok_B[j];
      }
      if (j < p.n_ok) {
        okA += int64_t(1) << p.ok_A[j];
        okB += int64_t(1) << p.ok_B[j];
      }
      ++nok;
    }
    cpa_commit();
  };
  for (int s0 = 0; s0 < NS - 1; ++s0) issue(s0);
  for (int64_t it = 0; it < per; ++it) {
    cpa_wait<NS - 2>();  // this thread's copies of step `it` have landed
    __syncthreads();     // everyone's have, and everyone is done with step it - 1
    issue(it + NS - 1);  // refills the stage of step it - 1
    if (active) {
      const T* Ar = reinterpret_cast<const T*>(smem + uint32_t(it % NS) * stage_bytes);
      const T* Ai = Ar + nA;
      const T* Br = Ai + nA;
      const T* Bi = Br + nB;
      if (p.kvb == 0) {
        for (int k = grp; k < nk; k += p.kgroups) {
          const int ka = TAk[k], kb = TBk[k];
          float2 a[RM], b[RN];
#pragma unroll
          for (int i = 0; i < RM; ++i) a[i] = make_float2(Conv<T>::to_f(Ar[am[i] ^ ka]), Conv<T>::to_f(Ai[am[i] ^ ka]));
#pragma unroll
          for (int j = 0; j < RN; ++j) b[j] = make_float2(Conv<T>::to_f(Br[kb ^ bn[j]]), Conv<T>::to_f(Bi[kb ^ bn[j]]));
          cmac_tile<RM, RN>(acc, a, b);
        }
      } else {
        // chunks of VE consecutive k (kvb = log2 VE): the chunk of each tile row and column
        // is one contiguous, 8-byte aligned run (the low tile bits of both operands are K
        // bits 0..kvb-1, which the swizzle leaves alone); the lanes of a warp take adjacent
        // chunks, so one load instruction reads 256 contiguous bytes
        constexpr int VE = 8 / sizeof(T);
        for (int c = grp; c < nk / VE; c += p.kgroups) {
          const int ka = TAk[c * VE], kb = TBk[c * VE];
          uint2 vr[RM], vi[RM], wr[RN], wi[RN];
#pragma unroll
          for (int i = 0; i < RM; ++i) {
            vr[i] = *reinterpret_cast<const uint2*>(Ar + (am[i] ^ ka));
            vi[i] = *reinterpret_cast<const uint2*>(Ai + (am[i] ^ ka));
          }
#pragma unroll
          for (int j = 0; j < RN; ++j) {
            wr[j] = *reinterpret_cast<const uint2*>(Br + (kb ^ bn[j]));
            wi[j] = *reinterpret_cast<const uint2*>(Bi + (kb ^ bn[j]));
          }
          if constexpr (sizeof(T) == 2) {
#pragma unroll
            for (int v = 0; v < VE; ++v) cmac_tile16<T, RM, RN>(acc, vr, vi, wr, wi, v);
          } else {
#pragma unroll
            for (int v = 0; v < VE; ++v) {
              float2 a[RM], b[RN];
#pragma unroll
              for (int i = 0; i < RM; ++i)
                a[i] = make_float2(Conv<T>::to_f(reinterpret_cast<const T*>(&vr[i])[v]),
                                   Conv<T>::to_f(reinterpret_cast<const T*>(&vi[i])[v]));
#pragma unroll
              for (int j = 0; j < RN; ++j)
                b[j] = make_float2(Conv<T>::to_f(reinterpret_cast<const T*>(&wr[j])[v]),
                                   Conv<T>::to_f(reinterpret_cast<const T*>(&wi[j])[v]));
              cmac_tile<RM, RN>(acc, a, b);
            }
          }
        }
      }
    }
  }
  cpa_wait<0>();
  __syncthreads();  // the ring becomes the reduction buffer
  const int sh = p.splitk == 1 ? generic_shift(p, I) : 0;
  const float mx = generic_finish<T, RM, RN>(p, I, acc, active, grp, mi, ni, TM, TN, TCm, TCn, hiC, R, oC, ldexpf(1.f, -sh),
                                             blockIdx.y, blockIdx.z);
  if (p.splitk == 1) generic_publish(p, I, mx, red, sh, blockIdx.x == 0);
}

// Fixed-order sum of split-K partials (blocked summation, Eq. 3), then scale and store: block
// bx of launch index bz (k_splitk_reduce, and the reduce units of k_steps).
template <typename T>
__device__ __forceinline__ void splitk_reduce_cta(const GenParams& p, float* red, uint32_t bx, uint32_t bz) {
  const Inst3 I = map_inst(bz, p.im);
  const int64_t idx = int64_t(bx) * kThreads + threadIdx.x;
  const int64_t sa = I.a * p.n_slots, sbb = I.b * p.n_slots, sc = I.c * p.n_slots;
  const int sh = product_shift(p.maxabs[sa + p.slotA], p.maxabs[sbb + p.slotB], p.nK);
  const float scale = ldexpf(1.f, -sh);
  float mx = 0.f;
  if (idx < p.planeC) {
    const float2* part = p.partials + int64_t(bz) * p.splitk * p.planeC + idx;
    float2 s = part[0];
    for (int k = 1; k < p.splitk; ++k) {
      const float2 v = part[int64_t(k) * p.planeC];
      s.x += v.x;
      s.y += v.y;
    }
    T* Cre = reinterpret_cast<T*>(p.C) + I.c * p.strideC;
    const T re = Conv<T>::from_f(s.x * scale), im = Conv<T>::from_f(s.y * scale);
    Cre[idx] = re;
    Cre[p.planeC + idx] = im;
    mx = fmaxf(fabsf(Conv<T>::to_f(re)), fabsf(Conv<T>::to_f(im)));
  }
  const float bm = block_max(mx, red);
  if (threadIdx.x == 0) {
    atomic_max_nonneg(&p.maxabs[sc + p.slotC], bm);
    if (bx == 0) p.exps[sc + p.slotC] = p.exps[sa + p.slotA] + p.exps[sbb + p.slotB] + sh;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_splitk_reduce(const GenParams p) {
  __shared__ float red[32];
  splitk_reduce_cta<T>(p, red, blockIdx.x, blockIdx.z);
}

// The same sum for long splits over few outputs: one warp per output, lane l adds the
// partials l, l + 32, l + 64, ... in order, then the lanes combine in a fixed butterfly
// (xor 16, 8, 4, 2, 1), so the result is deterministic; 8 outputs per block.
template <typename T>
__device__ __forceinline__ void splitk_reduce_wide_cta(const GenParams& p, float* red, uint32_t bx, uint32_t bz) {
  const Inst3 I = map_inst(bz, p.im);
  const int lane = threadIdx.x & 31;
  const int64_t idx = int64_t(bx) * (kThreads / 32) + (threadIdx.x >> 5);
  const int64_t sa = I.a * p.n_slots, sbb = I.b * p.n_slots, sc = I.c * p.n_slots;
  const int sh = product_shift(p.maxabs[sa + p.slotA], p.maxabs[sbb + p.slotB], p.nK);
  const float scale = ldexpf(1.f, -sh);
  float mx = 0.f;
  float2 s = make_float2(0.f, 0.f);
  if (idx < p.planeC) {
    const float2* part = p.partials + int64_t(bz) * p.splitk * p.planeC + idx;
#pragma unroll 8
    for (int k = lane; k < p.splitk; k += 32) {
      const float2 v = part[int64_t(k) * p.planeC];
      s.x += v.x;
      s.y += v.y;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
    s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
  }
  if (idx < p.planeC && lane == 0) {
    T* Cre = reinterpret_cast<T*>(p.C) + I.c * p.strideC;
    const T re = Conv<T>::from_f(s.x * scale), im = Conv<T>::from_f(s.y * scale);
    Cre[idx] = re;
    Cre[p.planeC + idx] = im;
    mx = fmaxf(fabsf(Conv<T>::to_f(re)), fabsf(Conv<T>::to_f(im)));
  }
  const float bm = block_max(mx, red);
  if (threadIdx.x == 0) {
    atomic_max_nonneg(&p.maxabs[sc + p.slotC], bm);
    if (bx == 0) p.exps[sc + p.slotC] = p.exps[sa + p.slotA] + p.exps[sbb + p.slotB] + sh;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_splitk_reduce_wide(const GenParams p) {
  __shared__ float red[32];
  splitk_reduce_wide_cta<T>(p, red, blockIdx.x, blockIdx.z);
}

// Grid-wide barrier of the persistent steps kernel (all CTAs co-resident: cooperative launch).
// bar[0] counts arrivals, bar[1] is the generation.  The last CTA to arrive resets the count,
// then opens the next generation; the others wait for it, at most about two seconds, after
// which the wait records TNC_E_TIMEOUT and the kernel returns.
__device__ __forceinline__ bool grid_barrier(uint32_t* bar, int32_t* status) {
  __shared__ int ok_flag;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile uint32_t* gen = bar + 1;
    const uint32_t g = *gen;
    __threadfence();  // this CTA's writes before the arrival
    int ok = 1;
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      int it = 0;
      while (*gen == g) {
        if (++it > (1 << 24)) {
          atomicExch(status, 4);  // TNC_E_TIMEOUT
          ok = 0;
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();  // the other CTAs' writes before this CTA's next reads
    ok_flag = ok;
  }
  __syncthreads();
  return ok_flag != 0;
}

template <typename T>
__device__ __forceinline__ void generic_unit(int rm, int rn, const GenParams& p, unsigned char* smem, uint32_t bx,
                                             uint32_t gx, uint32_t by, uint32_t bz) {
#define TNC_UNIT(a, b) \
  if (rm == a && rn == b) return generic_cta<T, a, b, true>(p, smem, bx, gx, by, bz);
  TNC_UNIT(1, 1) TNC_UNIT(1, 2) TNC_UNIT(1, 4) TNC_UNIT(2, 1) TNC_UNIT(2, 2) TNC_UNIT(2, 4)
  TNC_UNIT(4, 1) TNC_UNIT(4, 2) TNC_UNIT(4, 4) TNC_UNIT(8, 4)
#undef TNC_UNIT
}

// One persistent launch for all SIMT steps of a wave (Sec. III-A: a wave's subtasks in one
// launch).  The steps come grouped in phases: a phase holds steps that depend on no step of
// the same phase (operands, arena memory, the shared partial-sum buffer), so their units run
// together, spread over the grid; a grid barrier closes each phase, and the reduces of its
// split steps run after it, before another barrier.  Results are bit-identical to per-step
// launches: every tile, split and reduce block computes the same sums in the same order
// wherever it runs.
struct StepUnits {
  uint32_t gx, gy;
  int64_t units;
};
__device__ __forceinline__ StepUnits step_units(const StepOp& op, int64_t n_inst, int reuse, int64_t target) {
  const InstMap im = reuse ? op.p.im : InstMap{-1, 0u, 0u, 0u};
  const int64_t nz = im.s < 0 ? n_inst : ((n_inst >> im.s) << __popc(im.dep_c));
  const uint32_t gy = (uint32_t)op.p.splitk;
  const int64_t n_tiles = int64_t(1) << (op.p.n_om + op.p.n_on);
  const int64_t cols = int64_t(gy) * nz;
  // tile strides per (split, launch index) column: about `target` units per step
  const uint32_t gx = (uint32_t)max(int64_t(1), min(n_tiles, (target + cols - 1) / cols));
  return StepUnits{gx, gy, int64_t(gx) * cols};
}
__device__ __forceinline__ int64_t reduce_units(const StepOp& op, int64_t n_inst, int reuse) {
  if (!op.reduce) return 0;
  const InstMap im = reuse ? op.p.im : InstMap{-1, 0u, 0u, 0u};
  const int64_t nz = im.s < 0 ? n_inst : ((n_inst >> im.s) << __popc(im.dep_c));
  const int64_t per =
      op.reduce == 2 ? (op.p.planeC + kThreads / 32 - 1) / (kThreads / 32) : (op.p.planeC + kThreads - 1) / kThreads;
  return per * nz;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_steps(const StepOp* __restrict__ ops, const int32_t* __restrict__ phases,
                                                   int n_phases, int64_t n_inst, int reuse, uint32_t* bar,
                                                   int32_t* status) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(16) GenParams P;
  __shared__ float red[32];
  int loaded = -1;
  // the op's parameters into shared memory (uniform per CTA: every thread takes part)
  auto load_op = [&](int o) {
    if (o == loaded) return;
    __syncthreads();
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&ops[o].p);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&P);
    for (int i = threadIdx.x; i < int(sizeof(GenParams) / 4); i += kThreads) dst[i] = src[i];
    __syncthreads();
    if (threadIdx.x == 0 && !reuse) P.im = InstMap{-1, 0u, 0u, 0u};
    __syncthreads();
    loaded = o;
  };
  const int64_t target = int64_t(8) * gridDim.x;
  for (int ph = 0; ph < n_phases; ++ph) {
    const int o0 = phases[ph], o1 = phases[ph + 1];
    int64_t total = 0;
    bool any_reduce = false;
    for (int o = o0; o < o1; ++o) {
      total += step_units(ops[o], n_inst, reuse, target).units;
      any_reduce |= ops[o].reduce != 0;
    }
    for (int64_t u = blockIdx.x; u < total; u += gridDim.x) {
      int o = o0;
      int64_t v = u;
      StepUnits su = step_units(ops[o], n_inst, reuse, target);
      while (v >= su.units) {
        v -= su.units;
        su = step_units(ops[++o], n_inst, reuse, target);
      }
      load_op(o);
      const uint32_t bx = (uint32_t)(v % su.gx);
      const int64_t r = v / su.gx;
      generic_unit<T>(ops[o].rm, ops[o].rn, P, smem, bx, su.gx, (uint32_t)(r % su.gy), (uint32_t)(r / su.gy));
      __syncthreads();
    }
    if (!grid_barrier(bar, status)) return;
    if (any_reduce) {
      int64_t rtotal = 0;
      for (int o = o0; o < o1; ++o) rtotal += reduce_units(ops[o], n_inst, reuse);
      for (int64_t u = blockIdx.x; u < rtotal; u += gridDim.x) {
        int o = o0;
        int64_t v = u;
        int64_t ru = reduce_units(ops[o], n_inst, reuse);
        while (v >= ru) {
          v -= ru;
          ru = reduce_units(ops[++o], n_inst, reuse);
        }
        load_op(o);
        const int64_t per = ops[o].reduce == 2 ? (P.planeC + kThreads / 32 - 1) / (kThreads / 32)
                                               : (P.planeC + kThreads - 1) / kThreads;
        if (ops[o].reduce == 2) splitk_reduce_wide_cta<T>(P, red, (uint32_t)(v % per), (uint32_t)(v / per));
        else splitk_reduce_cta<T>(P, red, (uint32_t)(v % per), (uint32_t)(v / per));
        __syncthreads();
      }
      if (!grid_barrier(bar, status)) return;
    }
  }
}

// One warp per (leaf, instance).  Leaves have at most 4 free legs after fixing.
template <typename T>
__global__ void k_leaf_gather(const LeafDesc* __restrict__ leaves, const double2* __restrict__ src, T* arena,
                              int64_t inst_stride, const int64_t* __restrict__ inst_slice,
                              const int32_t* __restrict__ inst_row, const uint8_t* __restrict__ bits, int n_qubits,
                              float* maxabs, int32_t* exps, int n_slots, int64_t inst_base, double2* leaf_r,
                              int n_leaves) {
  const LeafDesc d = leaves[blockIdx.x];
  const int64_t inst = blockIdx.y;
  const int64_t slice = inst_slice[inst_base + inst];
  const int row = inst_row[inst_base + inst];
  const int lane = threadIdx.x;
  const int n = 1 << d.rank;
  double2 v = make_double2(0.0, 0.0);
  if (lane < n) {
    // place the free index bits and the fixed values into the full leaf index
    int64_t full = 0;
    int fb = 0, f = 0;
    for (int pos = 0; pos < d.rank_full; ++pos) {
      int bit;
      if (f < d.nfix && d.fix_pos[f] == pos) {
        bit = d.fix_kind[f] == 0 ? (d.fix_idx[f] < 63 ? int((slice >> d.fix_idx[f]) & 1) : 0)
                                 : int(bits[int64_t(row) * n_qubits + d.fix_idx[f]]);
        ++f;
      } else {
        bit = (lane >> fb) & 1;
        ++fb;
      }
      full |= int64_t(bit) << pos;
    }
    v = src[d.src + full];
  }
  double m = fmax(fabs(v.x), fabs(v.y));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  int e = 0;
  if (m > 0.0) {
    frexp(m, &e);  // m < 2^e: stored values below 1
  }
  const double s = ldexp(1.0, -e);
  T* dst = arena + inst * inst_stride + d.dst;
  float mx = 0.f;
  // least-squares scale r of the rounded leaf q against the exact one v: v ~ r q.  The
  // amplitude is linear in every leaf, so multiplying it by the product of the instance's
  // r removes the coherent part of the storage rounding (the same few gate values round
  // the same way in every leaf); the rest of the rounding error stays
  double nr = 0.0, ni = 0.0, dd = 0.0;
  if (lane < n) {
    const T re = Conv<T>::from_f((float)(v.x * s)), im = Conv<T>::from_f((float)(v.y * s));
    dst[lane] = re;
    dst[n + lane] = im;
    mx = fmaxf(fabsf(Conv<T>::to_f(re)), fabsf(Conv<T>::to_f(im)));
    const double qr = (double)Conv<T>::to_f(re), qi = (double)Conv<T>::to_f(im);
    const double vr = v.x * s, vi = v.y * s;
    nr = qr * vr + qi * vi;  // conj(q) * v
    ni = qr * vi - qi * vr;
    dd = qr * qr + qi * qi;
  }
  for (int o = 16; o > 0; o >>= 1) {
    nr += __shfl_xor_sync(0xffffffffu, nr, o);
    ni += __shfl_xor_sync(0xffffffffu, ni, o);
    dd += __shfl_xor_sync(0xffffffffu, dd, o);
  }
  if (leaf_r && lane == 0) leaf_r[inst * n_leaves + blockIdx.x] = dd > 0.0 ? make_double2(nr / dd, ni / dd) : make_double2(1.0, 0.0);
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) {
    maxabs[inst * n_slots + d.slot] = mx;
    exps[inst * n_slots + d.slot] = e;
  }
}

// c[i] = product over the leaves (in leaf order) of instance i's leaf scales r.
__global__ void k_inst_scale(const double2* __restrict__ leaf_r, int n_leaves, int64_t n_inst, double2* c) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_inst) return;
  double pr = 1.0, pi = 0.0;
  for (int l = 0; l < n_leaves; ++l) {
    const double2 r = leaf_r[i * n_leaves + l];
    const double t = pr * r.x - pi * r.y;
    pi = pr * r.y + pi * r.x;
    pr = t;
  }
  c[i] = make_double2(pr, pi);
}

cudaError_t launch_inst_scale(const double2* leaf_r, int n_leaves, int64_t n_inst, double2* c, cudaStream_t s) {
  k_inst_scale<<<(unsigned)((n_inst + 127) / 128), 128, 0, s>>>(leaf_r, n_leaves, n_inst, c);
  return cudaGetLastError();
}

// acc[row, o] += sum over the segment's instances (in order) of root[o] * 2^E (times the
// instance's leaf-rounding scale c when given).
template <typename T>
__global__ void k_root_accum(const T* __restrict__ arena, int64_t inst_stride, int64_t root_off, int64_t plane,
                             const int8_t* __restrict__ open_pos, int n_open, const RootSeg* __restrict__ segs,
                             const int32_t* __restrict__ exps, int n_slots, int root_slot, double2* acc,
                             const double2* __restrict__ cfac, InstMap rm, uint32_t merged) {
  const int64_t o = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t n_out = int64_t(1) << n_open;
  if (o >= n_out) return;
  const RootSeg s = segs[blockIdx.y];
  int64_t idx = 0;
  for (int j = 0; j < n_open; ++j) idx |= ((o >> (n_open - 1 - j)) & 1) << open_pos[j];
  // added one instance at a time, in slice order, onto the running value: the same
  // association whatever the wave size
  double2* a = acc + int64_t(s.row) * n_out + o;
  double re = a->x, im = a->y;
  for (int i = s.begin; i < s.end; ++i) {
    // slices whose merged indices (post-lifetime merging) are not all 0 are already summed
    // into the slice with those indices 0
    if (rm.s >= 0 && (uint32_t(i) & merged)) continue;
    // the root of a slice is stored at the instance that keeps only the slice bits it
    // depends on (tree-like reuse); the leaf-rounding scale is per instance
    const int64_t ir = rm.s < 0 ? int64_t(i) : ((int64_t(i) >> rm.s << rm.s) | (int64_t(i) & int64_t(rm.dep_c)));
    const T* root = arena + ir * inst_stride + root_off;
    const double sc = ldexp(1.0, exps[ir * n_slots + root_slot]);
    const double xr = (double)Conv<T>::to_f(root[idx]) * sc, xi = (double)Conv<T>::to_f(root[plane + idx]) * sc;
    if (cfac) {
      const double2 c = cfac[i];
      re += xr * c.x - xi * c.y;
      im += xr * c.y + xi * c.x;
    } else {
      re += xr;
      im += xi;
    }
  }
  a->x = re;
  a->y = im;
}

// Post-lifetime merging (Sec. III-B: (sum_i A_i) B in place of sum_i A_i B).  Once the
// step that contracts sliced index t has run, its result X depends on t only through its
// values and everything downstream is linear in X, so the two values of t are summed at once
// and the rest of the tree runs once for both:
//   X'(t=0) = X(t=0) 2^(E0-E) + f X(t=1) 2^(E1-E),   E = max(E0, E1) + 2,
// stored in place at the t = 0 instance, exponent E.  f = r_u r_v (t=1) / r_u r_v (t=0) is the
// ratio of the leaf-rounding scales of the two leaves holding t (the only leaves whose
// values differ between the two instances), so that the root's per-slice scale of the t = 0
// slice stays exact for the merged sum.  Launch index y enumerates (row, assignment of the
// result's other sliced indices) through `im` (dep_c without t).
__device__ __forceinline__ double2 merge_factor(const double2* leaf_r, int n_leaves, int lu, int lv, int64_t i0,
                                                int64_t i1) {
  if (!leaf_r) return make_double2(1.0, 0.0);
  auto mul = [](double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); };
  const double2 n = mul(leaf_r[i1 * n_leaves + lu], leaf_r[i1 * n_leaves + lv]);
  const double2 d = mul(leaf_r[i0 * n_leaves + lu], leaf_r[i0 * n_leaves + lv]);
  const double dd = d.x * d.x + d.y * d.y;
  return make_double2((n.x * d.x + n.y * d.y) / dd, (n.y * d.x - n.x * d.y) / dd);
}

template <typename T>
__global__ void __launch_bounds__(256) k_merge(T* arena, int64_t inst_stride, int64_t off, int64_t plane,
                                               const int32_t* __restrict__ exps, int n_slots, int slot,
                                               const double2* __restrict__ leaf_r, int n_leaves, int lu, int lv,
                                               int bit, InstMap im) {
  const Inst3 I = map_inst(blockIdx.y, im);
  const int64_t i0 = I.c, i1 = I.c | (int64_t(1) << bit);
  const int E0 = exps[i0 * n_slots + slot], E1 = exps[i1 * n_slots + slot];
  const int E = max(E0, E1) + 2;
  const float s0 = ldexpf(1.f, E0 - E), s1 = ldexpf(1.f, E1 - E);
  const double2 f = merge_factor(leaf_r, n_leaves, lu, lv, i0, i1);
  const float fr = (float)f.x * s1, fi = (float)f.y * s1;
  T* x0 = arena + i0 * inst_stride + off;
  const T* x1 = arena + i1 * inst_stride + off;
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < plane; j += int64_t(gridDim.x) * blockDim.x) {
    const float ar = Conv<T>::to_f(x0[j]) * s0, ai = Conv<T>::to_f(x0[plane + j]) * s0;
    const float br = Conv<T>::to_f(x1[j]), bi = Conv<T>::to_f(x1[plane + j]);
    x0[j] = Conv<T>::from_f(ar + fr * br - fi * bi);
    x0[plane + j] = Conv<T>::from_f(ai + fr * bi + fi * br);
  }
}

// The merged tensor's exponent and a bound on its stored |re|, |im| (for the next producer's
// scaling): |x0| s0 + |f| (|re x1| + |im x1|) s1 <= m0 s0 + 2 |f| m1 s1.  Runs after k_merge,
// which reads the old exponents.
__global__ void k_merge_meta(int32_t* exps, float* maxabs, int n_slots, int slot, const double2* __restrict__ leaf_r,
                             int n_leaves, int lu, int lv, int bit, InstMap im, int64_t nz) {
  const int64_t z = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (z >= nz) return;
  const Inst3 I = map_inst(z, im);
  const int64_t i0 = I.c, i1 = I.c | (int64_t(1) << bit);
  const int E0 = exps[i0 * n_slots + slot], E1 = exps[i1 * n_slots + slot];
  const int E = max(E0, E1) + 2;
  const double2 f = merge_factor(leaf_r, n_leaves, lu, lv, i0, i1);
  const double af = sqrt(f.x * f.x + f.y * f.y);
  const double m = maxabs[i0 * n_slots + slot] * ldexp(1.0, E0 - E) + 2.0 * af * maxabs[i1 * n_slots + slot] * ldexp(1.0, E1 - E);
  maxabs[i0 * n_slots + slot] = (float)(m * (1.0 + 0x1p-8));
  exps[i0 * n_slots + slot] = E;
}

cudaError_t launch_merge(int precision, void* arena, int64_t inst_stride, int64_t off, int64_t plane, int32_t* exps,
                         float* maxabs, int n_slots, int slot, const double2* leaf_r, int n_leaves, int lu, int lv,
                         int bit, InstMap im, int64_t nz, cudaStream_t s) {
  if (nz <= 0) return cudaSuccess;
  const int64_t per = (plane + 255) / 256;
  const unsigned bx = (unsigned)std::min<int64_t>(per, std::max<int64_t>(1, (4 * 152 + nz - 1) / nz));
  const dim3 grid(bx, (unsigned)nz, 1);
  if (precision == 0)
    k_merge<float><<<grid, 256, 0, s>>>((float*)arena, inst_stride, off, plane, exps, n_slots, slot, leaf_r, n_leaves, lu,
                                        lv, bit, im);
  else if (precision == 1)
    k_merge<__half><<<grid, 256, 0, s>>>((__half*)arena, inst_stride, off, plane, exps, n_slots, slot, leaf_r, n_leaves,
                                         lu, lv, bit, im);
  else
    k_merge<__nv_bfloat16><<<grid, 256, 0, s>>>((__nv_bfloat16*)arena, inst_stride, off, plane, exps, n_slots, slot,
                                                leaf_r, n_leaves, lu, lv, bit, im);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_merge_meta<<<(unsigned)((nz + 127) / 128), 128, 0, s>>>(exps, maxabs, n_slots, slot, leaf_r, n_leaves, lu, lv, bit,
                                                             im, nz);
  return cudaGetLastError();
}

// Root cotangent of every instance: dL/droot[o] = w[row, o] (holomorphic derivative of
// L = sum w * amp), stored as FP32 times 2^-e_row with e_row from the row's largest |w|.
__global__ void k_adj_root_init(float* arena, int64_t inst_stride, int64_t root_off, int64_t plane,
                                const int8_t* __restrict__ open_pos, int n_open, const int32_t* __restrict__ inst_row,
                                int64_t inst_base, const double2* __restrict__ w, const int32_t* __restrict__ erow,
                                float* maxabs, int32_t* exps, int n_slots, int slot) {
  __shared__ float red[32];
  const int64_t n_out = int64_t(1) << n_open;
  const int64_t o = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t inst = blockIdx.y;
  const int row = inst_row[inst_base + inst];
  const int e = erow[row];
  float mx = 0.f;
  if (o < n_out) {
    int64_t idx = 0;
    for (int j = 0; j < n_open; ++j) idx |= ((o >> (n_open - 1 - j)) & 1) << open_pos[j];
    const double2 v = w[int64_t(row) * n_out + o];
    float* r = arena + inst * inst_stride + root_off;
    const float re = (float)ldexp(v.x, -e), im = (float)ldexp(v.y, -e);
    r[idx] = re;
    r[plane + idx] = im;
    mx = fmaxf(fabsf(re), fabsf(im));
  }
  const float bm = block_max(mx, red);
  if (threadIdx.x == 0) {
    atomic_max_nonneg(&maxabs[inst * n_slots + slot], bm);
    if (blockIdx.x == 0) exps[inst * n_slots + slot] = e;
  }
}

cudaError_t launch_adj_root_init(float* arena, int64_t inst_stride, int64_t root_off, int64_t plane,
                                 const int8_t* open_pos, int n_open, const int32_t* inst_row, int64_t inst_base,
                                 int64_t n_inst, const double2* w, const int32_t* erow, float* maxabs, int32_t* exps,
                                 int n_slots, int slot, cudaStream_t s) {
  const int64_t n_out = int64_t(1) << n_open;
  dim3 grid((unsigned)((n_out + 255) / 256), (unsigned)n_inst);
  k_adj_root_init<<<grid, 256, 0, s>>>(arena, inst_stride, root_off, plane, open_pos, n_open, inst_row, inst_base, w,
                                       erow, maxabs, exps, n_slots, slot);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_maxabs(const T* __restrict__ x, int64_t n, float* out) {
  __shared__ float red[32];
  float m = 0.f;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    m = fmaxf(m, fabsf(Conv<T>::to_f(x[i])));
  const float bm = block_max(m, red);
  if (threadIdx.x == 0) atomic_max_nonneg(out, bm);
}

// Permutation (TTGT transposes): each CTA loads one tile in the input's order with
// contiguous vector loads, and writes it in the output's order with contiguous vector stores,
// reading shared memory through the split permutation table.  Values are copied exactly.
template <typename T, int V>
__device__ __forceinline__ void store_perm_v(T* __restrict__ re, T* __restrict__ im, int bits, int run,
                                             const uint32_t* __restrict__ hi, const float2* __restrict__ buf,
                                             const uint16_t* __restrict__ plo, const uint16_t* __restrict__ phi) {
  const int n = 1 << bits;
  const uint32_t lowmask = (1u << run) - 1u;
  for (int u = threadIdx.x * V; u < n; u += kThreads * V) {
    const uint32_t off = hi[u >> run] + (uint32_t(u) & lowmask);
    Vec<T, V> r, i;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int uu = u + v;
      const float2 x = buf[plo[uu & 63] + phi[uu >> 6]];
      r.v[v] = Conv<T>::from_f(x.x);
      i.v[v] = Conv<T>::from_f(x.y);
    }
    *reinterpret_cast<Vec<T, V>*>(re + off) = r;
    *reinterpret_cast<Vec<T, V>*>(im + off) = i;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_permute(const PermParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* buf = reinterpret_cast<float2*>(smem);                          // [2^bits]
  uint32_t* hiI = reinterpret_cast<uint32_t*>(buf + (1 << p.bits));       // [2^(bits - run_in)]
  uint32_t* hiO = hiI + (1 << (p.bits - p.run_in));                        // [2^(bits - run_out)]
  uint16_t* plo = reinterpret_cast<uint16_t*>(hiO + (1 << (p.bits - p.run_out)));  // [64]
  uint16_t* phi = plo + 64;                                                // [64]
  const int tid = threadIdx.x;
  int64_t oI = 0, oO = 0;
  for (int j = 0; j < p.n_o; ++j)
    if ((blockIdx.x >> j) & 1u) oI += int64_t(1) << p.o_in[j], oO += int64_t(1) << p.o_out[j];
  for (int h = tid; h < (1 << (p.bits - p.run_in)); h += kThreads) hiI[h] = deposit_hi(h, p.mask_in, p.run_in);
  for (int h = tid; h < (1 << (p.bits - p.run_out)); h += kThreads) hiO[h] = deposit_hi(h, p.mask_out, p.run_out);
  if (tid < 64) {
    plo[tid] = p.plo[tid];
    phi[tid] = p.phi[tid];
  }
  __syncthreads();
  const T* in = reinterpret_cast<const T*>(p.in) + oI;
  load_tile<T>(in, in + p.plane, p.bits, p.run_in, hiI, buf);
  __syncthreads();
  T* out = reinterpret_cast<T*>(p.out) + oO;
  constexpr int VMAX = 16 / sizeof(T);
  const int v = min(1 << p.run_out, VMAX);
  if (v >= 8) store_perm_v<T, (VMAX >= 8 ? 8 : 1)>(out, out + p.plane, p.bits, p.run_out, hiO, buf, plo, phi);
  else if (v == 4) store_perm_v<T, 4>(out, out + p.plane, p.bits, p.run_out, hiO, buf, plo, phi);
  else if (v == 2) store_perm_v<T, 2>(out, out + p.plane, p.bits, p.run_out, hiO, buf, plo, phi);
  else store_perm_v<T, 1>(out, out + p.plane, p.bits, p.run_out, hiO, buf, plo, phi);
}

size_t permute_smem_bytes(const PermParams& p) {
  return (size_t(1) << p.bits) * 8 + (size_t(1) << (p.bits - p.run_in)) * 4 + (size_t(1) << (p.bits - p.run_out)) * 4 +
         128 * 2 + 16;
}

cudaError_t launch_permute(int precision, const PermParams& p, cudaStream_t s) {
  const size_t smem = permute_smem_bytes(p);
  const dim3 grid(1u << p.n_o);
  cudaError_t e;
  if (precision == 0) {
    if ((e = set_smem_once(reinterpret_cast<const void*>(k_permute<float>), smem)) != cudaSuccess) return e;
    k_permute<float><<<grid, kThreads, smem, s>>>(p);
  } else if (precision == 1) {
    if ((e = set_smem_once(reinterpret_cast<const void*>(k_permute<__half>), smem)) != cudaSuccess) return e;
    k_permute<__half><<<grid, kThreads, smem, s>>>(p);
  } else {
    if ((e = set_smem_once(reinterpret_cast<const void*>(k_permute<__nv_bfloat16>), smem)) != cudaSuccess) return e;
    k_permute<__nv_bfloat16><<<grid, kThreads, smem, s>>>(p);
  }
  return cudaGetLastError();
}

// Fused chain: load a tile of A0 over the on-chip labels, apply every link in FP32 in
// shared memory (out[x] = sum_k in[in_tab[x] + kin[k]] * g[g_tab[x] + kg[k]]), store the
// result tile once.  The result is scaled by the power of two that brings the bound
// sqrt2 * max|A0| * prod_links max_n sum_k |g[k, n]| below 2^15 (|C| cannot exceed it).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_chain(const ChainParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* buf0 = reinterpret_cast<float2*>(smem);
  float2* buf1 = buf0 + (1 << kChainMaxBits);
  float2* gs = buf1 + (1 << kChainMaxBits);                        // [64]
  uint16_t* kin = reinterpret_cast<uint16_t*>(gs + 64);              // [64]
  uint16_t* ibl = kin + 64;                                          // [64]
  uint16_t* ibh = ibl + 64;                                          // [64]
  uint8_t* kg = reinterpret_cast<uint8_t*>(ibh + 64);                // [64]
  uint8_t* gbl = kg + 64;                                            // [64]
  uint8_t* gbh = gbl + 64;                                           // [64]
  float* red = reinterpret_cast<float*>(gbh + 64);                   // [36]
  uint32_t* hiA = reinterpret_cast<uint32_t*>(red + 36);             // [2^(bits0 - runA0)]
  uint32_t* hiC = hiA + (1 << (p.bits0 - p.runA0));                  // [2^(bitsC - runC)]
  const int tid = threadIdx.x;
  const int64_t inst = blockIdx.z;
  const uint32_t o = blockIdx.x;
  int64_t oA = 0, oC = 0;
  for (int j = 0; j < p.n_o; ++j)
    if ((o >> j) & 1u) oA += int64_t(1) << p.o_A[j], oC += int64_t(1) << p.o_C[j];
  for (int h = tid; h < (1 << (p.bits0 - p.runA0)); h += kThreads) hiA[h] = deposit_hi(h, p.maskA0, p.runA0);
  for (int h = tid; h < (1 << (p.bitsC - p.runC)); h += kThreads) hiC[h] = deposit_hi(h, p.maskC, p.runC);
  __syncthreads();
  const T* base = reinterpret_cast<const T*>(p.arena) + inst * p.stride;
  const T* A0 = base + p.offA0 + oA;
  load_tile<T>(A0, A0 + p.planeA0, p.bits0, p.runA0, hiA, buf0);
  const int64_t sb = inst * p.n_slots;
  float bound = 1.41421356f * p.maxabs[sb + p.slotA0];
  int esum = p.exps[sb + p.slotA0];
  float2* in = buf0;
  float2* out = buf1;
  for (int l = 0; l < p.n_links; ++l) {
    const ChainLink* L = p.links + l;
    const T* g = base + L->g_off;
    for (int t = tid; t < L->g_size; t += kThreads) gs[t] = make_float2(Conv<T>::to_f(g[t]), Conv<T>::to_f(g[L->g_plane + t]));
    const int nk = 1 << L->k_bits;
    if (tid < 64) {
      kin[tid] = L->kin[tid];
      kg[tid] = L->kg[tid];
      ibl[tid] = L->ib_lo[tid];
      ibh[tid] = L->ib_hi[tid];
      gbl[tid] = L->gb_lo[tid];
      gbh[tid] = L->gb_hi[tid];
    }
    __syncthreads();
    if (tid == 0) {
      // column norm of the small operand: max over free-label assignments of sum_k |g|
      float cn = 0.f;
      for (int n = 0; n < (1 << L->n_bits); ++n) {
        float s = 0.f;
        for (int q = 0; q < nk; ++q) {
          const float2 v = gs[L->gn[n] + kg[q]];
          s += sqrtf(v.x * v.x + v.y * v.y);
        }
        cn = fmaxf(cn, s);
      }
      red[32] = cn;
    }
    const int nout = 1 << L->out_bits;
    for (int x = tid; x < nout; x += kThreads) {
      const int ib = ibl[x & 63] + ibh[x >> 6], gb = gbl[x & 63] + gbh[x >> 6];
      float2 acc = make_float2(0.f, 0.f);
      for (int q = 0; q < nk; ++q) {
        const float2 a = in[ib + kin[q]];
        const float2 b = gs[gb + kg[q]];
        acc.x = fmaf(a.x, b.x, acc.x);
        acc.x = fmaf(-a.y, b.y, acc.x);
        acc.y = fmaf(a.x, b.y, acc.y);
        acc.y = fmaf(a.y, b.x, acc.y);
      }
      out[x] = acc;
    }
    __syncthreads();
    bound *= red[32];
    esum += p.exps[sb + L->slot_g];
    float2* t = in;
    in = out;
    out = t;
  }
  int sh = 0;
  if (bound > 0.f) {
    frexpf(bound, &sh);  // bound < 2^sh
    sh -= 15;
  }
  const float scale = ldexpf(1.f, -sh);
  T* C = reinterpret_cast<T*>(const_cast<void*>(p.arena)) + inst * p.stride + p.offC + oC;
  const float mx = store_tile<T>(C, C + p.planeC, p.bitsC, p.runC, hiC, in, scale);
  const float bm = block_max(mx, red);
  if (tid == 0) {
    atomic_max_nonneg(&p.maxabs[sb + p.slotC], bm);
    if (blockIdx.x == 0) p.exps[sb + p.slotC] = esum + sh;
  }
}

// Cluster-cooperative chain (Sec. IV: the core array's fused sections, with the cluster's
// distributed shared memory in the role of the CPEs' RMA).  A cluster of 2^cl_bits CTAs holds
// one tile of up to 2^(12 + cl_bits) entries: every tile of the chain (the first operand's,
// each link's result) is spread by its top cl_bits labels (the inter-CTA indices), CTA r
// holding the entries whose inter-CTA indices spell r.  The compiler keeps as inter-CTA
// indices the labels contracted latest (Eq. 2: chosen by remaining lifetime), so most links
// read only their own CTA's entries; where a link contracts one of them, or the last tile
// takes the result's order, its inputs come from the other CTAs' shared memory (DSMEM)
// -- the batched index swap of Eq. 2, done while the link computes.  Such a link is
// bracketed by cluster barriers (every input written before anyone reads it; every read of a
// buffer done before its owner overwrites it); a link that reads only its own CTA's entries
// needs a CTA barrier only.
template <typename T, int V>
__device__ __forceinline__ void load_range_v(const T* __restrict__ re, const T* __restrict__ im, int n, uint32_t base,
                                             int run, const uint32_t* __restrict__ hi, float2* __restrict__ dst) {
  const uint32_t lowmask = (1u << run) - 1u;
  for (int t = threadIdx.x * V; t < n; t += kThreads * V) {
    const uint32_t g = base + uint32_t(t);
    const uint32_t off = hi[g >> run] + (g & lowmask);
    const Vec<T, V> r = *reinterpret_cast<const Vec<T, V>*>(re + off);
    const Vec<T, V> i = *reinterpret_cast<const Vec<T, V>*>(im + off);
#pragma unroll
    for (int v = 0; v < V; ++v) dst[t + v] = make_float2(Conv<T>::to_f(r.v[v]), Conv<T>::to_f(i.v[v]));
  }
}

template <typename T, int V>
__device__ __forceinline__ float store_range_v(T* __restrict__ re, T* __restrict__ im, int n, uint32_t base, int run,
                                               const uint32_t* __restrict__ hi, const float2* __restrict__ src,
                                               float scale) {
  const uint32_t lowmask = (1u << run) - 1u;
  float mx = 0.f;
  for (int t = threadIdx.x * V; t < n; t += kThreads * V) {
    const uint32_t g = base + uint32_t(t);
    const uint32_t off = hi[g >> run] + (g & lowmask);
    Vec<T, V> r, i;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const float2 x = src[t + v];
      r.v[v] = Conv<T>::from_f(x.x * scale);
      i.v[v] = Conv<T>::from_f(x.y * scale);
      mx = fmaxf(mx, fmaxf(fabsf(Conv<T>::to_f(r.v[v])), fabsf(Conv<T>::to_f(i.v[v]))));
    }
    *reinterpret_cast<Vec<T, V>*>(re + off) = r;
    *reinterpret_cast<Vec<T, V>*>(im + off) = i;
  }
  return mx;
}

// the vector width of a run of 2^run entries, at most 16 bytes
template <typename T>
__device__ __forceinline__ int range_vec(int run) {
  constexpr int VMAX = 16 / sizeof(T);
  return min(1 << run, VMAX);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_chain_cluster(const ChainParams p) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ float2* peer[2][1 << kChainClusterBits];
  float2* buf[2];
  buf[0] = reinterpret_cast<float2*>(smem);
  buf[1] = buf[0] + (1 << kChainMaxBits);
  float2* gs = buf[1] + (1 << kChainMaxBits);                       // [64]
  uint16_t* kin = reinterpret_cast<uint16_t*>(gs + 64);              // [64]
  uint16_t* ibl = kin + 64;                                          // [64]
  uint16_t* ibh = ibl + 64;                                          // [64]
  uint16_t* ibt = ibh + 64;                                          // [8]
  uint8_t* kg = reinterpret_cast<uint8_t*>(ibt + 8);                 // [64]
  uint8_t* gbl = kg + 64;                                            // [64]
  uint8_t* gbh = gbl + 64;                                           // [64]
  uint8_t* gbt = gbh + 64;                                           // [8]
  float* red = reinterpret_cast<float*>(gbt + 8);                    // [36]
  uint32_t* hiA = reinterpret_cast<uint32_t*>(red + 36);             // [2^(bits0 - runA0)]
  uint32_t* hiC = hiA + (1 << (p.bits0 - p.runA0));                  // [2^(bitsC - runC)]
  const int tid = threadIdx.x;
  const uint32_t r = cluster.block_rank();
  const int cl = 1 << p.cl_bits;
  const int64_t inst = blockIdx.z;
  const uint32_t o = blockIdx.x >> p.cl_bits;  // a cluster = consecutive CTAs along x
  int64_t oA = 0, oC = 0;
  for (int j = 0; j < p.n_o; ++j)
    if ((o >> j) & 1u) oA += int64_t(1) << p.o_A[j], oC += int64_t(1) << p.o_C[j];
  for (int h = tid; h < (1 << (p.bits0 - p.runA0)); h += kThreads) hiA[h] = deposit_hi(h, p.maskA0, p.runA0);
  for (int h = tid; h < (1 << (p.bitsC - p.runC)); h += kThreads) hiC[h] = deposit_hi(h, p.maskC, p.runC);
  if (tid < cl) {
    peer[0][tid] = cluster.map_shared_rank(buf[0], tid);
    peer[1][tid] = cluster.map_shared_rank(buf[1], tid);
  }
  __syncthreads();
  const T* tbase = reinterpret_cast<const T*>(p.arena) + inst * p.stride;
  const T* A0 = tbase + p.offA0 + oA;
  {
    // the first tile in A0's position order: this CTA's entries share its top cl_bits bits
    const int ib0 = p.bits0 - p.cl_bits, v = range_vec<T>(min(p.runA0, ib0));
    const int n0 = 1 << ib0;
    const uint32_t base = r << ib0;
    if (v >= 8) load_range_v<T, (16 / sizeof(T) >= 8 ? 8 : 1)>(A0, A0 + p.planeA0, n0, base, p.runA0, hiA, buf[0]);
    else if (v == 4) load_range_v<T, 4>(A0, A0 + p.planeA0, n0, base, p.runA0, hiA, buf[0]);
    else if (v == 2) load_range_v<T, 2>(A0, A0 + p.planeA0, n0, base, p.runA0, hiA, buf[0]);
    else load_range_v<T, 1>(A0, A0 + p.planeA0, n0, base, p.runA0, hiA, buf[0]);
  }
  const int64_t sb = inst * p.n_slots;
  float bound = 1.41421356f * p.maxabs[sb + p.slotA0];
  int esum = p.exps[sb + p.slotA0];
  cluster.sync();  // every CTA's part of the first tile is on chip
  int cur = 0;
  for (int l = 0; l < p.n_links; ++l) {
    const ChainLink* L = p.links + l;
    const bool remote = L->remote != 0;
    if (remote && l > 0) cluster.sync();  // the other CTAs' inputs of this link are written
    const T* g = tbase + L->g_off;
    for (int t = tid; t < L->g_size; t += kThreads) gs[t] = make_float2(Conv<T>::to_f(g[t]), Conv<T>::to_f(g[L->g_plane + t]));
    const int nk = 1 << L->k_bits;
    if (tid < 64) {
      kin[tid] = L->kin[tid];
      kg[tid] = L->kg[tid];
      ibl[tid] = L->ib_lo[tid];
      ibh[tid] = L->ib_hi[tid];
      gbl[tid] = L->gb_lo[tid];
      gbh[tid] = L->gb_hi[tid];
      if (tid < 8) {
        ibt[tid] = L->ib_top[tid];
        gbt[tid] = L->gb_top[tid];
      }
    }
    __syncthreads();
    if (tid == 0) {
      float cn = 0.f;
      for (int n = 0; n < (1 << L->n_bits); ++n) {
        float sum = 0.f;
        for (int q = 0; q < nk; ++q) {
          const float2 v = gs[L->gn[n] + kg[q]];
          sum += sqrtf(v.x * v.x + v.y * v.y);
        }
        cn = fmaxf(cn, sum);
      }
      red[32] = cn;
    }
    const float2* in = buf[cur];
    float2* out = buf[cur ^ 1];
    const int nout = 1 << L->out_ibits, in_ib = L->in_ibits;
    const uint32_t ibr = ibt[r], gbr = gbt[r];
    for (int x = tid; x < nout; x += kThreads) {
      const uint32_t ib = ibl[x & 63] + ibh[(x >> 6) & 63] + ibr;
      const int gb = gbl[x & 63] + gbh[(x >> 6) & 63] + gbr;
      float2 acc = make_float2(0.f, 0.f);
      for (int q = 0; q < nk; ++q) {
        const uint32_t idx = ib + kin[q];
        const uint32_t owner = idx >> in_ib, loc = idx & ((1u << in_ib) - 1u);
        const float2 a = owner == r ? in[loc] : peer[cur][owner][loc];
        const float2 b = gs[gb + kg[q]];
        acc.x = fmaf(a.x, b.x, acc.x);
        acc.x = fmaf(-a.y, b.y, acc.x);
        acc.y = fmaf(a.x, b.y, acc.y);
        acc.y = fmaf(a.y, b.x, acc.y);
      }
      out[x] = acc;
    }
    if (remote) cluster.sync();  // every read of this CTA's inputs is done before reuse
    else __syncthreads();
    bound *= red[32];
    esum += p.exps[sb + L->slot_g];
    cur ^= 1;
  }
  int sh = 0;
  if (bound > 0.f) {
    frexpf(bound, &sh);  // bound < 2^sh
    sh -= 15;
  }
  const float scale = ldexpf(1.f, -sh);
  T* C = reinterpret_cast<T*>(const_cast<void*>(p.arena)) + inst * p.stride + p.offC + oC;
  float mx = 0.f;
  {
    const int ibC = p.bitsC - p.cl_bits, v = range_vec<T>(min(p.runC, ibC));
    const int nC = 1 << ibC;
    const uint32_t base = r << ibC;
    if (v >= 8) mx = store_range_v<T, (16 / sizeof(T) >= 8 ? 8 : 1)>(C, C + p.planeC, nC, base, p.runC, hiC, buf[cur], scale);
    else if (v == 4) mx = store_range_v<T, 4>(C, C + p.planeC, nC, base, p.runC, hiC, buf[cur], scale);
    else if (v == 2) mx = store_range_v<T, 2>(C, C + p.planeC, nC, base, p.runC, hiC, buf[cur], scale);
    else mx = store_range_v<T, 1>(C, C + p.planeC, nC, base, p.runC, hiC, buf[cur], scale);
  }
  const float bm = block_max(mx, red);
  if (tid == 0) {
    atomic_max_nonneg(&p.maxabs[sb + p.slotC], bm);
    if (o == 0 && r == 0) p.exps[sb + p.slotC] = esum + sh;
  }
}

size_t chain_smem_bytes(int bits0, int runA0, int bitsC, int runC) {
  return (size_t(2) << kChainMaxBits) * 8 + 64 * 8 + 3 * 64 * 2 + 3 * 64 + 36 * 4 + (size_t(1) << (bits0 - runA0)) * 4 +
         (size_t(1) << (bitsC - runC)) * 4 + 16 + 8 * 3;
}

template <typename T>
cudaError_t launch_chain_cluster_t(const ChainParams& p, int64_t n_inst, size_t smem, cudaStream_t s) {
  cudaError_t e = set_smem_once(reinterpret_cast<const void*>(k_chain_cluster<T>), smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((1u << p.n_o) << p.cl_bits, 1, (unsigned)n_inst);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1u << p.cl_bits;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_chain_cluster<T>, p);
}

cudaError_t launch_chain(int precision, const ChainParams& p, int64_t n_inst, cudaStream_t s) {
  const size_t smem = chain_smem_bytes(p.bits0, p.runA0, p.bitsC, p.runC);
  if (p.cl_bits > 0) {
    if (p.cl_bits > kChainClusterBits) return cudaErrorInvalidValue;
    if (precision == 0) return launch_chain_cluster_t<float>(p, n_inst, smem, s);
    if (precision == 1) return launch_chain_cluster_t<__half>(p, n_inst, smem, s);
    return launch_chain_cluster_t<__nv_bfloat16>(p, n_inst, smem, s);
  }
  dim3 grid(1u << p.n_o, 1, (unsigned)n_inst);
  cudaError_t e;
  if (precision == 0) {
    e = set_smem_once(reinterpret_cast<const void*>(k_chain<float>), smem);
    if (e == cudaSuccess) k_chain<float><<<grid, kThreads, smem, s>>>(p);
  } else if (precision == 1) {
    e = set_smem_once(reinterpret_cast<const void*>(k_chain<__half>), smem);
    if (e == cudaSuccess) k_chain<__half><<<grid, kThreads, smem, s>>>(p);
  } else {
    e = set_smem_once(reinterpret_cast<const void*>(k_chain<__nv_bfloat16>), smem);
    if (e == cudaSuccess) k_chain<__nv_bfloat16><<<grid, kThreads, smem, s>>>(p);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// ------------------------------------------------------------------ launch helpers
template <typename T>
using GenKernel = void (*)(const GenParams);

template <typename T>
GenKernel<T> pick_stream(int rm, int rn) {
#define TNC_CASE(a, b) \
  if (rm == a && rn == b) return k_stream<T, a, b>;
  TNC_CASE(1, 1) TNC_CASE(1, 2) TNC_CASE(1, 4) TNC_CASE(2, 1) TNC_CASE(2, 2) TNC_CASE(2, 4)
  TNC_CASE(4, 1) TNC_CASE(4, 2) TNC_CASE(4, 4)
#undef TNC_CASE
  return nullptr;
}

template <typename T>
GenKernel<T> pick_generic(int rm, int rn) {
#define TNC_CASE(a, b) \
  if (rm == a && rn == b) return k_generic<T, a, b>;
  TNC_CASE(1, 1) TNC_CASE(1, 2) TNC_CASE(1, 4) TNC_CASE(2, 1) TNC_CASE(2, 2) TNC_CASE(2, 4)
  TNC_CASE(4, 1) TNC_CASE(4, 2) TNC_CASE(4, 4) TNC_CASE(8, 4)
#undef TNC_CASE
  return nullptr;
}

cudaError_t launch_generic(int precision, int rm, int rn, const GenParams& p, dim3 grid, size_t smem, cudaStream_t s) {
  void (*k)(const GenParams) = nullptr;
  if (p.stream) {
    if (precision == 0) k = pick_stream<float>(rm, rn);
    else if (precision == 1) k = pick_stream<__half>(rm, rn);
    else k = pick_stream<__nv_bfloat16>(rm, rn);
  } else if (precision == 0) k = pick_generic<float>(rm, rn);
  else if (precision == 1) k = pick_generic<__half>(rm, rn);
  else k = pick_generic<__nv_bfloat16>(rm, rn);
  if (!k) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = set_smem_once(reinterpret_cast<const void*>(k), smem);
    if (e != cudaSuccess) return e;
  }
  if (!p.stream) {
    // k_generic strides over its outer tiles: about 32 CTAs per SM over the grid's
    // (split, instance) columns, so each CTA builds its index tables once for many tiles
    const unsigned cols = grid.y * grid.z;
    const unsigned cap = std::max(1u, (152u * 32u + cols - 1) / cols);
    grid.x = std::min(grid.x, cap);
  }
  k<<<grid, kThreads, smem, s>>>(p);
  return cudaGetLastError();
}

// The persistent steps kernel: one cooperative launch (every CTA resident, as the grid
// barrier needs) of as many CTAs as fit on the device at `smem` bytes each.
cudaError_t launch_steps(int precision, const StepOp* ops, const int32_t* phases, int n_phases, int64_t n_inst,
                         int reuse, uint32_t* bar, int32_t* status, size_t smem, cudaStream_t s) {
  const void* k = precision == 0 ? reinterpret_cast<const void*>(k_steps<float>)
                  : precision == 1 ? reinterpret_cast<const void*>(k_steps<__half>)
                                   : reinterpret_cast<const void*>(k_steps<__nv_bfloat16>);
  // always opt in: the kernel's static shared memory (the op's parameters) comes on top
  if (smem > 0) {
    cudaError_t e = set_smem_once(k, smem);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, n_sm = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1 || n_sm < 1) return cudaErrorInvalidConfiguration;
  void* args[] = {&ops, &phases, &n_phases, &n_inst, &reuse, &bar, &status};
  return cudaLaunchCooperativeKernel(k, dim3((unsigned)(per_sm * n_sm)), dim3(kThreads), args, smem, s);
}

cudaError_t launch_splitk_reduce(int precision, const GenParams& p, int64_t n_inst, cudaStream_t s) {
  if (p.splitk >= kWideReduceSplit) {
    constexpr int OPB = kThreads / 32;  // outputs per block
    dim3 grid((unsigned)((p.planeC + OPB - 1) / OPB), 1, (unsigned)n_inst);
    if (precision == 0) k_splitk_reduce_wide<float><<<grid, kThreads, 0, s>>>(p);
    else if (precision == 1) k_splitk_reduce_wide<__half><<<grid, kThreads, 0, s>>>(p);
    else k_splitk_reduce_wide<__nv_bfloat16><<<grid, kThreads, 0, s>>>(p);
    return cudaGetLastError();
  }
  dim3 grid((unsigned)((p.planeC + kThreads - 1) / kThreads), 1, (unsigned)n_inst);
  if (precision == 0) k_splitk_reduce<float><<<grid, kThreads, 0, s>>>(p);
  else if (precision == 1) k_splitk_reduce<__half><<<grid, kThreads, 0, s>>>(p);
  else k_splitk_reduce<__nv_bfloat16><<<grid, kThreads, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_leaf_gather(int precision, const LeafDesc* leaves, int n_leaves, const double2* src, void* arena,
                               int64_t inst_stride, const int64_t* inst_slice, const int32_t* inst_row,
                               const uint8_t* bits, int n_qubits, float* maxabs, int32_t* exps, int n_slots,
                               int64_t inst_base, int64_t n_inst, double2* leaf_r, cudaStream_t s) {
  dim3 grid((unsigned)n_leaves, (unsigned)n_inst);
  if (precision == 0)
    k_leaf_gather<float><<<grid, 32, 0, s>>>(leaves, src, (float*)arena, inst_stride, inst_slice, inst_row, bits,
                                             n_qubits, maxabs, exps, n_slots, inst_base, leaf_r, n_leaves);
  else if (precision == 1)
    k_leaf_gather<__half><<<grid, 32, 0, s>>>(leaves, src, (__half*)arena, inst_stride, inst_slice, inst_row, bits,
                                              n_qubits, maxabs, exps, n_slots, inst_base, leaf_r, n_leaves);
  else
    k_leaf_gather<__nv_bfloat16><<<grid, 32, 0, s>>>(leaves, src, (__nv_bfloat16*)arena, inst_stride, inst_slice,
                                                     inst_row, bits, n_qubits, maxabs, exps, n_slots, inst_base, leaf_r,
                                                     n_leaves);
  return cudaGetLastError();
}

cudaError_t launch_root_accum(int precision, const void* arena, int64_t inst_stride, int64_t root_off, int64_t plane,
                              const int8_t* open_pos, int n_open, const RootSeg* segs, int n_segs,
                              const int32_t* exps, int n_slots, int root_slot, double2* acc, const double2* cfac,
                              InstMap rm, cudaStream_t s, uint32_t merged) {
  const int64_t n_out = int64_t(1) << n_open;
  dim3 grid((unsigned)((n_out + 255) / 256), (unsigned)n_segs);
  if (precision == 0)
    k_root_accum<float><<<grid, 256, 0, s>>>((const float*)arena, inst_stride, root_off, plane, open_pos, n_open, segs,
                                             exps, n_slots, root_slot, acc, cfac, rm, merged);
  else if (precision == 1)
    k_root_accum<__half><<<grid, 256, 0, s>>>((const __half*)arena, inst_stride, root_off, plane, open_pos, n_open,
                                              segs, exps, n_slots, root_slot, acc, cfac, rm, merged);
  else
    k_root_accum<__nv_bfloat16><<<grid, 256, 0, s>>>((const __nv_bfloat16*)arena, inst_stride, root_off, plane,
                                                     open_pos, n_open, segs, exps, n_slots, root_slot, acc, cfac, rm, merged);
  return cudaGetLastError();
}

cudaError_t launch_maxabs(int precision, const void* x, int64_t n, float* out, cudaStream_t s) {
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  if (blocks < 1) blocks = 1;
  if (precision == 0) k_maxabs<float><<<blocks, 256, 0, s>>>((const float*)x, n, out);
  else if (precision == 1) k_maxabs<__half><<<blocks, 256, 0, s>>>((const __half*)x, n, out);
  else k_maxabs<__nv_bfloat16><<<blocks, 256, 0, s>>>((const __nv_bfloat16*)x, n, out);
  return cudaGetLastError();
}

}  // namespace tnc
