// Device executor: contexts, per-plan device programs, and the amplitude / contraction
// entry points of the C boundary.
//
// An *instance* is one full contraction of the plan for one bitstring row and one
// slice id (Sec. III-A: a subtask).  Instances run in waves: every kernel of the step
// program covers all instances of a wave in one launch (grid.z), and the per-wave
// root tensors are added into an FP64 accumulator in a fixed order.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "capi_internal.h"
#include "device.cuh"
#include <cudaTypedefs.h>

namespace tnc {

cudaError_t launch_generic(int precision, int rm, int rn, const GenParams& p, dim3 grid, size_t smem, cudaStream_t s);
cudaError_t launch_splitk_reduce(int precision, const GenParams& p, int64_t n_inst, cudaStream_t s);
cudaError_t launch_steps(int precision, const StepOp* ops, const int32_t* phases, int n_phases, int64_t n_inst,
                         int reuse, uint32_t* bar, int32_t* status, size_t smem, cudaStream_t s);
cudaError_t launch_leaf_gather(int precision, const LeafDesc* leaves, int n_leaves, const double2* src, void* arena,
                               int64_t inst_stride, const int64_t* inst_slice, const int32_t* inst_row,
                               const uint8_t* bits, int n_qubits, float* maxabs, int32_t* exps, int n_slots,
                               int64_t inst_base, int64_t n_inst, double2* leaf_r, cudaStream_t s);
cudaError_t launch_root_accum(int precision, const void* arena, int64_t inst_stride, int64_t root_off, int64_t plane,
                              const int8_t* open_pos, int n_open, const RootSeg* segs, int n_segs,
                              const int32_t* exps, int n_slots, int root_slot, double2* acc, const double2* cfac,
                              InstMap rm, cudaStream_t s, uint32_t merged = 0);
cudaError_t launch_merge(int precision, void* arena, int64_t inst_stride, int64_t off, int64_t plane, int32_t* exps,
                         float* maxabs, int n_slots, int slot, const double2* leaf_r, int n_leaves, int lu, int lv,
                         int bit, InstMap im, int64_t nz, cudaStream_t s);
cudaError_t launch_inst_scale(const double2* leaf_r, int n_leaves, int64_t n_inst, double2* c, cudaStream_t s);
cudaError_t launch_maxabs(int precision, const void* x, int64_t n, float* out, cudaStream_t s);
cudaError_t launch_adj_root_init(float* arena, int64_t inst_stride, int64_t root_off, int64_t plane,
                                 const int8_t* open_pos, int n_open, const int32_t* inst_row, int64_t inst_base,
                                 int64_t n_inst, const double2* w, const int32_t* erow, float* maxabs, int32_t* exps,
                                 int n_slots, int slot, cudaStream_t s);
cudaError_t launch_tc_gemm(int precision, const TcParams& p, dim3 grid, cudaStream_t s);
cudaError_t launch_tc_tma(int precision, const TcParams& p, dim3 grid, cudaStream_t s);
cudaError_t launch_chain(int precision, const ChainParams& p, int64_t n_inst, cudaStream_t s);
cudaError_t launch_permute(int precision, const PermParams& p, cudaStream_t s);
TileSpec tile_for(const std::vector<int>& la, const std::vector<int>& lb, const std::vector<int>& lc, int n_inst,
                  int& kind);
bool tc_tile_for(const std::vector<int>& la, const std::vector<int>& lb, const std::vector<int>& lc, TileSpec& t,
                 bool& swap, int& bn, int& bk);

#define CUDA_OK(expr)                                                                             \
  do {                                                                                            \
    cudaError_t _e = (expr);                                                                      \
    if (_e != cudaSuccess) fail(TNC_E_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)

static size_t elem_bytes(int precision) { return precision == TNC_C64 ? 4 : 2; }

// ------------------------------------------------------------------ device buffers
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  void reserve(size_t n) {
    if (n <= bytes) return;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      fail(TNC_E_OOM, "device allocation of " + std::to_string(n) + " bytes failed: " + cudaGetErrorString(e));
    }
    bytes = n;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <class T>
  T* as() const {
    return reinterpret_cast<T*>(p);
  }
};

// ------------------------------------------------------------------ GenParams from a tile
static int pos_of(const std::vector<int>& l, int x) {
  for (size_t i = 0; i < l.size(); ++i)
    if (l[i] == x) return (int)i;
  fail(TNC_E_PLAN, "label missing from operand layout");
}

static int rank_in_mask(uint32_t mask, int pos) { return __builtin_popcount(mask & ((1u << pos) - 1u)); }

static int low_run(uint32_t mask) {
  int r = 0;
  while (r < 32 && ((mask >> r) & 1u)) ++r;
  return r;
}

struct StepLaunch {
  int kind;  // K_GENERIC, K_SPLITK, K_TC, K_TMA or K_CHAIN
  GenParams p;
  TcParams tp;
  ChainParams cp;
  dim3 grid;
  size_t smem;
  int rm, rn;
  double flops = 0, bytes = 0;  // algorithmic, per instance (real flops 8MNK; bytes read + written)
  int plan_step = -1;           // the plan step a tensor-core launch runs
  bool stream = false;          // a SIMT step that may stream its tiles (see make_stream)
  // post-lifetime merges run after the step (tree-like reuse only): sum the result over the
  // two values of each sliced index whose edge this step contracts (see k_merge)
  struct MergeOp {
    int bit, lu, lv, slot;
    int64_t off, plane;
    InstMap im;  // launch index -> the t = 0 instance (the result's dependence without t)
    void* arena;
    int64_t inst_stride;
    int32_t* exps;
    float* maxabs;
    int n_slots, n_leaves;
    const double2* leaf_r;
  };
  std::vector<MergeOp> merges;
};

// Tensor-core launch of a step whose tile satisfies choose_tc_tile's rules.  la / lb are the
// kernel's A (row side) and B operands (already swapped when the tile asked for it).
// n_inst sizes the split over the outer common labels: enough CTAs for two waves.
// Instances assumed when a step's split over K is sized: every slice of the plan for one
// bitstring row (the unit of work of a full-plan call), at most 2^12, and at most the largest
// power of two of instances whose arenas fit in 60% of the device's total memory (bytes_per_inst
// each).  Neither the wave size a call picks nor the free memory enters, so a plan's results do
// not depend on how many instances share a launch.
static int64_t split_instances(const Plan& P, double bytes_per_inst, double total_mem) {
  const int64_t all = int64_t(1) << std::min<size_t>(P.sliced.size(), 12);
  const double fit = std::max(1.0, 0.6 * total_mem / std::max(1.0, bytes_per_inst));
  int64_t cap = 1;
  while (cap * 2 <= all && double(cap * 2) <= fit) cap *= 2;
  return std::min(all, cap);
}

static void make_tc_launch(StepLaunch& L, const TileSpec& t, const std::vector<int>& la, const std::vector<int>& lb,
                           const std::vector<int>& lc, int precision, int bn, int bk, int64_t n_inst,
                           int force_split = 0) {
  TcParams& q = L.tp;
  std::memset(&q, 0, sizeof(q));
  const size_t nt = bn == 256 ? 8 : (bn == 128 ? 7 : (bn == 64 ? 6 : 5)), kt = bk == 32 ? 5 : 4;
  if (t.Mt.size() != 7 || t.Nt.size() != nt || t.Kt.size() != kt) fail(TNC_E_PLAN, "bad tensor-core tile");
  for (int j = 0; j < 3; ++j)
    if (pos_of(la, t.Kt[j]) != j || pos_of(lb, t.Kt[j]) != j) fail(TNC_E_PLAN, "tensor-core operands not K-major");
  uint32_t maskC = 0;
  for (int x : t.Mt) maskC |= 1u << pos_of(lc, x);
  for (int x : t.Nt) maskC |= 1u << pos_of(lc, x);
  q.bn = bn;
  q.bk = bk;
  q.maskC = maskC;
  q.runC = low_run(maskC);
  if (q.runC < 3) fail(TNC_E_PLAN, "tensor-core output run too short");
  // direct epilogue: tile columns 0..2 at C positions 0..2 (runs of 8 per thread) and row 0
  // at position 3, so lanes write whole 32-byte sectors (scattered 16-byte halves of sectors
  // measured slower than staging)
  q.direct = (pos_of(lc, t.Nt[0]) == 0 && pos_of(lc, t.Nt[1]) == 1 && pos_of(lc, t.Nt[2]) == 2 &&
              pos_of(lc, t.Mt[0]) == 3) ? 1 : 0;
  for (int j = 0; j < 7; ++j) {
    q.pAm[j] = (int8_t)pos_of(la, t.Mt[j]);
    q.pCm[j] = (int8_t)rank_in_mask(maskC, pos_of(lc, t.Mt[j]));
  }
  for (size_t j = 0; j < nt; ++j) {
    q.pBn[j] = (int8_t)pos_of(lb, t.Nt[j]);
    q.pCn[j] = (int8_t)rank_in_mask(maskC, pos_of(lc, t.Nt[j]));
  }
  for (size_t j = 3; j < kt; ++j) {
    q.pAk[j - 3] = (int8_t)pos_of(la, t.Kt[j]);
    q.pBk[j - 3] = (int8_t)pos_of(lb, t.Kt[j]);
  }
  q.n_om = (int)t.Mo.size();
  q.n_on = (int)t.No.size();
  q.n_ok = (int)t.Ko.size();
  if (q.n_om > kMaxOuter || q.n_on > kMaxOuter || q.n_ok > kMaxOuter) fail(TNC_E_UNSUPPORTED, "too many outer labels");
  for (int j = 0; j < q.n_om; ++j) q.om_A[j] = (int8_t)pos_of(la, t.Mo[j]), q.om_C[j] = (int8_t)pos_of(lc, t.Mo[j]);
  for (int j = 0; j < q.n_on; ++j) q.on_B[j] = (int8_t)pos_of(lb, t.No[j]), q.on_C[j] = (int8_t)pos_of(lc, t.No[j]);
  for (int j = 0; j < q.n_ok; ++j) q.ok_A[j] = (int8_t)pos_of(la, t.Ko[j]), q.ok_B[j] = (int8_t)pos_of(lb, t.Ko[j]);
  q.planeA = int64_t(1) << la.size();
  q.planeB = int64_t(1) << lb.size();
  q.planeC = int64_t(1) << lc.size();
  q.nK = (int)t.Kt.size() + q.n_ok;
  q.bf16 = precision == TNC_CBF16 ? 1 : 0;
  const int64_t tiles = (int64_t(1) << (q.n_om + q.n_on)) * std::max<int64_t>(1, n_inst);
  const int64_t kit = int64_t(1) << q.n_ok;  // K tiles per output tile
  // persistent TMA kernels overlap each tile's epilogue with the next tile's loads and MMAs:
  // short K loops over many tiles (two TMEM accumulators: BN <= 128), and 256-wide tiles
  // with the direct epilogue whenever every SM gets two tiles or more and a tile's K loop is
  // at most 256 K tiles (longer loops hide their epilogue, and the hardware's dynamic CTA
  // scheduling balances long tiles better than a fixed tile order)
  q.persistent = ((bn >= 64 && bn <= 128 && q.n_ok <= 3 && tiles >= 4 * 152) ||
                  (bn == 256 && q.direct && tiles >= 2 * 152 && q.n_ok <= 8)) ? 1 : 0;
  // otherwise split over the outer common labels: at least two CTAs per SM (every split
  // keeping at least 4 K tiles), and whole waves (the last one at least 90% busy) when each
  // split keeps at least 256 K tiles, so the FP32 partial sums cost little
  auto wave_eff = [](int64_t ctas) {
    const double w = double(ctas) / 152.0;
    return w / std::ceil(w);
  };
  int split = 1;
  if (force_split > 0) {
    // a tuned split (1 <= split <= K tiles; the caller decides about the persistent kernel)
    if (force_split > kit || (force_split & (force_split - 1))) fail(TNC_E_PLAN, "bad tensor-core split");
    q.persistent = 0;
    split = force_split;
  } else if (!q.persistent)
    while (kit / (split * 2) >= 4 && split < 1024 &&
           (tiles * split < 2 * 152 || (wave_eff(tiles * split) < 0.9 && kit / (split * 2) >= 256)))
      split *= 2;
  q.splitk = split;
  // short K loops: a 3-stage pipeline leaves room for two CTAs per SM
  q.stages = (kit / split) <= 3 ? 3 : 0;
  L.kind = K_TC;
  L.grid = dim3(1u << (q.n_om + q.n_on), (unsigned)split, 1);
  L.smem = 0;
  // the fixed-order reduction of the partials reuses the SIMT split-K reduce kernel
  std::memset(&L.p, 0, sizeof(L.p));
  L.p.planeC = q.planeC;
  L.p.splitk = split;
  L.p.nK = q.nK;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    CUDA_OK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !ptr) fail(TNC_E_UNSUPPORTED, "cuTensorMapEncodeTiled is not available");
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }
  return fn;
}

// 4-D view of a planar 16-bit tensor laid out [Kt (2^kt entries) | rows ...]:
// (k, row, plane, instance) with a box of 2^kt x box_rows x 1 x 1, swizzled to match the
// K-major shared-memory layout of the MMA (32B swizzle for 32-byte rows, 64B for 64-byte).
// FP32 entries (the complex64 3xTF32 kernel) take 16 entries (64 bytes) per box row: a
// 16-entry K run is the 4-D view with a 64B swizzle; a 32-entry run is the 5-D view
// (k low 16, k high bit, row, plane, instance) whose box takes one half.
static void encode_tile_map(CUtensorMap* m, const void* base, int rank, int kt, int box_rows, int64_t inst_stride,
                            int64_t n_inst, size_t eb = 2) {
  if ((int64_t(1) << (rank - kt)) < box_rows || rank > 32) fail(TNC_E_PLAN, "tensor map: operand rank out of range");
  if ((reinterpret_cast<uintptr_t>(base) & 15u) != 0) fail(TNC_E_PLAN, "tensor map: base not 16-byte aligned");
  const int64_t plane = int64_t(1) << rank;
  const int64_t istr = std::max<int64_t>(inst_stride, 2 * plane);
  const cuuint64_t ni = (cuuint64_t)std::max<int64_t>(1, n_inst);
  CUresult r;
  if (eb == 2) {
    cuuint64_t dims[4] = {cuuint64_t(1) << kt, cuuint64_t(1) << (rank - kt), 2, ni};
    cuuint64_t strides[3] = {(cuuint64_t(1) << kt) * 2, (cuuint64_t)plane * 2, (cuuint64_t)istr * 2};
    cuuint32_t box[4] = {1u << kt, (cuuint32_t)box_rows, 1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUtensorMapSwizzle sw = kt == 5 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B;
    r = tensor_map_encoder()(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 4, const_cast<void*>(base), dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else if (kt == 4) {
    cuuint64_t dims[4] = {16, cuuint64_t(1) << (rank - 4), 2, ni};
    cuuint64_t strides[3] = {16 * 4, (cuuint64_t)plane * 4, (cuuint64_t)istr * 4};
    cuuint32_t box[4] = {16, (cuuint32_t)box_rows, 1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    r = tensor_map_encoder()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(base), dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    cuuint64_t dims[5] = {16, 2, cuuint64_t(1) << (rank - 5), 2, ni};
    cuuint64_t strides[4] = {16 * 4, 32 * 4, (cuuint64_t)plane * 4, (cuuint64_t)istr * 4};
    cuuint32_t box[5] = {16, 1, (cuuint32_t)box_rows, 1, 1};
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    r = tensor_map_encoder()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<void*>(base), dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  if (r != CUDA_SUCCESS) fail(TNC_E_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
}

// Operands already laid out for the TMA kernel: A leads with Kt then 7 of its free labels, B
// with Kt then 6 or 7 of its free labels, and C's lowest three labels are tile labels.
static bool tma_tile_from_layout(const std::vector<int>& la, const std::vector<int>& lb, const std::vector<int>& lc,
                                 TileSpec& t, int& bn, int& bk) {
  std::vector<int> K, M, N;
  for (int x : la) (std::find(lb.begin(), lb.end(), x) != lb.end() ? K : M).push_back(x);
  for (int x : lb)
    if (std::find(la.begin(), la.end(), x) == la.end()) N.push_back(x);
  if (M.size() < 7 || N.size() < 5 || K.size() < 4) return false;
  bk = K.size() >= 5 ? 32 : 16;
  // 256-wide tiles (all of TMEM, one CTA per SM) only for K loops of more than 8 K tiles;
  // shorter loops take 128-wide tiles and the persistent kernel; 32 columns when N = 2^5
  bn = (N.size() >= 8 && K.size() > size_t(bk == 32 ? 8 : 7)) ? 256
       : (N.size() >= 7 ? 128 : (N.size() >= 6 ? 64 : 32));
  const size_t kt = bk == 32 ? 5 : 4, nt = bn == 256 ? 8 : (bn == 128 ? 7 : (bn == 64 ? 6 : 5));
  if (la.size() < kt + 7 || lb.size() < kt + nt || lc.size() < 3) return false;
  auto in = [](const std::vector<int>& v, int x) { return std::find(v.begin(), v.end(), x) != v.end(); };
  t = TileSpec();
  for (size_t j = 0; j < kt; ++j) {
    if (la[j] != lb[j] || !in(K, la[j])) return false;
    t.Kt.push_back(la[j]);
  }
  for (size_t j = 0; j < 7; ++j) {
    if (!in(M, la[kt + j])) return false;
    t.Mt.push_back(la[kt + j]);
  }
  for (size_t j = 0; j < nt; ++j) {
    if (!in(N, lb[kt + j])) return false;
    t.Nt.push_back(lb[kt + j]);
  }
  for (int j = 0; j < 3; ++j)
    if (!in(t.Mt, lc[j]) && !in(t.Nt, lc[j])) return false;
  for (int x : M)
    if (!in(t.Mt, x)) t.Mo.push_back(x);
  for (int x : N)
    if (!in(t.Nt, x)) t.No.push_back(x);
  for (int x : K)
    if (!in(t.Kt, x)) t.Ko.push_back(x);
  return t.Mo.size() + t.No.size() <= 30 && t.Ko.size() <= 24;
}

// Permutation from layout `lin` to layout `lout` (same label set): the tile holds the six
// lowest positions of each layout, widened with further input positions up to 12 labels.
static PermParams make_permute(const std::vector<int>& lin, const std::vector<int>& lout) {
  PermParams q;
  std::memset(&q, 0, sizeof(q));
  const int r = (int)lin.size();
  std::vector<int> T;
  auto add = [&](int x) {
    if (std::find(T.begin(), T.end(), x) == T.end()) T.push_back(x);
  };
  for (int j = 0; j < std::min(r, 6); ++j) add(lin[j]);
  for (int j = 0; j < std::min(r, 6); ++j) add(lout[j]);
  for (int j = 6; j < r && T.size() < 12; ++j) add(lin[j]);
  for (int x : T) q.mask_in |= 1u << pos_of(lin, x), q.mask_out |= 1u << pos_of(lout, x);
  q.bits = (int)T.size();
  q.run_in = low_run(q.mask_in);
  q.run_out = low_run(q.mask_out);
  // tile-native orders: bit i of a tile index is the i-th lowest tile position of the layout
  std::vector<int> tin = T, tout = T;
  std::sort(tin.begin(), tin.end(), [&](int x, int y) { return pos_of(lin, x) < pos_of(lin, y); });
  std::sort(tout.begin(), tout.end(), [&](int x, int y) { return pos_of(lout, x) < pos_of(lout, y); });
  auto scatter = [&](uint32_t v, int shift) {
    uint32_t t = 0;
    for (int j = 0; j < 6 && j + shift < q.bits; ++j)
      if ((v >> j) & 1u) t |= 1u << pos_of(tin, tout[j + shift]);
    return (uint16_t)t;
  };
  for (uint32_t v = 0; v < 64; ++v) {
    q.plo[v] = scatter(v, 0);
    q.phi[v] = scatter(v, 6);
  }
  for (int x : lin)
    if (std::find(T.begin(), T.end(), x) == T.end()) {
      if (q.n_o >= kMaxOuter) fail(TNC_E_UNSUPPORTED, "permutation: too many outer labels");
      q.o_in[q.n_o] = (int8_t)pos_of(lin, x);
      q.o_out[q.n_o] = (int8_t)pos_of(lout, x);
      ++q.n_o;
    }
  q.plane = int64_t(1) << r;
  return q;
}

// TTGT layouts for a single contraction whose operands the tensor-core kernels cannot load
// in place: A' = [Kt | Mt | other M | other K], B' = [Kt | Nt | other N | other K] (the
// layouts the compiler gives tensor-core steps) and C' = [3 of Nt | Mt | ...].  False when the
// step is too small for tensor-core tiles.
static bool ttgt_layouts(const std::vector<int>& la, const std::vector<int>& lb, std::vector<int>& la2,
                         std::vector<int>& lb2, std::vector<int>& lc2) {
  std::vector<int> K, M, N;
  for (int x : la) (std::find(lb.begin(), lb.end(), x) != lb.end() ? K : M).push_back(x);
  for (int x : lb)
    if (std::find(la.begin(), la.end(), x) == la.end()) N.push_back(x);
  if (M.size() < N.size()) return false;  // the caller swaps the operands first
  if (M.size() < 7 || N.size() < 6 || K.size() < 4) return false;
  const size_t kt = K.size() >= 5 ? 5 : 4;
  const size_t nt = (N.size() >= 8 && K.size() > kt + 3) ? 8 : (N.size() >= 7 ? 7 : 6);
  la2.assign(K.begin(), K.begin() + kt);
  la2.insert(la2.end(), M.begin(), M.end());
  la2.insert(la2.end(), K.begin() + kt, K.end());
  lb2.assign(K.begin(), K.begin() + kt);
  lb2.insert(lb2.end(), N.begin(), N.end());
  lb2.insert(lb2.end(), K.begin() + kt, K.end());
  // C' leads with three tile columns, then the tile rows: each thread stores runs of 8
  // columns straight from registers (the direct epilogue) and the 32 rows of a warp are
  // adjacent, so one warp store covers a contiguous 512-byte block
  lc2.assign(N.begin(), N.begin() + 3);
  lc2.insert(lc2.end(), M.begin(), M.begin() + 7);
  lc2.insert(lc2.end(), N.begin() + 3, N.end());
  lc2.insert(lc2.end(), M.begin() + 7, M.end());
  return true;
}

// TTGT scratch (A', B', C') must fit in half of the free device memory.
static bool ttgt_fits(size_t ra, size_t rb, size_t rc, size_t eb) {
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return false;
  const double need = (std::ldexp(1.0, (int)ra) + std::ldexp(1.0, (int)rb) + std::ldexp(1.0, (int)rc)) * 2.0 * double(eb);
  return need <= 0.5 * double(free_b);
}

// Fills the pointers of a tensor-core launch (and of its reduce, when split).
static void bind_tc(StepLaunch& L, const void* a, const void* b, void* c, int64_t stride, float* maxabs, int32_t* exps,
                    int n_slots, int slot_a, int slot_b, int slot_c, int32_t* status, float2* partials) {
  TcParams& q = L.tp;
  q.A = a;
  q.B = b;
  q.C = c;
  q.strideA = q.strideB = q.strideC = stride;
  q.maxabs = maxabs;
  q.exps = exps;
  q.n_slots = n_slots;
  q.slotA = slot_a;
  q.slotB = slot_b;
  q.slotC = slot_c;
  q.status = status;
  q.partials = partials;
  GenParams& r = L.p;
  r.C = c;
  r.strideC = stride;
  r.maxabs = maxabs;
  r.exps = exps;
  r.n_slots = n_slots;
  r.slotA = slot_a;
  r.slotB = slot_b;
  r.slotC = slot_c;
  r.partials = partials;
}

static StepLaunch make_launch(const TileSpec& t, int kind, const std::vector<int>& la, const std::vector<int>& lb,
                              const std::vector<int>& lc) {
  StepLaunch L;
  std::memset(&L.p, 0, sizeof(L.p));
  GenParams& p = L.p;
  if (t.Mt.size() > (size_t)kMaxTileBits || t.Nt.size() > (size_t)kMaxTileBits || t.Kt.size() > (size_t)kMaxTileBits ||
      t.Mo.size() > (size_t)kMaxOuter || t.No.size() > (size_t)kMaxOuter || t.Ko.size() > (size_t)kMaxOuter)
    fail(TNC_E_UNSUPPORTED, "tile exceeds kernel limits");
  if (la.size() > 32 || lb.size() > 32 || lc.size() > 32) fail(TNC_E_UNSUPPORTED, "rank above 32");
  p.mt = (int)t.Mt.size();
  p.nt = (int)t.Nt.size();
  p.kt = (int)t.Kt.size();
  for (int x : t.Mt) p.maskA |= 1u << pos_of(la, x), p.maskC |= 1u << pos_of(lc, x);
  for (int x : t.Kt) p.maskA |= 1u << pos_of(la, x), p.maskB |= 1u << pos_of(lb, x);
  for (int x : t.Nt) p.maskB |= 1u << pos_of(lb, x), p.maskC |= 1u << pos_of(lc, x);
  p.runA = low_run(p.maskA);
  p.runB = low_run(p.maskB);
  p.runC = low_run(p.maskC);
  for (int j = 0; j < p.mt; ++j) {
    p.pAm[j] = (int8_t)rank_in_mask(p.maskA, pos_of(la, t.Mt[j]));
    p.pCm[j] = (int8_t)rank_in_mask(p.maskC, pos_of(lc, t.Mt[j]));
  }
  for (int j = 0; j < p.kt; ++j) {
    p.pAk[j] = (int8_t)rank_in_mask(p.maskA, pos_of(la, t.Kt[j]));
    p.pBk[j] = (int8_t)rank_in_mask(p.maskB, pos_of(lb, t.Kt[j]));
  }
  for (int j = 0; j < p.nt; ++j) {
    p.pBn[j] = (int8_t)rank_in_mask(p.maskB, pos_of(lb, t.Nt[j]));
    p.pCn[j] = (int8_t)rank_in_mask(p.maskC, pos_of(lc, t.Nt[j]));
  }
  p.n_om = (int)t.Mo.size();
  p.n_on = (int)t.No.size();
  p.n_ok = (int)t.Ko.size();
  for (int j = 0; j < p.n_om; ++j) p.om_A[j] = (int8_t)pos_of(la, t.Mo[j]), p.om_C[j] = (int8_t)pos_of(lc, t.Mo[j]);
  for (int j = 0; j < p.n_on; ++j) p.on_B[j] = (int8_t)pos_of(lb, t.No[j]), p.on_C[j] = (int8_t)pos_of(lc, t.No[j]);
  for (int j = 0; j < p.n_ok; ++j) p.ok_A[j] = (int8_t)pos_of(la, t.Ko[j]), p.ok_B[j] = (int8_t)pos_of(lb, t.Ko[j]);
  p.planeA = int64_t(1) << la.size();
  p.planeB = int64_t(1) << lb.size();
  p.planeC = int64_t(1) << lc.size();
  p.splitk = t.splitk;
  p.kgroups = t.kgroups;
  p.nK = p.kt + p.n_ok;
  if (p.n_om + p.n_on > 30) fail(TNC_E_UNSUPPORTED, "too many outer tiles");
  // shared memory: operand tiles / reduction buffer, then index tables
  const size_t ab = ((size_t(1) << (p.mt + p.kt)) + (size_t(1) << (p.kt + p.nt))) * 8;
  const size_t rb = size_t(t.kgroups) * (size_t(1) << (p.mt + p.nt)) * 8;
  size_t region = std::max(ab, rb);
  region = (region + 15) & ~size_t(15);
  p.smem_tables = (int32_t)region;
  size_t tables = ((size_t(1) << (p.mt + p.kt - p.runA)) + (size_t(1) << (p.kt + p.nt - p.runB)) +
                   (size_t(1) << (p.mt + p.nt - p.runC))) * 4 +
                  ((size_t(2) << p.mt) + (size_t(2) << p.kt) + (size_t(2) << p.nt) + 2) * 2 + 32 * 4;
  L.smem = region + tables;
  if (L.smem > 200 * 1024) fail(TNC_E_UNSUPPORTED, "tile needs too much shared memory");
  L.grid = dim3(1u << (p.n_om + p.n_on), (unsigned)t.splitk, 1);
  L.kind = kind;
  L.rm = t.rm;
  L.rn = t.rn;
  L.stream = t.stream;
  return L;
}

// Memory-bound long-K steps (GEPDOTs, thin operands) with runs of at least 16 bytes in both
// operands and two or more K steps per CTA stream their raw tiles through the k_stream ring
// (elements of eb bytes).
//
// When both operands lead with the same K tile labels (K tile bits 0..c-1 at tile positions
// 0..c-1 of A and of B, 2^c entries = 8 bytes), each K group takes k in chunks of 2^c: a
// chunk of one tile row is one 8-byte shared-memory load in k_stream.  k_generic visits k
// in the same order (the chunk order is set whether or not the step streams), so the two
// kernels stay bit-identical.
static void make_stream(StepLaunch& L, size_t eb, bool disabled) {
  GenParams& p = L.p;
  p.kvb = 0;
  if (L.stream) {
    const int c = eb == 2 ? 2 : 1;
    bool lead = p.kt >= c;
    for (int v = 0; lead && v < c; ++v) lead = p.pAk[v] == v && p.pBk[v] == v;
    if (lead) {
      p.kvb = c;
      p.kgroups = std::max(1, std::min(p.kgroups, (1 << p.kt) >> c));
    }
  }
  if (disabled || !L.stream) return;
  const int need = eb == 2 ? 3 : 2;  // log2 entries per 16 bytes
  if (p.runA < need || p.runB < need) return;
  if (((int64_t(1) << p.n_ok) / p.splitk) < 2) return;
  const size_t stage = 2 * ((size_t(1) << (p.mt + p.kt)) + (size_t(1) << (p.kt + p.nt))) * eb;
  const size_t rb = size_t(p.kgroups) * (size_t(1) << (p.mt + p.nt)) * 8;
  size_t region = std::max(size_t(kStreamStages) * stage, rb);
  region = (region + 15) & ~size_t(15);
  const size_t tables = L.smem - size_t(p.smem_tables);
  if (region + tables > 220 * 1024) return;  // within the 227 KB a CTA may take
  p.stream = 1;
  p.smem_tables = (int32_t)region;
  L.smem = region + tables;
}

// ------------------------------------------------------------------ per-plan device program
struct DeviceProgram {
  int device = 0, precision = 0, W = 0;
  bool fused = false;       // chains fused: tensors at their fused-arena offsets
  int64_t split_inst = 1;   // instances the tensor-core splits over K are sized for
  int64_t inst_stride = 0;  // scalars
  int n_slots = 0, n_leaves = 0;
  DevBuf arena, maxabs, exps, leaf_src, leaf_desc, partials, open_pos, chain_links;
  DevBuf leaf_r, inst_c;  // per (instance, leaf) rounding scale and per-instance product
  InstMap root_map{-1, 0, 0, 0};  // instance holding each slice's root (tree-like reuse)
  bool reuse_ok = false;          // the step maps above are set (waves of whole rows)
  bool merge = false;             // post-lifetime merging requested for this program
  uint32_t merged_mask = 0;       // slice bits summed by merges (the root sum skips them)
  std::vector<StepLaunch> steps;
  int root = 0;
  int64_t root_off = 0, root_plane = 1;
  int n_open = 0;
  int n_qubits = 0;
  uint64_t leaf_version = 0;
  std::vector<int64_t> leaf_dst;  // arena offsets of the reduced leaves in this program
  // CUDA graphs of one wave, keyed by the wave's launch parameters (see tnc_amplitudes)
  std::map<std::string, cudaGraphExec_t> graphs;
  std::map<std::string, int> graph_seen;
  // concurrent schedule of the launches (see make_schedule): the lane each runs on and, per
  // launch, the latest launch it must follow on every other lane (-1: none); a launch records
  // its event only when a launch on another lane waits for it
  int n_lanes = 1;
  std::vector<int> lane;
  std::vector<std::vector<int>> wait_on;  // [launch][lane]
  std::vector<char> signals;
  std::vector<cudaEvent_t> done_ev;
  // one persistent launch for the steps (programs of SIMT steps only; tnc_exec_opts.reserved[2])
  bool persist_ok = false;
  int n_phases = 0;
  size_t steps_smem = 0;
  DevBuf step_ops, step_phases, steps_bar;
  ~DeviceProgram() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    for (auto e : done_ev)
      if (e) cudaEventDestroy(e);
    arena.release();
    maxabs.release();
    exps.release();
    leaf_src.release();
    leaf_desc.release();
    partials.release();
    open_pos.release();
    chain_links.release();
    leaf_r.release();
    inst_c.release();
    step_ops.release();
    step_phases.release();
    steps_bar.release();
    cudaGetLastError();  // a failed release must not surface as the next launch's error
  }
};

}  // namespace tnc

using namespace tnc;

// Events of the last profiled call: per (wave, step) a start/end pair, plus the call.
struct ProfState {
  bool valid = false;
  int n_steps = 0, waves = 0;
  std::vector<cudaEvent_t> ev;
  std::vector<double> flops, bytes;
  std::vector<int> kind, kernels;  // kernels: launches per wave (2 when a split step reduces)
  cudaStream_t stream = nullptr;
  cudaEvent_t& at(int w, int s, int which) { return ev[(size_t(w) * n_steps + s) * 2 + which]; }
  void ensure(int steps, int w) {
    const size_t need = size_t(steps) * w * 2 + 2;
    while (ev.size() < need) {
      cudaEvent_t x;
      if (cudaEventCreate(&x) != cudaSuccess) fail(TNC_E_CUDA, "cudaEventCreate failed");
      ev.push_back(x);
    }
    n_steps = steps;
    waves = w;
  }
  cudaEvent_t& call_start() { return ev[size_t(n_steps) * waves * 2]; }
  cudaEvent_t& call_end() { return ev[size_t(n_steps) * waves * 2 + 1]; }
  ~ProfState() {
    for (auto x : ev) cudaEventDestroy(x);
  }
};

struct tnc_context_s {
  int device = 0;
  int id = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  size_t total_mem = 0;
  DevBuf bits, inst_slice, inst_row, segs, acc, scratch, partials, status, ttgt;
  bool no_tc = false;  // TNC_NO_TC=1 in the environment: every step on the SIMT kernels
  bool no_tc64 = false; // TNC_NO_TC64=1: complex64 steps on the SIMT kernels (3xTF32 off)
  bool no_tma = false; // TNC_NO_TMA=1: tensor-core steps gather their tiles with cp.async
  bool no_persist = false;  // TNC_NO_PERSIST=1: short-K TMA steps use one CTA per tile
  bool no_reuse = false;    // TNC_NO_REUSE=1: every step runs for every (row, slice)
  bool no_stream = false;   // TNC_NO_STREAM=1: GEPDOT steps load tiles synchronously (k_generic)
  bool serial = false;      // TNC_SERIAL=1: every launch of a wave on one stream
  cudaStream_t lanes[4] = {nullptr, nullptr, nullptr, nullptr};  // streams of concurrent branches
  cudaEvent_t fork_ev = nullptr, join_ev[4] = {nullptr, nullptr, nullptr, nullptr};
  ProfState prof;
  ~tnc_context_s() {
    for (auto l : lanes)
      if (l) cudaStreamDestroy(l);
    if (fork_ev) cudaEventDestroy(fork_ev);
    for (auto e : join_ev)
      if (e) cudaEventDestroy(e);
    bits.release();
    inst_slice.release();
    inst_row.release();
    segs.release();
    acc.release();
    scratch.release();
    partials.release();
    status.release();
    ttgt.release();
  }
};

static std::atomic<int> g_ctx_ids{1};

namespace tnc {

void release_plan_device(tnc_plan_s* p) { p->programs.clear(); }

// FP64 leaf sources and gather descriptors; dst[i] = arena offset (scalars) of reduced leaf i.
// Synchronous copies: callers drain the stream first when buffers may be in use.
static void upload_leaves(const Plan& P, const std::vector<int64_t>& dst, DevBuf& srcb, DevBuf& descb) {
  std::vector<double2> src;
  std::vector<LeafDesc> desc;
  for (size_t i = 0; i < P.net.leaves.size(); ++i) {
    const Leaf& lf = P.net.leaves[i];
    LeafDesc d;
    std::memset(&d, 0, sizeof(d));
    d.src = (int64_t)src.size();
    for (const cd& v : lf.t.data) src.push_back(make_double2(v.real(), v.imag()));
    d.dst = dst[i];
    d.rank_full = (int)lf.t.labels.size();
    d.rank = (int)P.tensors[i].labels.size();
    d.slot = (int)i;
    const auto& fx = P.leaf_fix[i];
    if (fx.size() > 8 || d.rank > 5) fail(TNC_E_UNSUPPORTED, "leaf with too many legs");
    d.nfix = (int)fx.size();
    for (size_t f = 0; f < fx.size(); ++f) {
      d.fix_pos[f] = (int8_t)fx[f].pos;
      d.fix_kind[f] = (int8_t)fx[f].kind;
      d.fix_idx[f] = (int16_t)fx[f].index;
    }
    desc.push_back(d);
  }
  srcb.reserve(std::max<size_t>(1, src.size()) * sizeof(double2));
  descb.reserve(std::max<size_t>(1, desc.size()) * sizeof(LeafDesc));
  CUDA_OK(cudaMemcpy(srcb.p, src.data(), src.size() * sizeof(double2), cudaMemcpyHostToDevice));
  CUDA_OK(cudaMemcpy(descb.p, desc.data(), desc.size() * sizeof(LeafDesc), cudaMemcpyHostToDevice));
}

// Host-side construction of a fused chain's launch and index tables (see k_chain).
template <class OffFn>
static StepLaunch make_chain_launch(const Plan& P, const Chain& ch, std::vector<ChainLink>& links, OffFn OFF) {
  auto pos = [](const std::vector<int>& v, int x) {
    for (size_t i = 0; i < v.size(); ++i)
      if (v[i] == x) return (int)i;
    return -1;
  };
  auto order_by = [&](std::vector<int> v, const std::vector<int>& layout) {
    std::sort(v.begin(), v.end(), [&](int x, int y) { return pos(layout, x) < pos(layout, y); });
    return v;
  };
  StepLaunch L;
  std::memset(&L.p, 0, sizeof(L.p));
  std::memset(&L.tp, 0, sizeof(L.tp));
  std::memset(&L.cp, 0, sizeof(L.cp));
  L.kind = K_CHAIN;
  L.smem = 0;
  L.rm = L.rn = 1;
  ChainParams& c = L.cp;
  const Step& first = P.steps[ch.steps.front()];
  const Step& last = P.steps[ch.steps.back()];
  const std::vector<int>& la0 = P.tensors[first.a].labels;
  const std::vector<int>& lcn = P.tensors[last.c].labels;
  std::vector<int> prev = order_by(ch.inner0, la0);
  if (prev.size() > size_t(kChainMaxBits + kChainClusterBits)) fail(TNC_E_PLAN, "chain tile too large");
  for (int x : prev) c.maskA0 |= 1u << pos(la0, x);
  c.runA0 = low_run(c.maskA0);
  c.bits0 = (int)prev.size();
  c.offA0 = OFF(first.a);
  c.planeA0 = int64_t(1) << la0.size();
  c.slotA0 = first.a;
  c.n_links = (int)ch.steps.size();
  // the labels each link contracts, and the largest on-chip tile of the chain: above 2^12
  // entries the tile is spread over a cluster of 2^cb CTAs by its top cb bits
  const size_t nl = ch.steps.size();
  std::vector<std::vector<int>> Ks(nl);
  size_t max_bits = prev.size();
  {
    std::vector<int> I = prev;
    for (size_t l = 0; l < nl; ++l) {
      const Step& st = P.steps[ch.steps[l]];
      const std::vector<int>& la = P.tensors[st.a].labels;
      const std::vector<int>& lg = P.tensors[st.b].labels;
      std::vector<int> nI;
      for (int x : lg)
        if (pos(la, x) >= 0) Ks[l].push_back(x);
      for (int x : I)
        if (pos(Ks[l], x) < 0) nI.push_back(x);
      for (int x : lg)
        if (pos(la, x) < 0) nI.push_back(x);
      I = nI;
      max_bits = std::max(max_bits, I.size());
    }
  }
  const int cb = max_bits > size_t(kChainMaxBits) ? int(max_bits) - kChainMaxBits : 0;
  // inter-CTA labels (the top cb bits of a tile) of the intermediate tiles: those contracted
  // latest, keeping the previous tile's where they tie (Sec. IV, Eq. 2: indices chosen by
  // their remaining lifetime, so that most links read only their own CTA's entries)
  std::vector<int> J(prev.end() - cb, prev.end());
  double bytes = double(int64_t(1) << la0.size());
  for (size_t l = 0; l < nl; ++l) {
    const int sidx = ch.steps[l];
    const Step& st = P.steps[sidx];
    const std::vector<int>& la = P.tensors[st.a].labels;
    const std::vector<int>& lg = P.tensors[st.b].labels;
    const std::vector<int>& lc = P.tensors[st.c].labels;
    std::vector<int> K, N, cur;
    for (int x : lg) (pos(la, x) >= 0 ? K : N).push_back(x);
    for (int x : prev)
      if (pos(K, x) < 0) cur.push_back(x);
    for (int x : K)
      if (pos(prev, x) < 0) fail(TNC_E_PLAN, "chain: contracted label not on chip");
    cur.insert(cur.end(), N.begin(), N.end());
    if (l + 1 == nl || cb == 0) {
      cur = order_by(cur, lc);  // the result's own order (the last tile is stored in it)
    } else {
      auto next_use = [&](int x) {
        for (size_t m = l + 1; m < nl; ++m)
          if (pos(Ks[m], x) >= 0) return int(m);
        return int(nl);
      };
      // the labels contracted latest (never, for most); among equals, those that are
      // inter-CTA already (no swap now), then the result's top labels (no swap at the end)
      const std::vector<int>& lcl = P.tensors[last.c].labels;
      std::vector<int> final_top = order_by(std::vector<int>(lcl.begin(), lcl.end()), lcl);
      final_top.erase(final_top.begin(), final_top.end() - std::min<size_t>(final_top.size(), size_t(cb)));
      std::vector<int> cand = cur;
      std::stable_sort(cand.begin(), cand.end(), [&](int x, int y) {
        const int ux = next_use(x), uy = next_use(y);
        if (ux != uy) return ux > uy;
        const bool jx = pos(J, x) >= 0, jy = pos(J, y) >= 0;
        if (jx != jy) return jx;
        return (pos(final_top, x) >= 0) > (pos(final_top, y) >= 0);
      });
      std::vector<int> nJ(cand.begin(), cand.begin() + cb);
      // kept labels stay in their previous top positions
      std::vector<int> top;
      for (int x : J)
        if (pos(nJ, x) >= 0) top.push_back(x);
      for (int x : nJ)
        if (pos(top, x) < 0) top.push_back(x);
      std::vector<int> intra;
      for (int x : cur)
        if (pos(top, x) < 0) intra.push_back(x);
      cur = order_by(intra, lc);
      cur.insert(cur.end(), top.begin(), top.end());
      J = top;
    }
    if (cur.size() > size_t(kChainMaxBits + kChainClusterBits) || K.size() > 6 || N.size() > 6)
      fail(TNC_E_PLAN, "chain link too large");
    ChainLink lk;
    std::memset(&lk, 0, sizeof(lk));
    lk.g_off = OFF(st.b);
    lk.g_plane = int64_t(1) << lg.size();
    lk.g_size = 1 << (int)lg.size();
    lk.slot_g = st.b;
    lk.out_bits = (int)cur.size();
    lk.k_bits = (int)K.size();
    lk.n_bits = (int)N.size();
    lk.in_ibits = (int)prev.size() - cb;
    lk.out_ibits = (int)cur.size() - cb;
    if (lk.in_ibits < 0 || lk.out_ibits < 0 || lk.in_ibits > kChainMaxBits || lk.out_ibits > kChainMaxBits)
      fail(TNC_E_PLAN, "chain: tile not divisible over the cluster");
    for (int k = 0; k < (1 << K.size()); ++k) {
      uint32_t ai = 0, gi = 0;
      for (size_t j = 0; j < K.size(); ++j)
        if ((k >> j) & 1) ai |= 1u << pos(prev, K[j]), gi |= 1u << pos(lg, K[j]);
      lk.kin[k] = (uint16_t)ai;
      lk.kg[k] = (uint8_t)gi;
    }
    for (int n = 0; n < (1 << N.size()); ++n) {
      uint32_t gi = 0;
      for (size_t j = 0; j < N.size(); ++j)
        if ((n >> j) & 1) gi |= 1u << pos(lg, N[j]);
      lk.gn[n] = (uint8_t)gi;
    }
    // bit scatters of the output index: `count` bits of v placed at output bits shift..
    auto scatter = [&](uint32_t v, int shift, int count, bool want_in) {
      uint32_t r = 0;
      for (int j = 0; j < count && size_t(j + shift) < cur.size(); ++j) {
        if (!((v >> j) & 1)) continue;
        const int lab = cur[j + shift];
        const int pi = pos(prev, lab);
        if (want_in && pi >= 0) r |= 1u << pi;
        if (!want_in && pi < 0) r |= 1u << pos(lg, lab);
      }
      return r;
    };
    // single CTA: x = the whole output index; cluster: x = its low out_ibits bits, the rank
    // = its top cb bits
    const int xb = cb ? lk.out_ibits : (int)cur.size();
    for (uint32_t v = 0; v < 64; ++v) {
      lk.ib_lo[v] = (uint16_t)scatter(v, 0, std::min(6, xb), true);
      lk.ib_hi[v] = (uint16_t)scatter(v, 6, std::max(0, std::min(6, xb - 6)), true);
      lk.gb_lo[v] = (uint8_t)scatter(v, 0, std::min(6, xb), false);
      lk.gb_hi[v] = (uint8_t)scatter(v, 6, std::max(0, std::min(6, xb - 6)), false);
    }
    for (uint32_t v = 0; v < 8; ++v) {
      lk.ib_top[v] = (uint16_t)scatter(v, xb, cb, true);
      lk.gb_top[v] = (uint8_t)scatter(v, xb, cb, false);
    }
    // local link: the output's inter-CTA labels are the input's, in the same order, and
    // neither the other output labels nor the contracted ones are inter-CTA in the input
    lk.remote = 0;
    if (cb) {
      for (int j = 0; j < cb; ++j)
        if (pos(prev, cur[xb + j]) != lk.in_ibits + j) lk.remote = 1;
      for (int j = 0; j < xb; ++j) {
        const int pi = pos(prev, cur[j]);
        if (pi >= lk.in_ibits) lk.remote = 1;
      }
      for (int x : K)
        if (pos(prev, x) >= lk.in_ibits) lk.remote = 1;
    }
    links.push_back(lk);
    L.flops += 8.0 * std::ldexp(1.0, (int)(la.size() + N.size()));
    bytes += std::ldexp(1.0, (int)lg.size());
    prev = cur;
  }
  for (int x : prev) c.maskC |= 1u << pos(lcn, x);
  c.runC = low_run(c.maskC);
  c.bitsC = (int)prev.size();
  c.cl_bits = cb;
  c.offC = OFF(last.c);
  c.planeC = int64_t(1) << lcn.size();
  c.slotC = last.c;
  for (int x : la0) {
    if (pos(ch.inner0, x) >= 0) continue;
    if (pos(lcn, x) < 0) fail(TNC_E_PLAN, "chain: outer label lost");
    if (c.n_o >= kMaxOuter) fail(TNC_E_UNSUPPORTED, "chain: too many outer labels");
    c.o_A[c.n_o] = (int8_t)pos(la0, x);
    c.o_C[c.n_o] = (int8_t)pos(lcn, x);
    c.n_o++;
  }
  if (c.n_o > 30) fail(TNC_E_UNSUPPORTED, "chain: grid too large");
  bytes += std::ldexp(1.0, (int)lcn.size());
  L.bytes = bytes * 2;  // two planes; times the element size by the caller
  L.grid = dim3(1u << c.n_o, 1, 1);
  return L;
}

// ------------------------------------------------------------------ tensor-core step configurations
// What the tuner may choose for a tensor-core step.  Every choice computes the same
// contraction; only the split over K changes the grouping of the FP32 sums.
struct TcChoice {
  int bn = 0;          // tile width 64, 128 or 256, at most the compiled one (a prefix of Nt)
  int persistent = 0;  // one CTA per SM walking the tiles (no split; BN 256 needs the direct epilogue)
  int split = 0;       // split over the outer common labels; 0: the heuristics of make_tc_launch
  int stages = 0;      // pipeline (BN < 256): 0 heuristics, 3 three stages (two CTAs per SM), 1 deep
};

// Process-wide cache of tuned choices keyed by step shape: tnc_autotune fills it,
// build_program reads it, tnc_tune_save / tnc_tune_load keep it in a text file.
static std::mutex g_tune_mu;
static std::map<std::string, TcChoice> g_tune;

static bool tune_lookup(const std::string& key, TcChoice* ch) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(key);
  if (it == g_tune.end()) return false;
  *ch = it->second;
  return true;
}

// Shape of a tensor-core step as the tuner sees it: precision, operand and result ranks,
// compiled tile width and depth, outer label counts of the heuristic launch `D`, direct
// epilogue, and the instances one launch covers.
static std::string tune_key(int precision, const Plan& P, const Step& st, const StepLaunch& D, int64_t nz) {
  const int ta = st.tc_swap ? st.b : st.a, tb = st.tc_swap ? st.a : st.b;
  char buf[192];
  std::snprintf(buf, sizeof buf, "p%d.a%zu.b%zu.c%zu.bn%d.bk%d.om%d.on%d.ok%d.d%d.z%lld", precision,
                P.tensors[ta].labels.size(), P.tensors[tb].labels.size(), P.tensors[st.c].labels.size(), st.tc_bn,
                st.tc_bk, D.tp.n_om, D.tp.n_on, D.tp.n_ok, D.tp.direct, (long long)nz);
  return buf;
}

static int64_t prog_off(const Plan& P, const DeviceProgram* prog, int t) {
  const int64_t o = prog->fused ? P.tensors[t].offset_fused : P.tensors[t].offset;
  if (o < 0) fail(TNC_E_PLAN, "tensor has no arena slot in this program");
  return o;
}

// Tensor-core launch of plan step `si` in `prog` with configuration `ch` (nullptr: the
// heuristics of make_tc_launch and the wave-size rule for the persistent kernel).  The split
// over K is sized from the plan's slice count, not the wave size, so results do not depend on
// how many instances share a launch.
static StepLaunch tc_launch(const tnc_context_s* ctx, const Plan& P, const DeviceProgram* prog, int si,
                            const TcChoice* ch) {
  const Step& st = P.steps[si];
  const int ta = st.tc_swap ? st.b : st.a, tb = st.tc_swap ? st.a : st.b;
  const auto& la = P.tensors[ta].labels;
  const auto& lb = P.tensors[tb].labels;
  const auto& lc = P.tensors[st.c].labels;
  TileSpec t = st.tc_tile;
  int bn = st.tc_bn;
  if (prog->precision == TNC_C64 && bn == 256) {
    // the 3xTF32 kernel keeps hi and lo parts of every stage: 128-wide tiles at most
    t.No.insert(t.No.begin(), t.Nt.begin() + 7, t.Nt.end());
    t.Nt.resize(7);
    bn = 128;
  }
  if (ch && ch->bn && ch->bn < bn) {
    // a narrower tile loads a prefix of B's tile labels (B is laid out [Kt | Nt | ...]); the
    // rest become the lowest outer labels
    if (ch->bn != 64 && ch->bn != 128) fail(TNC_E_PLAN, "bad tuned tile width");
    const size_t nt = ch->bn == 128 ? 7 : 6;
    t.No.insert(t.No.begin(), t.Nt.begin() + nt, t.Nt.end());
    t.Nt.resize(nt);
    bn = ch->bn;
  }
  StepLaunch L;
  std::memset(&L.cp, 0, sizeof(L.cp));
  L.rm = L.rn = 0;
  L.plan_step = si;
  make_tc_launch(L, t, la, lb, lc, prog->precision, bn, st.tc_bk, prog->split_inst, ch ? ch->split : 0);
  // persistent kernels: two TMEM buffers up to 128 columns; 256-wide tiles hand their one
  // buffer back after draining it into registers, which needs the direct epilogue
  const bool can_persist = L.tp.splitk == 1 && bn >= 64 && (bn <= 128 || L.tp.direct);
  const int64_t tiles_w = (int64_t(1) << (L.tp.n_om + L.tp.n_on)) * prog->W;
  const bool heuristic =
      (bn <= 128 && L.tp.n_ok <= 3 && tiles_w >= 4 * 152) || (bn == 256 && L.tp.n_ok <= 8 && tiles_w >= 2 * 152);
  L.tp.persistent = (ch ? ch->persistent != 0 : heuristic) && can_persist ? 1 : 0;
  if (prog->precision == TNC_C64) L.tp.persistent = 0;  // one CTA per tile (3xTF32 kernel)
  if (ch && ch->stages) L.tp.stages = ch->stages == 3 ? 3 : 0;
  const size_t eb = elem_bytes(prog->precision);
  char* arena = prog->arena.as<char>();
  bind_tc(L, arena + prog_off(P, prog, ta) * eb, arena + prog_off(P, prog, tb) * eb,
          arena + prog_off(P, prog, st.c) * eb, prog->inst_stride, prog->maxabs.as<float>(), prog->exps.as<int32_t>(),
          prog->n_slots, ta, tb, st.c, ctx->status.as<int32_t>(), prog->partials.as<float2>());
  if (!ctx->no_tma) {
    // operands are laid out [Kt | Mt/Nt | ...] by the compiler: load tiles with TMA
    const int kt = st.tc_bk == 32 ? 5 : 4;
    encode_tile_map(&L.tp.tmA, L.tp.A, (int)la.size(), kt, 128, prog->inst_stride, prog->W, eb);
    encode_tile_map(&L.tp.tmB, L.tp.B, (int)lb.size(), kt, bn, prog->inst_stride, prog->W, eb);
    L.kind = K_TMA;
    if (ctx->no_persist) L.tp.persistent = 0;
  }
  int common = 0;
  for (int x : la) common += std::find(lb.begin(), lb.end(), x) != lb.end();
  L.flops = 8.0 * std::ldexp(1.0, (int)(la.size() + lb.size()) - common);
  L.bytes =
      (std::ldexp(1.0, (int)la.size()) + std::ldexp(1.0, (int)lb.size()) + std::ldexp(1.0, (int)lc.size())) * 2.0 * double(eb);
  return L;
}

// Concurrent schedule of an unfused program's launches (launch k = plan step k).  Launch k
// must follow: the producers of its operands; every earlier launch that read or wrote arena
// memory overlapping its result (the arena reuses the memory of dead tensors, assuming the
// plan's order); and, when it splits over K, the previous launch that used the shared
// partial-sum buffer.  Launches are dealt greedily to kLanes lanes: onto the lane of the
// latest launch they follow when that launch is the lane's last, else onto the lane idle
// longest.  Results do not change: every launch computes the same values in any order that
// respects these dependencies.
constexpr int kLanes = 4;

// The launches each launch k must follow: its operands' producers, every earlier launch whose
// tensors share arena memory with its result (the arena reuses regions), and the previous
// split launch (split launches share one partial-sum buffer).  Programs of plan steps only.
static std::vector<std::vector<int>> step_deps(const Plan& P, const DeviceProgram* prog) {
  const int n = (int)prog->steps.size();
  auto region = [&](int t) {
    const int64_t off = prog_off(P, prog, t);
    return std::make_pair(off, off + 2 * (int64_t(1) << P.tensors[t].labels.size()));
  };
  auto overlap = [](std::pair<int64_t, int64_t> x, std::pair<int64_t, int64_t> y) {
    return x.first < y.second && y.first < x.second;
  };
  std::vector<int> producer(P.tensors.size(), -1);
  std::vector<std::vector<int>> deps(n);
  int last_split = -1;
  for (int k = 0; k < n; ++k) {
    const Step& st = P.steps[k];
    const auto rc = region(st.c);
    std::vector<int>& d = deps[k];
    for (int t : {st.a, st.b})
      if (producer[t] >= 0) d.push_back(producer[t]);
    for (int j = 0; j < k; ++j) {
      const Step& sj = P.steps[j];
      if (overlap(rc, region(sj.c)) || overlap(rc, region(sj.a)) || overlap(rc, region(sj.b))) d.push_back(j);
    }
    const StepLaunch& L = prog->steps[k];
    const bool split = L.kind == K_SPLITK || ((L.kind == K_TC || L.kind == K_TMA) && L.tp.splitk > 1);
    if (split) {
      if (last_split >= 0) d.push_back(last_split);
      last_split = k;
    }
    producer[st.c] = k;
  }
  return deps;
}

static void make_schedule(const Plan& P, DeviceProgram* prog) {
  const int n = (int)prog->steps.size();
  for (auto e : prog->done_ev)
    if (e) cudaEventDestroy(e);
  prog->done_ev.clear();
  prog->n_lanes = 1;
  prog->lane.assign(n, 0);
  prog->wait_on.assign(n, std::vector<int>(kLanes, -1));
  prog->signals.assign(n, 0);
  if (n != (int)P.steps.size() || n < 2) return;
  for (const auto& L : prog->steps)
    if (L.kind == K_CHAIN) return;
  const std::vector<std::vector<int>> deps = step_deps(P, prog);
  // lanes
  std::vector<int> lane_last(kLanes, -1);
  for (int k = 0; k < n; ++k) {
    int pick = -1, best_dep = -1;
    for (int j : deps[k])
      for (int l = 0; l < kLanes; ++l)
        if (lane_last[l] == j && j > best_dep) best_dep = j, pick = l;
    if (pick < 0) {
      pick = 0;
      for (int l = 1; l < kLanes; ++l)
        if (lane_last[l] < lane_last[pick]) pick = l;
    }
    prog->lane[k] = pick;
    lane_last[pick] = k;
    for (int j : deps[k]) {
      const int l = prog->lane[j];
      if (l != pick && j > prog->wait_on[k][l]) prog->wait_on[k][l] = j;
    }
    for (int l = 0; l < kLanes; ++l)
      if (prog->wait_on[k][l] >= 0) prog->signals[prog->wait_on[k][l]] = 1;
  }
  prog->n_lanes = kLanes;
  prog->done_ev.assign(n, nullptr);
  for (int k = 0; k < n; ++k)
    if (prog->signals[k]) CUDA_OK(cudaEventCreateWithFlags(&prog->done_ev[k], cudaEventDisableTiming));
}

static std::shared_ptr<DeviceProgram> build_program(tnc_context_s* ctx, tnc_plan_s* plan, int precision, int W,
                                                    bool fuse, bool merge = false) {
  const Plan& P = plan->p;
  auto prog = std::make_shared<DeviceProgram>();
  prog->merge = merge;
  prog->device = ctx->device;
  prog->precision = precision;
  prog->W = W;
  prog->n_qubits = P.net.circ.n;
  const bool fused = fuse && !P.chains.empty();
  prog->fused = fused;
  prog->inst_stride = ((fused ? P.arena_elems_fused : P.arena_elems) + 63) & ~int64_t(63);
  auto OFF = [&](int t) { return prog_off(P, prog.get(), t); };
  // tree-like reuse across slices (see the step maps below) needs waves of whole rows and no
  // fused chains
  const int sbits = (int)P.sliced.size();
  const bool reuse_shape = !ctx->no_reuse && sbits >= 1 && sbits <= 20 && W % (int64_t(1) << sbits) == 0 && !fused;
  prog->n_slots = (int)P.tensors.size();
  prog->n_leaves = (int)P.net.leaves.size();
  const size_t eb = elem_bytes(precision);
  prog->split_inst = split_instances(P, double(prog->inst_stride) * double(eb) * 1.25 + 4096.0, double(ctx->total_mem));
  prog->arena.reserve(size_t(prog->inst_stride) * eb * W + 256);
  prog->maxabs.reserve(size_t(prog->n_slots) * W * sizeof(float));
  prog->exps.reserve(size_t(prog->n_slots) * W * sizeof(int32_t));
  prog->leaf_r.reserve(size_t(std::max(1, prog->n_leaves)) * W * sizeof(double2));
  prog->inst_c.reserve(size_t(W) * sizeof(double2));
  // leaves: FP64 sources + descriptors
  {
    std::vector<int64_t> dst(prog->n_leaves);
    for (int i = 0; i < prog->n_leaves; ++i) dst[i] = OFF(i);
    upload_leaves(P, dst, prog->leaf_src, prog->leaf_desc);
    prog->leaf_version = P.gate_version;
    prog->leaf_dst = dst;
  }
  // steps
  size_t partial_elems = 0;
  std::vector<ChainLink> chain_links;
  std::vector<std::pair<size_t, size_t>> chain_at;  // (launch index, first link index)
  for (size_t s = 0; s < P.steps.size(); ++s) {
    const Step& st = P.steps[s];
    const auto& la = P.tensors[st.a].labels;
    const auto& lb = P.tensors[st.b].labels;
    const auto& lc = P.tensors[st.c].labels;
    if (fuse && s < P.step_chain.size() && P.step_chain[s] >= 0) {
      const Chain& ch = P.chains[P.step_chain[s]];
      if ((int)s != ch.steps.back()) continue;  // the chain runs at its last step
      const size_t first_link = chain_links.size();
      StepLaunch L = make_chain_launch(P, ch, chain_links, OFF);
      L.cp.stride = prog->inst_stride;
      L.cp.arena = prog->arena.p;
      L.cp.maxabs = prog->maxabs.as<float>();
      L.cp.exps = prog->exps.as<int32_t>();
      L.cp.n_slots = prog->n_slots;
      L.bytes *= (double)eb;
      chain_at.emplace_back(prog->steps.size(), first_link);
      prog->steps.push_back(L);
      continue;
    }
    // the plan's SIMT tiles size their splits over K for every slice in flight (at most
    // 2^12); a program whose device holds fewer instances re-sizes them (only the split and
    // the kind that follows from it change)
    TileSpec tile = st.tile;
    int kind = st.kind;
    if (prog->split_inst < (int64_t(1) << std::min<size_t>(P.sliced.size(), 12)))
      tile = tile_for(la, lb, lc, (int)prog->split_inst, kind);
    StepLaunch L = make_launch(tile, kind, la, lb, lc);
    {
      int common = 0;
      for (int x : la) common += std::find(lb.begin(), lb.end(), x) != lb.end();
      L.flops = 8.0 * std::ldexp(1.0, (int)(la.size() + lb.size()) - common);
      L.bytes = (std::ldexp(1.0, (int)la.size()) + std::ldexp(1.0, (int)lb.size()) + std::ldexp(1.0, (int)lc.size())) *
                2.0 * double(eb);
    }
    // 32-wide tiles exist only in the TMA kernel
    const bool tc64 = precision == TNC_C64 && !ctx->no_tc64 && !ctx->no_tma;
    if ((precision != TNC_C64 || tc64) && st.tc_ok && !ctx->no_tc && !(ctx->no_tma && st.tc_bn == 32)) {
      StepLaunch T = tc_launch(ctx, P, prog.get(), (int)s, nullptr);
      if (T.kind == K_TMA) {
        // a configuration tuned for this shape (tnc_autotune) replaces the heuristics
        const int64_t nz = reuse_shape ? (int64_t(W) >> sbits) << __builtin_popcount((uint32_t)P.tensors[st.c].dep) : W;
        TcChoice ch;
        if (tune_lookup(tune_key(precision, P, st, T, nz), &ch)) {
          try {
            T = tc_launch(ctx, P, prog.get(), (int)s, &ch);
          } catch (const Error&) {
            // a cached choice this step's layouts cannot take (a hand-edited cache file):
            // the heuristics stay
          }
        }
      }
      if (T.tp.splitk > 1) partial_elems = std::max(partial_elems, size_t(W) * T.tp.splitk * T.tp.planeC);
      prog->steps.push_back(T);
      continue;
    }
    L.p.A = prog->arena.as<char>() + OFF(st.a) * eb;
    L.p.B = prog->arena.as<char>() + OFF(st.b) * eb;
    L.p.C = prog->arena.as<char>() + OFF(st.c) * eb;
    L.p.strideA = L.p.strideB = L.p.strideC = prog->inst_stride;
    L.p.maxabs = prog->maxabs.as<float>();
    L.p.exps = prog->exps.as<int32_t>();
    L.p.n_slots = prog->n_slots;
    L.p.slotA = st.a;
    L.p.slotB = st.b;
    L.p.slotC = st.c;
    make_stream(L, eb, ctx->no_stream);
    if (L.kind == K_SPLITK) partial_elems = std::max(partial_elems, size_t(W) * L.p.splitk * L.p.planeC);
    prog->steps.push_back(L);
  }
  if (partial_elems) {
    prog->partials.reserve(partial_elems * sizeof(float2));
    for (auto& L : prog->steps) {
      if (L.kind == K_SPLITK) L.p.partials = prog->partials.as<float2>();
      if ((L.kind == K_TC || L.kind == K_TMA) && L.tp.splitk > 1) L.tp.partials = L.p.partials = prog->partials.as<float2>();
    }
  }
  if (!chain_links.empty()) {
    prog->chain_links.reserve(chain_links.size() * sizeof(ChainLink));
    CUDA_OK(cudaMemcpy(prog->chain_links.p, chain_links.data(), chain_links.size() * sizeof(ChainLink),
                       cudaMemcpyHostToDevice));
    for (auto& ca : chain_at) prog->steps[ca.first].cp.links = prog->chain_links.as<ChainLink>() + ca.second;
  }
  // tree-like reuse across slices (Sec. III-B): a step runs once per assignment of the sliced
  // indices its result depends on.  Needs waves of whole rows (all 2^s slices of a bitstring)
  // and launches that map one to one onto the plan's steps (no fused chains); a call uses the
  // maps only when it covers every slice (see tnc_amplitudes).
  {
    const bool reuse = reuse_shape && chain_links.empty() && prog->steps.size() == P.steps.size();
    // post-lifetime merging (Sec. III-B): the step whose two operands both depend on sliced
    // index t contracts t's edge; its result is summed over t right after it (not at the
    // root step, where the root sum does the same), and every later tensor depends on t no
    // longer.  mdep = the dependence masks with merged indices removed.
    std::vector<uint32_t> mdep(P.tensors.size(), 0);
    for (size_t i = 0; i < P.tensors.size(); ++i) mdep[i] = (uint32_t)P.tensors[i].dep;
    std::vector<uint32_t> full(P.steps.size(), 0), mbits(P.steps.size(), 0);
    for (size_t si = 0; si < P.steps.size(); ++si) {
      const Step& st = P.steps[si];
      full[si] = mdep[st.a] | mdep[st.b];
      if (merge && reuse && si + 1 < P.steps.size()) mbits[si] = mdep[st.a] & mdep[st.b];
      mdep[st.c] = full[si] & ~mbits[si];
    }
    // the two leaves holding each sliced index (its leaf-rounding scales enter the merge)
    std::vector<std::vector<int>> holders(P.sliced.size());
    for (size_t i = 0; i < P.leaf_fix.size(); ++i)
      for (const auto& lf : P.leaf_fix[i])
        if (lf.kind == 0 && lf.index < (int)holders.size()) holders[lf.index].push_back((int)i);
    prog->merged_mask = 0;
    for (size_t si = 0; si < prog->steps.size(); ++si) {
      StepLaunch& L = prog->steps[si];
      L.merges.clear();
      InstMap m{-1, 0, 0, 0};
      if (reuse) {
        const Step& st = P.steps[si];
        const bool tcs = (L.kind == K_TC || L.kind == K_TMA) && st.tc_swap;
        const int ta = tcs ? st.b : st.a, tb = tcs ? st.a : st.b;
        m = InstMap{sbits, full[si], mdep[ta], mdep[tb]};
        uint32_t left = full[si];
        for (int t = 0; t < sbits; ++t) {
          if (!((mbits[si] >> t) & 1u)) continue;
          if (holders[t].size() != 2) fail(TNC_E_PLAN, "merge: a sliced index must sit in two leaves");
          left &= ~(1u << t);
          StepLaunch::MergeOp op;
          op.bit = t;
          op.lu = holders[t][0];
          op.lv = holders[t][1];
          op.slot = st.c;
          op.off = OFF(st.c);
          op.plane = int64_t(1) << P.tensors[st.c].labels.size();
          op.im = InstMap{sbits, left, 0, 0};
          op.arena = prog->arena.p;
          op.inst_stride = prog->inst_stride;
          op.exps = prog->exps.as<int32_t>();
          op.maxabs = prog->maxabs.as<float>();
          op.n_slots = prog->n_slots;
          op.n_leaves = prog->n_leaves;
          op.leaf_r = prog->leaf_r.as<double2>();
          L.merges.push_back(op);
          prog->merged_mask |= 1u << t;
        }
      }
      L.p.im = m;
      L.tp.im = m;
    }
    prog->reuse_ok = reuse;
    prog->root_map = reuse ? InstMap{sbits, mdep[P.root], 0, 0} : InstMap{-1, 0, 0, 0};
  }
  // the steps as one persistent launch (k_steps), for programs whose steps are all SIMT
  // contractions without merges.  Streamed steps run their tiled form (bit-identical; their
  // shared-memory region also fits the tiled layout).  Phases: a step's phase is one past the
  // latest phase of the launches it must follow (step_deps), and the steps go in phase order.
  {
    std::vector<StepOp> ops;
    bool ok = !prog->steps.empty() && prog->steps.size() == P.steps.size();
    for (const auto& L : prog->steps)
      if ((L.kind != K_GENERIC && L.kind != K_SPLITK) || !L.merges.empty()) ok = false;
    std::vector<int> order, phases;
    if (ok) {
      const auto deps = step_deps(P, prog.get());
      std::vector<int> level(prog->steps.size(), 0);
      for (size_t k = 0; k < level.size(); ++k)
        for (int j : deps[k]) level[k] = std::max(level[k], level[j] + 1);
      for (size_t k = 0; k < level.size(); ++k) order.push_back((int)k);
      std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return level[x] < level[y]; });
      for (size_t i = 0; i < order.size(); ++i)
        if (i == 0 || level[order[i]] != level[order[i - 1]]) phases.push_back((int)i);
      phases.push_back((int)order.size());
    }
    size_t smem = 0;
    for (int k : order) {
      const StepLaunch& L = prog->steps[k];
      StepOp op;
      std::memset(&op, 0, sizeof(op));
      op.p = L.p;
      op.p.stream = 0;
      op.rm = L.rm;
      op.rn = L.rn;
      op.reduce = L.kind == K_SPLITK ? (L.p.splitk >= kWideReduceSplit ? 2 : 1) : 0;
      ops.push_back(op);
      smem = std::max(smem, L.smem);
    }
    if (ok) {
      prog->step_ops.reserve(ops.size() * sizeof(StepOp));
      CUDA_OK(cudaMemcpy(prog->step_ops.p, ops.data(), ops.size() * sizeof(StepOp), cudaMemcpyHostToDevice));
      prog->step_phases.reserve(phases.size() * sizeof(int32_t));
      CUDA_OK(cudaMemcpy(prog->step_phases.p, phases.data(), phases.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
      prog->steps_bar.reserve(16);
      CUDA_OK(cudaMemset(prog->steps_bar.p, 0, 16));
      prog->n_phases = (int)phases.size() - 1;
      prog->steps_smem = smem;
      prog->persist_ok = true;
    }
  }
  // root
  prog->root = P.root;
  prog->root_off = OFF(P.root);
  prog->root_plane = int64_t(1) << P.tensors[P.root].labels.size();
  prog->n_open = (int)P.net.open_qubits.size();
  std::vector<int8_t> opos(std::max(1, prog->n_open), 0);
  for (int j = 0; j < prog->n_open; ++j) opos[j] = (int8_t)pos_of(P.tensors[P.root].labels, P.net.open_edge[j]);
  prog->open_pos.reserve(opos.size());
  CUDA_OK(cudaMemcpy(prog->open_pos.p, opos.data(), opos.size(), cudaMemcpyHostToDevice));
  if (!ctx->serial) make_schedule(P, prog.get());
  return prog;
}

static void set_device(tnc_context_s* ctx) { CUDA_OK(cudaSetDevice(ctx->device)); }

// The context's lane streams and fork / join events, created on first use.
static void ensure_lanes(tnc_context_s* ctx) {
  if (ctx->fork_ev) return;
  for (int l = 0; l < kLanes; ++l) {
    CUDA_OK(cudaStreamCreateWithFlags(&ctx->lanes[l], cudaStreamNonBlocking));
    CUDA_OK(cudaEventCreateWithFlags(&ctx->join_ev[l], cudaEventDisableTiming));
  }
  CUDA_OK(cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming));
}

// Reads and clears the device status word (after the stream has drained).
static void check_status(tnc_context_s* ctx) {
  int32_t st = 0;
  CUDA_OK(cudaMemcpy(&st, ctx->status.p, sizeof(st), cudaMemcpyDeviceToHost));
  if (std::getenv("TNC_DEBUG_STATUS")) {
    int32_t w[16];
    CUDA_OK(cudaMemcpy(w, ctx->status.p, sizeof(w), cudaMemcpyDeviceToHost));
    std::fprintf(stderr, "tnc status words:");
    for (int i = 0; i < 16; ++i) std::fprintf(stderr, " %d", w[i]);
    std::fprintf(stderr, "\n");
  }
  if (st != 0) {
    CUDA_OK(cudaMemset(ctx->status.p, 0, sizeof(st)));
    fail(TNC_E_TIMEOUT, "a device-side bounded wait ran out (status " + std::to_string(st) + ")");
  }
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Launch one step of a program (or a one-off step) for n_inst instances.
// Launch indices of a step over a wave of n_inst instances: every instance, or with
// tree-like reuse one per (row, assignment of the result's sliced indices).
static int64_t launch_count(const InstMap& m, int64_t n_inst) {
  if (m.s < 0) return n_inst;
  return (n_inst >> m.s) << __builtin_popcount(m.dep_c);
}

static void run_step(int precision, const StepLaunch& L0, int64_t n_inst, cudaStream_t s, bool reuse = false) {
  StepLaunch L = L0;
  if (!reuse) L.p.im = L.tp.im = InstMap{-1, 0, 0, 0};
  if (L.kind == K_CHAIN) {
    L.grid.z = (unsigned)n_inst;
    CUDA_OK(launch_chain(precision, L.cp, n_inst, s));
    return;
  }
  const bool tc = L.kind == K_TC || L.kind == K_TMA;
  const int64_t nz = launch_count(tc ? L.tp.im : L.p.im, n_inst);
  L.grid.z = (unsigned)nz;
  if (tc) {
    if (L.kind == K_TMA) {
      L.tp.n_inst = (int32_t)nz;
      CUDA_OK(launch_tc_tma(precision, L.tp, L.grid, s));
    }
    else CUDA_OK(launch_tc_gemm(precision, L.tp, L.grid, s));
    if (L.tp.splitk > 1) CUDA_OK(launch_splitk_reduce(precision, L.p, nz, s));
  } else {
    CUDA_OK(launch_generic(precision, L.rm, L.rn, L.p, L.grid, L.smem, s));
    if (L.kind == K_SPLITK) CUDA_OK(launch_splitk_reduce(precision, L.p, nz, s));
  }
  if (reuse)
    for (const auto& m : L.merges)
      CUDA_OK(launch_merge(precision, m.arena, m.inst_stride, m.off, m.plane, m.exps, m.maxabs, m.n_slots, m.slot,
                           m.leaf_r, m.n_leaves, m.lu, m.lv, m.bit, m.im, launch_count(m.im, n_inst), s));
}

}  // namespace tnc

// ------------------------------------------------------------------ C entry points
tnc_status tnc_context_create(int32_t device, tnc_context* out) {
  return guarded([&] {
    if (!out) fail(TNC_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int n = 0;
    CUDA_OK(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) fail(TNC_E_INVALID_ARG, "no such device");
    cudaDeviceProp prop;
    CUDA_OK(cudaGetDeviceProperties(&prop, device));
    if (prop.major != 10 || prop.minor != 3)
      fail(TNC_E_UNSUPPORTED, std::string("this library is built for sm_103 (GB300); device is ") + prop.name);
    auto* c = new tnc_context_s();
    c->device = device;
    c->id = g_ctx_ids++;
    c->sm_count = prop.multiProcessorCount;
    c->total_mem = prop.totalGlobalMem;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete c;
      fail(TNC_E_CUDA, std::string("stream creation failed: ") + cudaGetErrorString(e));
    }
    try {
      c->status.reserve(64);
      CUDA_OK(cudaMemset(c->status.p, 0, 64));
    } catch (...) {
      delete c;
      throw;
    }
    const char* env = std::getenv("TNC_NO_TC");
    c->no_tc = env && env[0] == '1';
    const char* env2 = std::getenv("TNC_NO_TMA");
    c->no_tma = env2 && env2[0] == '1';
    const char* env3 = std::getenv("TNC_NO_PERSIST");
    c->no_persist = env3 && env3[0] == '1';
    const char* env4 = std::getenv("TNC_NO_REUSE");
    c->no_reuse = env4 && env4[0] == '1';
    const char* env5 = std::getenv("TNC_NO_STREAM");
    c->no_stream = env5 && env5[0] == '1';
    const char* env6 = std::getenv("TNC_SERIAL");
    c->serial = env6 && env6[0] == '1';
    const char* env7 = std::getenv("TNC_NO_TC64");
    c->no_tc64 = env7 && env7[0] == '1';
    *out = c;
  });
}

void tnc_context_destroy(tnc_context ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) {
    cudaStreamSynchronize(ctx->stream);
    cudaStreamDestroy(ctx->stream);
  }
  delete ctx;
}

tnc_status tnc_sync(tnc_context ctx) {
  return guarded([&] {
    if (!ctx) fail(TNC_E_INVALID_ARG, "NULL context");
    set_device(ctx);
    CUDA_OK(cudaStreamSynchronize(ctx->stream));
    check_status(ctx);
  });
}

// The program a call of tnc_amplitudes ran, and whether its steps used tree-like reuse.
struct AmpRun {
  std::shared_ptr<DeviceProgram> prog;
  bool reuse = false;
  cudaStream_t stream = nullptr;
};

// Slices [slice_begin, slice_begin + slice_count), or, when `ids` is given, the slice_count
// slice ids listed there (slice_begin unused).
static AmpRun run_amplitudes(tnc_context ctx, tnc_plan plan, const tnc_exec_opts* opts, const uint8_t* bitstrings,
                             int64_t batch, int64_t slice_begin, int64_t slice_count, double* out, void* stream,
                             const int64_t* ids = nullptr) {
  {
    if (!ctx || !plan || !opts || !out) fail(TNC_E_INVALID_ARG, "NULL argument");
    const Plan& P = plan->p;
    const int n = P.net.circ.n;
    const int precision = opts->precision;
    if (precision < TNC_C64 || precision > TNC_CBF16) fail(TNC_E_INVALID_ARG, "bad precision");
    if (batch < 1) fail(TNC_E_INVALID_ARG, "batch must be >= 1");
    // slice ids are int64: with s >= 63 sliced indices the ids [0, 2^63) address the slices
    // whose higher sliced indices are all 0
    const int64_t n_slices = P.sliced.size() >= 63 ? INT64_MAX : int64_t(1) << P.sliced.size();
    if (ids) {
      if (slice_count < 1) fail(TNC_E_INVALID_ARG, "no slice ids");
      for (int64_t t = 0; t < slice_count; ++t)
        if (ids[t] < 0 || ids[t] >= n_slices) fail(TNC_E_INVALID_ARG, "slice id outside [0, 2^s)");
      slice_begin = 0;
    } else if (slice_begin < 0 || slice_count < 1 || slice_count > n_slices - slice_begin) {
      fail(TNC_E_INVALID_ARG, "slice range outside [0, 2^s)");
    }
    const bool all_open = (int)P.net.open_qubits.size() == n;
    if (!bitstrings && !(batch == 1 && all_open)) fail(TNC_E_INVALID_ARG, "bitstrings required");
    std::vector<uint8_t> bits(size_t(batch) * n, 0);
    if (bitstrings) {
      std::memcpy(bits.data(), bitstrings, bits.size());
      for (uint8_t b : bits)
        if (b > 1) fail(TNC_E_INVALID_ARG, "bitstring bytes must be 0 or 1");
    }
    set_device(ctx);
    cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
    const int64_t n_inst = batch * slice_count;
    // wave size
    const size_t eb = elem_bytes(precision);
    const int64_t stride =
        ((opts->fuse && !P.chains.empty() ? P.arena_elems_fused : P.arena_elems) + 63) & ~int64_t(63);
    int64_t W = opts->wave > 0 ? opts->wave : 0;
    if (W == 0) {
      size_t free_b = 0, total_b = 0;
      CUDA_OK(cudaMemGetInfo(&free_b, &total_b));
      const double per_inst = double(stride) * eb * 1.25 + 4096.0;
      const double budget = std::min(double(free_b) * 0.6, 96.0 * (1ull << 30));
      W = std::max<int64_t>(1, (int64_t)(budget / per_inst));
    }
    W = std::min<int64_t>({W, n_inst, 65535});
    const bool fuse = opts->fuse != 0;
    const bool merge = opts->reserved[1] != 0;
    const std::string key = std::to_string(ctx->id) + "/" + std::to_string(precision) + "/" + std::to_string(W) + "/" +
                            std::to_string(fuse ? 1 : 0) + "/" + std::to_string(merge ? 1 : 0);
    auto it = plan->programs.find(key);
    std::shared_ptr<DeviceProgram> prog;
    if (it == plan->programs.end()) {
      // drop programs of other wave sizes on this context before allocating a new arena
      for (auto jt = plan->programs.begin(); jt != plan->programs.end();) {
        if (jt->first.rfind(std::to_string(ctx->id) + "/", 0) == 0) jt = plan->programs.erase(jt);
        else ++jt;
      }
      prog = build_program(ctx, plan, precision, (int)W, fuse, merge);
      plan->programs[key] = prog;
    } else {
      prog = it->second;
      if (prog->leaf_version != P.gate_version) {
        CUDA_OK(cudaStreamSynchronize(s));
        upload_leaves(P, prog->leaf_dst, prog->leaf_src, prog->leaf_desc);
        prog->leaf_version = P.gate_version;
      }
    }
    // instance tables: row-major over (row, slice)
    std::vector<int64_t> inst_slice(n_inst);
    std::vector<int32_t> inst_row(n_inst);
    for (int64_t b = 0; b < batch; ++b)
      for (int64_t t = 0; t < slice_count; ++t) {
        inst_slice[b * slice_count + t] = ids ? ids[t] : slice_begin + t;
        inst_row[b * slice_count + t] = (int32_t)b;
      }
    std::vector<RootSeg> segs;
    std::vector<std::pair<int, int>> wave_segs;  // (first seg, count)
    for (int64_t base = 0; base < n_inst; base += W) {
      const int64_t cnt = std::min<int64_t>(W, n_inst - base);
      const int first = (int)segs.size();
      for (int64_t i = 0; i < cnt; ++i) {
        const int row = inst_row[base + i];
        if (i == 0 || segs.back().row != row) segs.push_back({row, (int32_t)i, (int32_t)i + 1});
        else segs.back().end = (int32_t)i + 1;
      }
      wave_segs.emplace_back(first, (int)segs.size() - first);
    }
    ctx->bits.reserve(std::max<size_t>(1, bits.size()));
    ctx->inst_slice.reserve(n_inst * sizeof(int64_t));
    ctx->inst_row.reserve(n_inst * sizeof(int32_t));
    ctx->segs.reserve(segs.size() * sizeof(RootSeg));
    const int64_t n_out = int64_t(1) << P.net.open_qubits.size();
    ctx->acc.reserve(size_t(batch) * n_out * sizeof(double2));
    CUDA_OK(cudaMemcpyAsync(ctx->bits.p, bits.data(), bits.size(), cudaMemcpyHostToDevice, s));
    CUDA_OK(cudaMemcpyAsync(ctx->inst_slice.p, inst_slice.data(), n_inst * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    CUDA_OK(cudaMemcpyAsync(ctx->inst_row.p, inst_row.data(), n_inst * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CUDA_OK(cudaMemcpyAsync(ctx->segs.p, segs.data(), segs.size() * sizeof(RootSeg), cudaMemcpyHostToDevice, s));
    CUDA_OK(cudaMemsetAsync(ctx->acc.p, 0, size_t(batch) * n_out * sizeof(double2), s));
    const bool prof = opts->profile != 0;
    // one persistent launch for the steps of each wave (requested and the program eligible);
    // profiled, it reports the launch as its first step, kind 8
    const bool persist = opts->reserved[2] != 0 && prog->persist_ok;
    const int n_waves = (int)((n_inst + W - 1) / W);
    // tree-like reuse needs instances laid out as whole rows of every slice
    const bool reuse =
        !ids && prog->reuse_ok && slice_begin == 0 && slice_count == (int64_t(1) << P.sliced.size());
    if (prof) {
      ProfState& ps = ctx->prof;
      ps.valid = false;
      ps.ensure((int)prog->steps.size(), n_waves);
      ps.stream = s;
      ps.flops.assign(prog->steps.size(), 0.0);
      ps.bytes.assign(prog->steps.size(), 0.0);
      ps.kind.assign(prog->steps.size(), 0);
      ps.kernels.assign(prog->steps.size(), 1);
      for (size_t k = 0; k < prog->steps.size(); ++k) {
        const StepLaunch& SL = prog->steps[k];
        const bool tcs = SL.kind == K_TC || SL.kind == K_TMA;
        const double nz = reuse ? double(launch_count(tcs ? SL.tp.im : SL.p.im, n_inst)) : double(n_inst);
        ps.flops[k] = SL.flops * nz;  // what runs: reused results are computed once
        ps.bytes[k] = SL.bytes * nz;
        ps.kind[k] = (SL.kind == K_TMA && SL.tp.persistent) ? 5
                     : ((SL.kind == K_GENERIC || SL.kind == K_SPLITK) && SL.p.stream) ? 7
                                                                                      : SL.kind;
        ps.kernels[k] = (SL.kind == K_SPLITK || ((SL.kind == K_TC || SL.kind == K_TMA) && SL.tp.splitk > 1)) ? 2 : 1;
        if (persist) {
          ps.kind[k] = 8;
          ps.kernels[k] = k == 0 ? 1 : 0;
        }
      }
      CUDA_OK(cudaEventRecord(ps.call_start(), s));
    }
    int w = 0;
    for (int64_t base = 0; base < n_inst; base += W, ++w) {
      const int64_t cnt = std::min<int64_t>(W, n_inst - base);
      // CUDA graph of the wave: the launch sequence depends on the wave's base, size, root
      // segments and the context's buffers; the first call with a key runs eagerly, later
      // calls capture once and replay (Sec. III-A subtasks of a wave in one graph launch)
      std::string gkey;
      if (opts->use_graph && !prof) {
        gkey = std::to_string(base) + "/" + std::to_string(cnt) + "/" + std::to_string(wave_segs[w].first) + "/" +
               std::to_string(wave_segs[w].second) + "/" + std::to_string((uintptr_t)ctx->inst_slice.p) + "/" +
               std::to_string((uintptr_t)ctx->inst_row.p) + "/" + std::to_string((uintptr_t)ctx->bits.p) + "/" +
               std::to_string((uintptr_t)ctx->segs.p) + "/" + std::to_string((uintptr_t)ctx->acc.p) + "/" +
               std::to_string((uintptr_t)s) + "/" + std::to_string(reuse ? 1 : 0) + "/" + std::to_string(persist ? 1 : 0);
        auto git = prog->graphs.find(gkey);
        if (git != prog->graphs.end()) {
          CUDA_OK(cudaGraphLaunch(git->second, s));
          continue;
        }
      }
      const bool capture = !gkey.empty() && prog->graph_seen[gkey]++ > 0;
      if (capture) CUDA_OK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      CUDA_OK(cudaMemsetAsync(prog->maxabs.p, 0, size_t(prog->n_slots) * cnt * sizeof(float), s));
      CUDA_OK(launch_leaf_gather(precision, prog->leaf_desc.as<LeafDesc>(), prog->n_leaves,
                                 prog->leaf_src.as<double2>(), prog->arena.p, prog->inst_stride,
                                 ctx->inst_slice.as<int64_t>(), ctx->inst_row.as<int32_t>(), ctx->bits.as<uint8_t>(),
                                 n, prog->maxabs.as<float>(), prog->exps.as<int32_t>(), prog->n_slots, base, cnt,
                                 prog->leaf_r.as<double2>(), s));
      if (persist) {
        CUDA_OK(cudaMemsetAsync(prog->steps_bar.p, 0, 16, s));
        if (prof) CUDA_OK(cudaEventRecord(ctx->prof.at(w, 0, 0), s));
        CUDA_OK(launch_steps(precision, prog->step_ops.as<StepOp>(), prog->step_phases.as<int32_t>(), prog->n_phases,
                             cnt, reuse ? 1 : 0, prog->steps_bar.as<uint32_t>(), ctx->status.as<int32_t>(),
                             prog->steps_smem, s));
        if (prof) {
          CUDA_OK(cudaEventRecord(ctx->prof.at(w, 0, 1), s));
          for (size_t k = 1; k < prog->steps.size(); ++k) {
            CUDA_OK(cudaEventRecord(ctx->prof.at(w, (int)k, 0), s));
            CUDA_OK(cudaEventRecord(ctx->prof.at(w, (int)k, 1), s));
          }
        }
      } else if (prog->n_lanes > 1) {
        // concurrent branches: fork the lanes from s, follow the schedule, join back into s
        ensure_lanes(ctx);
        CUDA_OK(cudaEventRecord(ctx->fork_ev, s));
        for (int l = 0; l < prog->n_lanes; ++l) CUDA_OK(cudaStreamWaitEvent(ctx->lanes[l], ctx->fork_ev, 0));
        for (size_t k = 0; k < prog->steps.size(); ++k) {
          cudaStream_t ls = ctx->lanes[prog->lane[k]];
          for (int l = 0; l < prog->n_lanes; ++l)
            if (prog->wait_on[k][l] >= 0) CUDA_OK(cudaStreamWaitEvent(ls, prog->done_ev[prog->wait_on[k][l]], 0));
          if (prof) CUDA_OK(cudaEventRecord(ctx->prof.at(w, (int)k, 0), ls));
          run_step(precision, prog->steps[k], cnt, ls, reuse);
          if (prof) CUDA_OK(cudaEventRecord(ctx->prof.at(w, (int)k, 1), ls));
          if (prog->signals[k]) CUDA_OK(cudaEventRecord(prog->done_ev[k], ls));
        }
        for (int l = 0; l < prog->n_lanes; ++l) {
          CUDA_OK(cudaEventRecord(ctx->join_ev[l], ctx->lanes[l]));
          CUDA_OK(cudaStreamWaitEvent(s, ctx->join_ev[l], 0));
        }
      } else {
        for (size_t k = 0; k < prog->steps.size(); ++k) {
          if (prof) CUDA_OK(cudaEventRecord(ctx->prof.at(w, (int)k, 0), s));
          run_step(precision, prog->steps[k], cnt, s, reuse);
          if (prof) CUDA_OK(cudaEventRecord(ctx->prof.at(w, (int)k, 1), s));
        }
      }
      CUDA_OK(launch_inst_scale(prog->leaf_r.as<double2>(), prog->n_leaves, cnt, prog->inst_c.as<double2>(), s));
      CUDA_OK(launch_root_accum(precision, prog->arena.p, prog->inst_stride, prog->root_off, prog->root_plane,
                                prog->open_pos.as<int8_t>(), prog->n_open, ctx->segs.as<RootSeg>() + wave_segs[w].first,
                                wave_segs[w].second, prog->exps.as<int32_t>(), prog->n_slots, prog->root,
                                ctx->acc.as<double2>(), prog->inst_c.as<double2>(),
                                reuse ? prog->root_map : InstMap{-1, 0, 0, 0}, s, reuse ? prog->merged_mask : 0u));
      if (capture) {
        cudaGraph_t g = nullptr;
        CUDA_OK(cudaStreamEndCapture(s, &g));
        cudaGraphExec_t ge = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        CUDA_OK(ie);
        prog->graphs[gkey] = ge;
        CUDA_OK(cudaGraphLaunch(ge, s));
      }
    }
    if (prof) {
      CUDA_OK(cudaEventRecord(ctx->prof.call_end(), s));
      ctx->prof.valid = true;
    }
    const size_t out_bytes = size_t(batch) * n_out * sizeof(double2);
    if (is_device_ptr(out)) {
      CUDA_OK(cudaMemcpyAsync(out, ctx->acc.p, out_bytes, cudaMemcpyDeviceToDevice, s));
    } else {
      CUDA_OK(cudaMemcpyAsync(out, ctx->acc.p, out_bytes, cudaMemcpyDeviceToHost, s));
      CUDA_OK(cudaStreamSynchronize(s));
      check_status(ctx);
    }
    return AmpRun{prog, reuse, s};
  }
}

tnc_status tnc_amplitudes(tnc_context ctx, tnc_plan plan, const tnc_exec_opts* opts, const uint8_t* bitstrings,
                          int64_t batch, int64_t slice_begin, int64_t slice_count, double* out, void* stream) {
  return guarded([&] { run_amplitudes(ctx, plan, opts, bitstrings, batch, slice_begin, slice_count, out, stream); });
}

tnc_status tnc_amplitudes_ids(tnc_context ctx, tnc_plan plan, const tnc_exec_opts* opts, const uint8_t* bitstrings,
                              int64_t batch, const int64_t* slice_ids, int64_t n_ids, double* out, void* stream) {
  return guarded([&] {
    if (!slice_ids) fail(TNC_E_INVALID_ARG, "NULL slice ids");
    run_amplitudes(ctx, plan, opts, bitstrings, batch, 0, n_ids, out, stream, slice_ids);
  });
}

// Times every admissible configuration of each TMA tensor-core step of `prog` at its wave
// size (inputs: the arena as the last wave left it), installs the fastest and records it in
// the cache under the step's shape.
static void tune_program(tnc_context_s* ctx, const Plan& P, DeviceProgram* prog, bool reuse, cudaStream_t s,
                         tnc_tune_info* info) {
  const int64_t W = prog->W;
  const int sbits = (int)P.sliced.size();
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_OK(cudaEventCreate(&e0));
  CUDA_OK(cudaEventCreate(&e1));
  struct Events {
    cudaEvent_t a, b;
    ~Events() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } ev{e0, e1};
  // mean device time of one launch: 3 timed launches after one untimed, 20 more when short
  auto time_launch = [&](const StepLaunch& L) {
    auto timed = [&](int reps) {
      CUDA_OK(cudaEventRecord(e0, s));
      for (int i = 0; i < reps; ++i) run_step(prog->precision, L, W, s, reuse);
      CUDA_OK(cudaEventRecord(e1, s));
      CUDA_OK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CUDA_OK(cudaEventElapsedTime(&ms, e0, e1));
      return double(ms) * 1e-3 / reps;
    };
    run_step(prog->precision, L, W, s, reuse);
    double t = timed(3);
    if (t < 2e-4) t = timed(20);
    return t;
  };
  // steps of one shape share a cache entry, so they are tuned together: a configuration's
  // time is the sum over the steps of that shape
  std::map<std::string, std::vector<size_t>> groups;
  std::vector<std::string> order;
  for (size_t k = 0; k < prog->steps.size(); ++k) {
    const StepLaunch& cur = prog->steps[k];
    if (cur.kind != K_TMA || cur.plan_step < 0) continue;
    const Step& st = P.steps[cur.plan_step];
    const StepLaunch D = tc_launch(ctx, P, prog, cur.plan_step, nullptr);
    const int64_t nz = reuse ? (W >> sbits) << __builtin_popcount((uint32_t)P.tensors[st.c].dep) : W;
    const std::string key = tune_key(prog->precision, P, st, D, nz);
    if (!groups.count(key)) order.push_back(key);
    groups[key].push_back(k);
  }
  int tuned = 0, changed = 0, cands = 0;
  double t_default = 0, t_tuned = 0;
  for (const std::string& key : order) {
    const std::vector<size_t>& ks = groups[key];
    // the launch of step k with choice c (nullptr: heuristics), keeping its instance map
    auto launch_of = [&](size_t k, const TcChoice* c) {
      StepLaunch L = tc_launch(ctx, P, prog, prog->steps[k].plan_step, c);
      L.p.im = L.tp.im = prog->steps[k].tp.im;
      return L;
    };
    // a choice the layouts cannot take (e.g. an output run shorter than 3 once the tile is
    // narrower) is rejected on the host, before anything is launched
    auto group_time = [&](const TcChoice* c) {
      std::vector<StepLaunch> ls;
      try {
        for (size_t k : ks) ls.push_back(launch_of(k, c));
      } catch (const Error&) {
        if (!c) throw;
        return HUGE_VAL;
      }
      double t = 0;
      for (const StepLaunch& L : ls) t += time_launch(L);
      return t;
    };
    const StepLaunch D = launch_of(ks[0], nullptr);
    const int tc_bn = P.steps[D.plan_step].tc_bn;
    // candidates: every tile width down to 64, the persistent kernel where it applies, and
    // splits (powers of two up to the program's partial-sum buffer) with either pipeline depth
    std::vector<TcChoice> cc;
    for (int bn = tc_bn; bn >= 64; bn /= 2) {
      if ((bn <= 128 || D.tp.direct) && !ctx->no_persist) cc.push_back(TcChoice{bn, 1, 1, 0});
      const int64_t kit = int64_t(1) << D.tp.n_ok;
      for (int64_t sp = 1; sp <= std::min<int64_t>(kit, 1024); sp *= 2) {
        if (sp > 1 && size_t(W) * sp * D.tp.planeC * sizeof(float2) > prog->partials.bytes) break;
        if (sp > 1 && kit / sp < 2) break;
        if (bn == 256) {
          cc.push_back(TcChoice{bn, 0, (int)sp, 0});
        } else {
          cc.push_back(TcChoice{bn, 0, (int)sp, 1});
          if (kit / sp <= 8) cc.push_back(TcChoice{bn, 0, (int)sp, 3});
        }
      }
    }
    // the configurations are timed in turn, three rounds, each keeping its fastest round:
    // clocks drift under the power cap, so a sequential sweep would favour whichever ran first
    std::vector<double> tbest(cc.size() + 1, HUGE_VAL);
    for (int round = 0; round < 3; ++round) {
      tbest[0] = std::min(tbest[0], group_time(nullptr));
      for (size_t ci = 0; ci < cc.size(); ++ci) tbest[ci + 1] = std::min(tbest[ci + 1], group_time(&cc[ci]));
    }
    cands += (int)cc.size();
    const double td = tbest[0];
    double best_t = td;
    TcChoice best;
    bool have = false;
    for (size_t ci = 0; ci < cc.size(); ++ci)
      if (tbest[ci + 1] < best_t) best_t = tbest[ci + 1], best = cc[ci], have = true;
    tuned += (int)ks.size();
    t_default += td;
    // keep the heuristics unless a choice is clearly faster (5%: run-to-run noise)
    const bool take = have && best_t < 0.95 * td;
    for (size_t k : ks) prog->steps[k] = launch_of(k, take ? &best : nullptr);
    t_tuned += take ? best_t : td;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (take) {
      changed += (int)ks.size();
      g_tune[key] = best;
    } else {
      g_tune.erase(key);
    }
  }
  // captured waves hold the old launch parameters, and a changed split changes the schedule
  for (auto& kv : prog->graphs) cudaGraphExecDestroy(kv.second);
  prog->graphs.clear();
  prog->graph_seen.clear();
  CUDA_OK(cudaStreamSynchronize(s));
  if (!ctx->serial) make_schedule(P, prog);
  CUDA_OK(cudaStreamSynchronize(s));
  check_status(ctx);
  if (info) {
    info->steps_tuned = tuned;
    info->steps_changed = changed;
    info->candidates = cands;
    info->seconds_default = t_default;
    info->seconds_tuned = t_tuned;
  }
}

tnc_status tnc_autotune(tnc_context ctx, tnc_plan plan, const tnc_exec_opts* opts, const uint8_t* bitstrings,
                        int64_t batch, int64_t slice_begin, int64_t slice_count, tnc_tune_info* info) {
  return guarded([&] {
    if (!ctx || !plan || !opts) fail(TNC_E_INVALID_ARG, "NULL argument");
    if (info) std::memset(info, 0, sizeof(*info));
    if (batch < 1) fail(TNC_E_INVALID_ARG, "batch must be >= 1");
    const int64_t n_out = int64_t(1) << plan->p.net.open_qubits.size();
    std::vector<double> out(size_t(batch) * n_out * 2);
    AmpRun r = run_amplitudes(ctx, plan, opts, bitstrings, batch, slice_begin, slice_count, out.data(), nullptr);
    tune_program(ctx, plan->p, r.prog.get(), r.reuse, r.stream, info);
  });
}

tnc_status tnc_tune_save(const char* path) {
  return guarded([&] {
    if (!path) fail(TNC_E_INVALID_ARG, "NULL path");
    std::string text = "tnc-tune 1\n";
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      for (const auto& kv : g_tune)
        text += kv.first + " " + std::to_string(kv.second.bn) + " " + std::to_string(kv.second.persistent) + " " +
                std::to_string(kv.second.split) + " " + std::to_string(kv.second.stages) + "\n";
    }
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f) fail(TNC_E_IO, std::string("cannot write ") + tmp);
    const bool ok = std::fwrite(text.data(), 1, text.size(), f) == text.size();
    if (std::fclose(f) != 0 || !ok) fail(TNC_E_IO, std::string("cannot write ") + tmp);
    if (std::rename(tmp.c_str(), path) != 0) fail(TNC_E_IO, std::string("cannot rename to ") + path);
  });
}

tnc_status tnc_tune_load(const char* path) {
  return guarded([&] {
    if (!path) fail(TNC_E_INVALID_ARG, "NULL path");
    FILE* f = std::fopen(path, "rb");
    if (!f) fail(TNC_E_IO, std::string("cannot read ") + path);
    std::map<std::string, TcChoice> got;
    char line[512];
    bool header = false, bad = false;
    while (std::fgets(line, sizeof line, f)) {
      if (!header) {
        header = std::strncmp(line, "tnc-tune 1", 10) == 0;
        if (!header) bad = true;
        if (bad) break;
        continue;
      }
      char key[256];
      TcChoice c;
      if (std::sscanf(line, "%255s %d %d %d %d", key, &c.bn, &c.persistent, &c.split, &c.stages) != 5 ||
          (c.bn != 64 && c.bn != 128 && c.bn != 256) || (c.persistent != 0 && c.persistent != 1) || c.split < 0 ||
          c.split > 1024 || (c.split & (c.split - 1)) || (c.stages != 0 && c.stages != 1 && c.stages != 3)) {
        bad = true;
        break;
      }
      got[key] = c;
    }
    std::fclose(f);
    if (bad || !header) fail(TNC_E_IO, std::string("not a tuning cache: ") + path);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto& kv : got) g_tune[kv.first] = kv.second;
  });
}

void tnc_tune_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
}

int64_t tnc_tune_size(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return (int64_t)g_tune.size();
}

tnc_status tnc_contract(tnc_context ctx, int32_t precision, const void* a, int32_t rank_a, const int32_t* labels_a,
                        const void* b, int32_t rank_b, const int32_t* labels_b, void* c, int32_t rank_c,
                        const int32_t* labels_c, int32_t* c_exp2, void* stream) {
  return guarded([&] {
    if (!ctx || !a || !b || !c || !c_exp2) fail(TNC_E_INVALID_ARG, "NULL argument");
    if (precision < TNC_C64 || precision > TNC_CBF16) fail(TNC_E_INVALID_ARG, "bad precision");
    if (rank_a < 0 || rank_b < 0 || rank_c < 0 || rank_a > 32 || rank_b > 32 || rank_c > 32)
      fail(TNC_E_INVALID_ARG, "ranks must be in [0, 32]");
    if ((rank_a && !labels_a) || (rank_b && !labels_b) || (rank_c && !labels_c)) fail(TNC_E_INVALID_ARG, "NULL labels");
    std::vector<int> la(labels_a, labels_a + rank_a), lb(labels_b, labels_b + rank_b), lc(labels_c, labels_c + rank_c);
    auto distinct = [](std::vector<int> v) {
      std::sort(v.begin(), v.end());
      return std::adjacent_find(v.begin(), v.end()) == v.end();
    };
    if (!distinct(la) || !distinct(lb) || !distinct(lc)) fail(TNC_E_INVALID_ARG, "repeated label within a tensor");
    std::vector<int> fr;
    for (int x : la)
      if (std::find(lb.begin(), lb.end(), x) == lb.end()) fr.push_back(x);
    for (int x : lb)
      if (std::find(la.begin(), la.end(), x) == la.end()) fr.push_back(x);
    std::vector<int> s1 = fr, s2 = lc;
    std::sort(s1.begin(), s1.end());
    std::sort(s2.begin(), s2.end());
    if (s1 != s2) fail(TNC_E_INVALID_ARG, "C's labels must be exactly the free labels of A and B");
    set_device(ctx);
    cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
    int kind = K_GENERIC;
    TileSpec t = tile_for(la, lb, lc, 1, kind);
    StepLaunch L = make_launch(t, kind, la, lb, lc);
    make_stream(L, elem_bytes(precision), ctx->no_stream);
    // per-launch events (read with tnc_profile_read): the contraction and the whole call
    ProfState& ps = ctx->prof;
    ps.valid = false;
    ps.ensure(1, 1);
    CUDA_OK(cudaEventRecord(ps.call_start(), s));
    ctx->scratch.reserve(256);
    float* mx = ctx->scratch.as<float>();
    int32_t* ex = reinterpret_cast<int32_t*>(ctx->scratch.as<char>() + 64);
    CUDA_OK(cudaMemsetAsync(ctx->scratch.p, 0, 256, s));
    const size_t eb = elem_bytes(precision);
    CUDA_OK(launch_maxabs(precision, a, int64_t(2) << rank_a, mx + 0, s));
    CUDA_OK(launch_maxabs(precision, b, int64_t(2) << rank_b, mx + 1, s));
    L.p.A = a;
    L.p.B = b;
    L.p.C = c;
    L.p.strideA = L.p.strideB = L.p.strideC = 0;
    L.p.maxabs = mx;
    L.p.exps = ex;
    L.p.n_slots = 3;
    L.p.slotA = 0;
    L.p.slotB = 1;
    L.p.slotC = 2;
    if (L.kind == K_SPLITK) {
      ctx->partials.reserve(size_t(L.p.splitk) * L.p.planeC * sizeof(float2));
      L.p.partials = ctx->partials.as<float2>();
    }
    TileSpec tct;
    bool swap = false;
    int bn = 128, bk = 64;
    bool ttgt = false;
    std::vector<int> la2, lb2, lc2;
    PermParams perm_a, perm_b, perm_c;
    // complex64 takes the 3xTF32 kernel on operands already in the TMA layouts
    const bool tc_ok = !ctx->no_tc && !ctx->no_tma && (precision != TNC_C64 || !ctx->no_tc64);
    const bool tma_a = tc_ok && tma_tile_from_layout(la, lb, lc, tct, bn, bk);
    const bool tma_b = !tma_a && tc_ok && tma_tile_from_layout(lb, la, lc, tct, bn, bk);
    if (tma_a || tma_b) {
      const std::vector<int>& ra = tma_a ? la : lb;
      const std::vector<int>& rb = tma_a ? lb : la;
      if (precision == TNC_C64 && bn == 256) {
        tct.No.insert(tct.No.begin(), tct.Nt.begin() + 7, tct.Nt.end());
        tct.Nt.resize(7);
        bn = 128;
      }
      make_tc_launch(L, tct, ra, rb, lc, precision, bn, bk, 1);
      float2* part = nullptr;
      if (L.tp.splitk > 1) {
        ctx->partials.reserve(size_t(L.tp.splitk) * L.tp.planeC * sizeof(float2));
        part = ctx->partials.as<float2>();
      }
      bind_tc(L, tma_a ? a : b, tma_a ? b : a, c, 0, mx, ex, 3, tma_a ? 0 : 1, tma_a ? 1 : 0, 2, ctx->status.as<int32_t>(),
              part);
      const int kt = bk == 32 ? 5 : 4;
      encode_tile_map(&L.tp.tmA, L.tp.A, (int)ra.size(), kt, 128, 0, 1, eb);
      encode_tile_map(&L.tp.tmB, L.tp.B, (int)rb.size(), kt, bn, 0, 1, eb);
      L.kind = K_TMA;
      if (ctx->no_persist || precision == TNC_C64) L.tp.persistent = 0;
    } else if (precision != TNC_C64 && !ctx->no_tc && !ctx->no_tma &&
               ttgt_layouts(la.size() >= lb.size() ? la : lb, la.size() >= lb.size() ? lb : la, la2, lb2, lc2) &&
               ttgt_fits(la2.size(), lb2.size(), lc2.size(), eb)) {
      // TTGT (Sec. V-A, Sec. V-B): permute the operands into the layouts the TMA kernel
      // loads, contract into a tile-first C, permute C into the requested layout
      ttgt = true;
      const bool sw = la.size() < lb.size();
      const void* ra = sw ? b : a;
      const void* rb = sw ? a : b;
      const std::vector<int>& oa = sw ? lb : la;
      const std::vector<int>& ob = sw ? la : lb;
      const size_t na = (size_t(2) << la2.size()) * eb, nb2 = (size_t(2) << lb2.size()) * eb,
                   nc = (size_t(2) << lc2.size()) * eb;
      ctx->ttgt.reserve(na + nb2 + nc + 1024);
      char* base = ctx->ttgt.as<char>();
      char* a2 = base;
      char* b2 = base + ((na + 255) & ~size_t(255));
      char* c2 = b2 + ((nb2 + 255) & ~size_t(255));
      perm_a = make_permute(oa, la2);
      perm_a.in = ra;
      perm_a.out = a2;
      perm_b = make_permute(ob, lb2);
      perm_b.in = rb;
      perm_b.out = b2;
      perm_c = make_permute(lc2, lc);
      perm_c.in = c2;
      perm_c.out = c;
      if (!tma_tile_from_layout(la2, lb2, lc2, tct, bn, bk)) fail(TNC_E_PLAN, "TTGT layouts do not fit the TMA tile");
      make_tc_launch(L, tct, la2, lb2, lc2, precision, bn, bk, 1);
      float2* part = nullptr;
      if (L.tp.splitk > 1) {
        ctx->partials.reserve(size_t(L.tp.splitk) * L.tp.planeC * sizeof(float2));
        part = ctx->partials.as<float2>();
      }
      bind_tc(L, a2, b2, c2, 0, mx, ex, 3, sw ? 1 : 0, sw ? 0 : 1, 2, ctx->status.as<int32_t>(), part);
      const int kt = bk == 32 ? 5 : 4;
      encode_tile_map(&L.tp.tmA, L.tp.A, (int)la2.size(), kt, 128, 0, 1);
      encode_tile_map(&L.tp.tmB, L.tp.B, (int)lb2.size(), kt, bn, 0, 1);
      L.kind = K_TMA;
      if (ctx->no_persist) L.tp.persistent = 0;
    } else if (precision != TNC_C64 && !ctx->no_tc && tc_tile_for(la, lb, lc, tct, swap, bn, bk)) {
      make_tc_launch(L, tct, swap ? lb : la, swap ? la : lb, lc, precision, bn, bk, 1);
      float2* part = nullptr;
      if (L.tp.splitk > 1) {
        ctx->partials.reserve(size_t(L.tp.splitk) * L.tp.planeC * sizeof(float2));
        part = ctx->partials.as<float2>();
      }
      bind_tc(L, swap ? b : a, swap ? a : b, c, 0, mx, ex, 3, swap ? 1 : 0, swap ? 0 : 1, 2, ctx->status.as<int32_t>(),
              part);
    }
    {
      int common = 0;
      for (int x : la) common += std::find(lb.begin(), lb.end(), x) != lb.end();
      ps.flops.assign(1, 8.0 * std::ldexp(1.0, rank_a + rank_b - common));
      ps.bytes.assign(1, (std::ldexp(1.0, rank_a) + std::ldexp(1.0, rank_b) + std::ldexp(1.0, rank_c)) * 2.0 * double(eb));
      ps.kind.assign(1, ttgt ? 6
                           : (L.kind == K_TMA && L.tp.persistent) ? 5
                           : ((L.kind == K_GENERIC || L.kind == K_SPLITK) && L.p.stream) ? 7
                                                                                          : L.kind);
      ps.kernels.assign(1, (L.kind == K_SPLITK || ((L.kind == K_TC || L.kind == K_TMA) && L.tp.splitk > 1)) ? 2 : 1);
      if (ttgt) ps.kernels[0] += 3;
    }
    CUDA_OK(cudaEventRecord(ps.at(0, 0, 0), s));
    if (ttgt) {
      CUDA_OK(launch_permute(precision, perm_a, s));
      CUDA_OK(launch_permute(precision, perm_b, s));
    }
    run_step(precision, L, 1, s);
    if (ttgt) CUDA_OK(launch_permute(precision, perm_c, s));
    CUDA_OK(cudaEventRecord(ps.at(0, 0, 1), s));
    CUDA_OK(cudaEventRecord(ps.call_end(), s));
    ps.valid = true;
    int32_t e = 0;
    CUDA_OK(cudaMemcpyAsync(&e, ex + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CUDA_OK(cudaStreamSynchronize(s));
    check_status(ctx);
    *c_exp2 = e;
  });
}

tnc_status tnc_profile_read(tnc_context ctx, double* ms, int32_t* launches, double* flops, double* bytes,
                            int32_t* kind, int32_t cap, int32_t* n) {
  return guarded([&] {
    if (!ctx || !n) fail(TNC_E_INVALID_ARG, "NULL argument");
    ProfState& ps = ctx->prof;
    if (!ps.valid) fail(TNC_E_INVALID_ARG, "no profiled call on this context");
    *n = ps.n_steps;
    if (cap < ps.n_steps || !ms || !launches || !flops || !bytes || !kind) fail(TNC_E_INVALID_ARG, "cap too small");
    set_device(ctx);
    CUDA_OK(cudaEventSynchronize(ps.call_end()));
    for (int s = 0; s < ps.n_steps; ++s) {
      double t = 0;
      for (int w = 0; w < ps.waves; ++w) {
        float x = 0;
        CUDA_OK(cudaEventElapsedTime(&x, ps.at(w, s, 0), ps.at(w, s, 1)));
        t += x;
      }
      ms[s] = t;
      launches[s] = ps.waves * ps.kernels[s];
      flops[s] = ps.flops[s];
      bytes[s] = ps.bytes[s];
      kind[s] = ps.kind[s];
    }
    float tot = 0;
    CUDA_OK(cudaEventElapsedTime(&tot, ps.call_start(), ps.call_end()));
    ms[ps.n_steps] = tot;
  });
}

// ------------------------------------------------------------------ allocation-free contraction
// tnc_contract_noalloc: the same single contraction as tnc_contract on the FP32 SIMT kernels
// (generic tile, or the split-K GEPDOT pair of kernels), for callers that must not allocate
// device memory.  Its scratch -- the per-operand max/exponent slots and the split-K partial
// sums -- lives in one file-scope device array instead of a context's cudaMalloc'd buffers.
namespace tnc {
namespace {
constexpr size_t kNoAllocScratchBytes = size_t(4) << 20;  // 4 MiB per device, held until exit
constexpr size_t kNoAllocSlotBytes = 256;                 // maxabs[3], exps[3] at the front
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
std::map<int, void*> g_noalloc_ptr;  // device ordinal -> device address of the array

// Device address of the array on the current device; looked up once per device (the
// host-side name of a __device__ array is not a device address).
void* noalloc_scratch(int* device_out) {
  int dev = -1;
  CUDA_OK(cudaGetDevice(&dev));
  *device_out = dev;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  auto it = g_noalloc_ptr.find(dev);
  if (it != g_noalloc_ptr.end()) return it->second;
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    fail(TNC_E_CUDA, std::string("cudaGetSymbolAddress(g_noalloc_scratch) failed: ") + cudaGetErrorString(e));
  g_noalloc_ptr[dev] = p;
  return p;
}
}  // namespace
}  // namespace tnc

tnc_status tnc_contract_noalloc(int32_t precision, const void* a, int32_t rank_a, const int32_t* labels_a,
                                const void* b, int32_t rank_b, const int32_t* labels_b, void* c, int32_t rank_c,
                                const int32_t* labels_c, int32_t* c_exp2, void* stream) {
  return guarded([&] {
    if (!a || !b || !c || !c_exp2) fail(TNC_E_INVALID_ARG, "NULL argument");
    if (precision < TNC_C64 || precision > TNC_CBF16) fail(TNC_E_INVALID_ARG, "bad precision");
    if (rank_a < 0 || rank_b < 0 || rank_c < 0 || rank_a > 32 || rank_b > 32 || rank_c > 32)
      fail(TNC_E_INVALID_ARG, "ranks must be in [0, 32]");
    if ((rank_a && !labels_a) || (rank_b && !labels_b) || (rank_c && !labels_c)) fail(TNC_E_INVALID_ARG, "NULL labels");
    std::vector<int> la(labels_a, labels_a + rank_a), lb(labels_b, labels_b + rank_b), lc(labels_c, labels_c + rank_c);
    auto distinct = [](std::vector<int> v) {
      std::sort(v.begin(), v.end());
      return std::adjacent_find(v.begin(), v.end()) == v.end();
    };
    if (!distinct(la) || !distinct(lb) || !distinct(lc)) fail(TNC_E_INVALID_ARG, "repeated label within a tensor");
    std::vector<int> fr;
    for (int x : la)
      if (std::find(lb.begin(), lb.end(), x) == lb.end()) fr.push_back(x);
    for (int x : lb)
      if (std::find(la.begin(), la.end(), x) == la.end()) fr.push_back(x);
    std::vector<int> s1 = fr, s2 = lc;
    std::sort(s1.begin(), s1.end());
    std::sort(s2.begin(), s2.end());
    if (s1 != s2) fail(TNC_E_INVALID_ARG, "C's labels must be exactly the free labels of A and B");
    int dev = -1;
    char* base = static_cast<char*>(noalloc_scratch(&dev));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int kind = K_GENERIC;
    TileSpec t = tile_for(la, lb, lc, 1, kind);
    // fewer splits over K (same tiles, longer K range per CTA) until the FP32 partial sums
    // fit the static array (the split policy's one wave of 304 CTAs over at most 2^10
    // outputs needs 2.4 MiB, so this only guards)
    const size_t room = kNoAllocScratchBytes - kNoAllocSlotBytes;
    while (t.splitk > 1 && size_t(t.splitk) * (size_t(1) << lc.size()) * sizeof(float2) > room) t.splitk /= 2;
    if (t.splitk == 1) kind = K_GENERIC;
    StepLaunch L = make_launch(t, kind, la, lb, lc);
    make_stream(L, elem_bytes(precision), false);
    if (L.kind == K_SPLITK) {
      const size_t need = size_t(L.p.splitk) * size_t(L.p.planeC) * sizeof(float2);
      if (need > kNoAllocScratchBytes - kNoAllocSlotBytes)
        fail(TNC_E_INVALID_ARG, "tnc_contract_noalloc: this contraction needs " + std::to_string(need) +
                                    " bytes of split-K scratch; the static array holds " +
                                    std::to_string(kNoAllocScratchBytes - kNoAllocSlotBytes));
      L.p.partials = reinterpret_cast<float2*>(base + kNoAllocSlotBytes);
    }
    float* mx = reinterpret_cast<float*>(base);
    int32_t* ex = reinterpret_cast<int32_t*>(base + 64);
    // the slots are shared by every call: clear what must start at zero
    CUDA_OK(cudaMemsetAsync(base, 0, kNoAllocSlotBytes, s));
    CUDA_OK(launch_maxabs(precision, a, int64_t(2) << rank_a, mx + 0, s));
    CUDA_OK(launch_maxabs(precision, b, int64_t(2) << rank_b, mx + 1, s));
    L.p.A = a;
    L.p.B = b;
    L.p.C = c;
    L.p.strideA = L.p.strideB = L.p.strideC = 0;
    L.p.maxabs = mx;
    L.p.exps = ex;
    L.p.n_slots = 3;
    L.p.slotA = 0;
    L.p.slotB = 1;
    L.p.slotC = 2;
    run_step(precision, L, 1, s);
    int32_t e = 0;
    CUDA_OK(cudaMemcpyAsync(&e, ex + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CUDA_OK(cudaStreamSynchronize(s));
    *c_exp2 = e;
  });
}

// ------------------------------------------------------------------ adjoint contraction
// Reverse-mode walk of the contraction tree (complex64 arithmetic, FP64 accumulation over
// instances).  Forward intermediates are kept (one arena slot each); every tensor X gets
// an adjoint slot X' = dL/dX.  For a forward step C = A * B the backward steps are
//   A' = C' * B   (summed over B's free labels, result in A's layout),
//   B' = A * C'   (summed over A's free labels, result in B's layout),
// the same pairwise contraction as the forward steps (Sec. II-A).  The leaves' adjoints
// are read back, placed at their fixed (sliced / output) leg values and summed in FP64;
// the host then applies the chain rule from leaves to gates.
tnc_status tnc_adjoint(tnc_context ctx, tnc_plan plan, const tnc_exec_opts* opts, const uint8_t* bitstrings,
                       int64_t batch, const double* weights, double* env_out, double* amp_out, void* stream) {
  return guarded([&] {
    if (!ctx || !plan || !weights || !env_out) fail(TNC_E_INVALID_ARG, "NULL argument");
    (void)opts;
    const Plan& P = plan->p;
    const int n = P.net.circ.n;
    if (batch < 1) fail(TNC_E_INVALID_ARG, "batch must be >= 1");
    const bool all_open = (int)P.net.open_qubits.size() == n;
    if (!bitstrings && !(batch == 1 && all_open)) fail(TNC_E_INVALID_ARG, "bitstrings required");
    std::vector<uint8_t> bits(size_t(batch) * n, 0);
    if (bitstrings) {
      std::memcpy(bits.data(), bitstrings, bits.size());
      for (uint8_t b : bits)
        if (b > 1) fail(TNC_E_INVALID_ARG, "bitstring bytes must be 0 or 1");
    }
    set_device(ctx);
    cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
    const int T = (int)P.tensors.size();
    const int L = (int)P.net.leaves.size();
    const int n_open = (int)P.net.open_qubits.size();
    const int64_t n_out = int64_t(1) << n_open;
    if (P.sliced.size() > 30) fail(TNC_E_UNSUPPORTED, "tnc_adjoint sums over every slice: at most 30 sliced indices");
    const int64_t n_slices = int64_t(1) << P.sliced.size();
    const int64_t n_inst = batch * n_slices;
    // Forward intermediates kept for the backward pass.  Under a memory budget the largest
    // ones are dropped and recomputed from their two children just before the backward step
    // that reads them; a dropped tensor's children and its consumer's output stay stored, so
    // one recomputation (the original forward step) always suffices.
    auto elems = [&](int t) { return ((int64_t(2) << P.tensors[t].labels.size()) + 63) & ~int64_t(63); };
    std::vector<int> consumer(T, -1);
    for (size_t k = 0; k < P.steps.size(); ++k) consumer[P.steps[k].a] = consumer[P.steps[k].b] = (int)k;
    std::vector<char> dropped(T, 0);
    const int64_t budget = int64_t(std::max(0, opts ? opts->reserved[0] : 0)) << 20;  // bytes per instance
    if (budget > 0) {
      int64_t kept = 0;
      for (int t = L; t < T; ++t) kept += elems(t) * 4;
      std::vector<int> cand;
      for (int t = L; t < T; ++t)
        if (t != P.root && consumer[t] >= 0) cand.push_back(t);
      std::stable_sort(cand.begin(), cand.end(), [&](int x, int y) { return elems(x) > elems(y); });
      for (int x : cand) {
        if (kept <= budget) break;
        const Step& px = P.steps[x - L];
        const int parent = L + consumer[x];
        if (dropped[px.a] || dropped[px.b] || dropped[parent]) continue;
        dropped[x] = 1;
        kept -= elems(x) * 4;
      }
    }
    // arena: kept forward tensors, then a pool for the dropped ones (forward liveness, first
    // fit; during the backward pass it holds the recomputed operands), then the adjoint
    // leaves (contiguous, for one read-back copy), then the other adjoints
    std::vector<int64_t> off(2 * T), off_b(T);
    int64_t top = 0;
    auto take = [&](int slot, int rank) {
      off[slot] = top;
      top += ((int64_t(2) << rank) + 63) & ~int64_t(63);
    };
    for (int t = 0; t < T; ++t)
      if (!dropped[t]) take(t, (int)P.tensors[t].labels.size());
    {
      const int64_t pool = top;
      std::vector<std::pair<int64_t, int64_t>> live;  // (offset, size) with end step
      std::vector<int> dend;
      int64_t pool_top = 0, biggest = 0;
      for (int t = L; t < T; ++t) {
        if (!dropped[t]) continue;
        const int born = t - L, dies = consumer[t];
        // first fit among slots whose tenants died before this one is born
        std::vector<std::pair<int64_t, int64_t>> busy;
        for (size_t i = 0; i < live.size(); ++i)
          if (dend[i] >= born) busy.push_back(live[i]);
        std::sort(busy.begin(), busy.end());
        int64_t at = 0;
        for (auto& b : busy) {
          if (at + elems(t) <= b.first) break;
          at = std::max(at, b.first + b.second);
        }
        off[t] = pool + at;
        live.push_back({at, elems(t)});
        dend.push_back(dies);
        pool_top = std::max(pool_top, at + elems(t));
        biggest = std::max(biggest, elems(t));
      }
      // backward: a step reads at most two dropped operands, recomputed into two fixed slots
      int next_slot = 0;
      for (int t = 0; t < T; ++t) off_b[t] = off[t];
      for (size_t k = P.steps.size(); k-- > 0;) {
        next_slot = 0;
        for (int t : {P.steps[k].a, P.steps[k].b})
          if (dropped[t]) off_b[t] = pool + (next_slot++) * biggest;
      }
      top = pool + std::max(pool_top, 2 * biggest);
    }
    const int64_t adj_leaf_begin = top;
    for (int t = 0; t < L; ++t) take(T + t, (int)P.tensors[t].labels.size());
    const int64_t adj_leaf_end = top;
    for (int t = L; t < T; ++t) take(T + t, (int)P.tensors[t].labels.size());
    const int64_t stride = (top + 63) & ~int64_t(63);
    size_t free_b = 0, total_b = 0;
    CUDA_OK(cudaMemGetInfo(&free_b, &total_b));
    int64_t W = std::max<int64_t>(1, (int64_t)(std::min(double(free_b) * 0.5, 64.0 * (1ull << 30)) / (double(stride) * 4 * 1.1)));
    W = std::min<int64_t>({W, n_inst, 4096});
    DevBuf arena, maxabs, exps, leaf_src, leaf_desc, partials, open_pos, wdev, erow;
    arena.reserve(size_t(stride) * 4 * W + 256);
    maxabs.reserve(size_t(2 * T) * W * sizeof(float));
    exps.reserve(size_t(2 * T) * W * sizeof(int32_t));
    {
      std::vector<int64_t> dst(L);
      for (int i = 0; i < L; ++i) dst[i] = off[i];
      upload_leaves(P, dst, leaf_src, leaf_desc);
    }
    // launches
    std::vector<StepLaunch> fwd, bwd;
    size_t partial_elems = 0;
    auto bind = [&](StepLaunch& Lh, int sa, int sb, int sc, bool backward = false) {
      char* base = arena.as<char>();
      auto at = [&](int slot) { return (backward && slot < T) ? off_b[slot] : off[slot]; };
      Lh.p.A = base + at(sa) * 4;
      Lh.p.B = base + at(sb) * 4;
      Lh.p.C = base + at(sc) * 4;
      Lh.p.strideA = Lh.p.strideB = Lh.p.strideC = stride;
      Lh.p.n_slots = 2 * T;
      Lh.p.slotA = sa;
      Lh.p.slotB = sb;
      Lh.p.slotC = sc;
      if (Lh.kind == K_SPLITK) partial_elems = std::max(partial_elems, size_t(W) * Lh.p.splitk * Lh.p.planeC);
    };
    for (const Step& st : P.steps) {
      StepLaunch Lh = make_launch(st.tile, st.kind, P.tensors[st.a].labels, P.tensors[st.b].labels, P.tensors[st.c].labels);
      bind(Lh, st.a, st.b, st.c);
      fwd.push_back(Lh);
    }
    for (size_t k = P.steps.size(); k-- > 0;) {
      const Step& st = P.steps[k];
      const auto& la = P.tensors[st.a].labels;
      const auto& lb = P.tensors[st.b].labels;
      const auto& lc = P.tensors[st.c].labels;
      // dropped operands: rerun their forward step into the backward slots (same kernels,
      // same inputs: the same values, max and exponent as in the forward pass)
      for (int t : {st.a, st.b}) {
        if (!dropped[t]) continue;
        const Step& pt = P.steps[t - L];
        StepLaunch Lr = make_launch(pt.tile, pt.kind, P.tensors[pt.a].labels, P.tensors[pt.b].labels,
                                    P.tensors[pt.c].labels);
        bind(Lr, pt.a, pt.b, pt.c, true);
        bwd.push_back(Lr);
      }
      int kind = K_GENERIC;
      TileSpec ta = tile_for(lc, lb, la, (int)W, kind);  // A' = C' * B
      StepLaunch La = make_launch(ta, kind, lc, lb, la);
      bind(La, T + st.c, st.b, T + st.a, true);
      bwd.push_back(La);
      kind = K_GENERIC;
      TileSpec tb = tile_for(la, lc, lb, (int)W, kind);  // B' = A * C'
      StepLaunch Lb = make_launch(tb, kind, la, lc, lb);
      bind(Lb, st.a, T + st.c, T + st.b, true);
      bwd.push_back(Lb);
    }
    if (partial_elems) {
      partials.reserve(partial_elems * sizeof(float2));
      for (auto* v : {&fwd, &bwd})
        for (auto& Lh : *v)
          if (Lh.kind == K_SPLITK) Lh.p.partials = partials.as<float2>();
    }
    for (auto* v : {&fwd, &bwd})
      for (auto& Lh : *v) {
        Lh.p.maxabs = maxabs.as<float>();
        Lh.p.exps = exps.as<int32_t>();
      }
    const int root = P.root;
    std::vector<int8_t> opos(std::max(1, n_open), 0);
    for (int j = 0; j < n_open; ++j) opos[j] = (int8_t)pos_of(P.tensors[root].labels, P.net.open_edge[j]);
    open_pos.reserve(opos.size());
    CUDA_OK(cudaMemcpy(open_pos.p, opos.data(), opos.size(), cudaMemcpyHostToDevice));
    // weights and their per-row exponents (stored cotangents below 1 in magnitude)
    std::vector<int32_t> er(batch, 0);
    for (int64_t b = 0; b < batch; ++b) {
      double m = 0;
      for (int64_t o = 0; o < n_out; ++o)
        m = std::max({m, std::fabs(weights[2 * (b * n_out + o)]), std::fabs(weights[2 * (b * n_out + o) + 1])});
      int ex = 0;
      if (m > 0) std::frexp(m, &ex);
      er[b] = ex;
    }
    wdev.reserve(size_t(batch) * n_out * sizeof(double2));
    erow.reserve(size_t(batch) * sizeof(int32_t));
    CUDA_OK(cudaMemcpy(wdev.p, weights, size_t(batch) * n_out * sizeof(double2), cudaMemcpyHostToDevice));
    CUDA_OK(cudaMemcpy(erow.p, er.data(), er.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    // instance tables (row-major over (row, slice)) and root segments per wave
    std::vector<int64_t> inst_slice(n_inst);
    std::vector<int32_t> inst_row(n_inst);
    for (int64_t b = 0; b < batch; ++b)
      for (int64_t t = 0; t < n_slices; ++t) {
        inst_slice[b * n_slices + t] = t;
        inst_row[b * n_slices + t] = (int32_t)b;
      }
    ctx->bits.reserve(std::max<size_t>(1, bits.size()));
    ctx->inst_slice.reserve(n_inst * sizeof(int64_t));
    ctx->inst_row.reserve(n_inst * sizeof(int32_t));
    CUDA_OK(cudaMemcpy(ctx->bits.p, bits.data(), bits.size(), cudaMemcpyHostToDevice));
    CUDA_OK(cudaMemcpy(ctx->inst_slice.p, inst_slice.data(), n_inst * sizeof(int64_t), cudaMemcpyHostToDevice));
    CUDA_OK(cudaMemcpy(ctx->inst_row.p, inst_row.data(), n_inst * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (amp_out) ctx->acc.reserve(size_t(batch) * n_out * sizeof(double2));
    if (amp_out) CUDA_OK(cudaMemsetAsync(ctx->acc.p, 0, size_t(batch) * n_out * sizeof(double2), s));
    // FP64 leaf environments (full leaf tensors, fixed legs included)
    std::vector<SmallTensor> leaf_env(L);
    for (int i = 0; i < L; ++i) {
      leaf_env[i].labels = P.net.leaves[i].t.labels;
      leaf_env[i].data.assign(P.net.leaves[i].t.data.size(), cd(0, 0));
    }
    const int64_t leaf_region = adj_leaf_end - adj_leaf_begin;
    std::vector<float> host_leaf(size_t(leaf_region) * W);
    std::vector<int32_t> host_exp(size_t(2 * T) * W);
    std::vector<RootSeg> segs;
    for (int64_t base = 0; base < n_inst; base += W) {
      const int64_t cnt = std::min<int64_t>(W, n_inst - base);
      CUDA_OK(cudaMemsetAsync(maxabs.p, 0, size_t(2 * T) * cnt * sizeof(float), s));
      CUDA_OK(launch_leaf_gather(TNC_C64, leaf_desc.as<LeafDesc>(), L, leaf_src.as<double2>(), arena.p, stride,
                                 ctx->inst_slice.as<int64_t>(), ctx->inst_row.as<int32_t>(), ctx->bits.as<uint8_t>(), n,
                                 maxabs.as<float>(), exps.as<int32_t>(), 2 * T, base, cnt, nullptr, s));
      for (const StepLaunch& Lh : fwd) run_step(TNC_C64, Lh, cnt, s);
      if (amp_out) {
        segs.clear();
        for (int64_t i = 0; i < cnt; ++i) {
          const int row = inst_row[base + i];
          if (i == 0 || segs.back().row != row) segs.push_back({row, (int32_t)i, (int32_t)i + 1});
          else segs.back().end = (int32_t)i + 1;
        }
        ctx->segs.reserve(segs.size() * sizeof(RootSeg));
        CUDA_OK(cudaMemcpyAsync(ctx->segs.p, segs.data(), segs.size() * sizeof(RootSeg), cudaMemcpyHostToDevice, s));
        CUDA_OK(launch_root_accum(TNC_C64, arena.p, stride, off[root], int64_t(1) << P.tensors[root].labels.size(),
                                  open_pos.as<int8_t>(), n_open, ctx->segs.as<RootSeg>(), (int)segs.size(),
                                  exps.as<int32_t>(), 2 * T, root, ctx->acc.as<double2>(), nullptr, InstMap{-1, 0, 0, 0},
                                  s));
      }
      CUDA_OK(launch_adj_root_init(arena.as<float>(), stride, off[T + root], int64_t(1) << P.tensors[root].labels.size(),
                                   open_pos.as<int8_t>(), n_open, ctx->inst_row.as<int32_t>(), base, cnt,
                                   wdev.as<double2>(), erow.as<int32_t>(), maxabs.as<float>(), exps.as<int32_t>(), 2 * T,
                                   T + root, s));
      for (const StepLaunch& Lh : bwd) run_step(TNC_C64, Lh, cnt, s);
      // read back the leaves' adjoints and exponents
      CUDA_OK(cudaMemcpy2DAsync(host_leaf.data(), size_t(leaf_region) * 4, arena.as<char>() + adj_leaf_begin * 4,
                                size_t(stride) * 4, size_t(leaf_region) * 4, (size_t)cnt, cudaMemcpyDeviceToHost, s));
      CUDA_OK(cudaMemcpyAsync(host_exp.data(), exps.p, size_t(2 * T) * cnt * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      CUDA_OK(cudaStreamSynchronize(s));
      check_status(ctx);
      for (int64_t i = 0; i < cnt; ++i) {
        const int64_t g = base + i;
        const int64_t slice = inst_slice[g];
        const int row = inst_row[g];
        for (int l = 0; l < L; ++l) {
          const int rk = (int)P.tensors[l].labels.size();
          const int64_t nrk = int64_t(1) << rk;
          const float* v = host_leaf.data() + size_t(i) * leaf_region + (off[T + l] - adj_leaf_begin);
          const double sc = std::ldexp(1.0, host_exp[size_t(i) * 2 * T + T + l]);
          const auto& fx = P.leaf_fix[l];
          const int rf = (int)P.net.leaves[l].t.labels.size();
          for (int64_t x = 0; x < nrk; ++x) {
            int64_t full = 0;
            int fb = 0;
            size_t f = 0;
            for (int pos = 0; pos < rf; ++pos) {
              int bit;
              if (f < fx.size() && fx[f].pos == pos) {
                bit = fx[f].kind == 0 ? int((slice >> fx[f].index) & 1) : int(bits[size_t(row) * n + fx[f].index]);
                ++f;
              } else {
                bit = int((x >> fb) & 1);
                ++fb;
              }
              full |= int64_t(bit) << pos;
            }
            leaf_env[l].data[full] += cd(double(v[x]) * sc, double(v[nrk + x]) * sc);
          }
        }
      }
    }
    std::vector<std::vector<cd>> genv;
    gate_envs_from_leaf_envs(P.net, leaf_env, genv);
    for (size_t g = 0; g < genv.size(); ++g)
      for (int i = 0; i < 16; ++i) {
        env_out[32 * g + 2 * i] = genv[g][i].real();
        env_out[32 * g + 2 * i + 1] = genv[g][i].imag();
      }
    if (amp_out) {
      CUDA_OK(cudaMemcpyAsync(amp_out, ctx->acc.p, size_t(batch) * n_out * sizeof(double2), cudaMemcpyDeviceToHost, s));
      CUDA_OK(cudaStreamSynchronize(s));
    }
    arena.release();
    partials.release();
  });
}
