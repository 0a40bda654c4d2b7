// Host-side structures of the tensor-network library: circuit, network, plan and the
// compiled per-step program that the device executor runs.
#pragma once

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

namespace tnc {

using cd = std::complex<double>;

// ------------------------------------------------------------------ errors
struct Error {
  int32_t code;
  std::string msg;
};
[[noreturn]] void fail(int32_t code, const std::string& msg);

// ------------------------------------------------------------------ circuit
struct Gate {
  int arity;
  int q[2];
  cd m[16];  // row-major U[out, in], arity 1 uses m[0..3]
};

struct Circuit {
  int n = 0;
  std::vector<Gate> gates;
};

// ------------------------------------------------------------------ network
// A wire segment of qubit `qubit` after `cut` gates on that qubit.
enum EdgeKind { EDGE_INNER = 0, EDGE_INPUT = 1, EDGE_OUTPUT = 2 };
struct Edge {
  int qubit = -1;
  int cut = -1;
  int kind = EDGE_INNER;
  bool open = false;  // output edge left open (a label of the result)
};

// A small tensor over edge labels; position p of `labels` is bit p of the flat index.
struct SmallTensor {
  std::vector<int> labels;
  std::vector<cd> data;
};

// How a leaf was formed from gates: a list of gate indices whose per-gate tensors
// (labels in the per-gate network) contract to the leaf.
struct Leaf {
  SmallTensor t;                 // labels include fixed legs (closed outputs); inputs removed
  std::vector<int> gates;        // constituent gates
};

struct Network {
  Circuit circ;
  std::vector<Edge> edges;
  std::vector<Leaf> leaves;
  std::vector<int> open_qubits;  // ascending
  std::vector<int> open_edge;    // per open qubit
  std::vector<int> out_edge;     // per qubit: edge id of its output segment
  // per-gate network (for the adjoint's chain rule): labels of gate g's tensor,
  // [out legs..., in legs...] in the gate's qubit order
  std::vector<std::vector<int>> gate_labels;
};

// Build the network; open_mask may be empty (all closed).
void build_network(const Circuit& c, const std::vector<uint8_t>& open_mask, Network& net);

// Small host contraction over labels (FP64), used for leaf formation and the adjoint's
// per-gate chain rule.  Result labels: `out_labels` (must be exactly the free labels).
SmallTensor small_contract(const SmallTensor& a, const SmallTensor& b, const std::vector<int>& out_labels);
SmallTensor small_fix(const SmallTensor& a, int label, int value);

// Replace the gate matrices (same structure) and re-form every leaf.
void update_gates(Network& net, const std::vector<Gate>& gates);

// Per-gate environments dL/dU_g from leaf environments (dL/d leaf over the leaf's labels):
// each leaf is multilinear in its gates, so dL/dU_g contracts the leaf environment with the
// leaf's other gates (and |0> on fixed input legs).  out[g] = d x d row-major [out, in].
void gate_envs_from_leaf_envs(const Network& net, const std::vector<SmallTensor>& leaf_env,
                              std::vector<std::vector<cd>>& out);

// ------------------------------------------------------------------ plan
// Modeled GB300 time (seconds) of one pairwise contraction of operands with a and b labels,
// k of them common, and a result with c labels: the larger of its flop time and its memory
// time (complex-half storage, 4 bytes per entry), at the rates this library's kernels reach
// on GB300.  Steps large enough for tensor-core tiles (M >= 2^7, N >= 2^6 or the reverse,
// K >= 2^4): 1.8 PF/s and 4.5 TB/s (the tensor-core GEMM and its direct epilogue).  Others:
// the FP32-lane rate of 40 TF/s and 1.5 TB/s (the SIMT tiled kernels), except absorptions
// into a large tensor (2^24 entries or more) through a thin operand, measured at 0.7 TB/s.
inline double step_model_seconds(int a, int b, int c, int k) {
  const int m = a - k, n = b - k;
  const double flops = 8.0 * std::ldexp(1.0, a + b - k);
  const double bytes = 4.0 * (std::ldexp(1.0, a) + std::ldexp(1.0, b) + std::ldexp(1.0, c));
  const bool tc = std::max(m, n) >= 7 && std::min(m, n) >= 6 && k >= 4;
  const double bw = std::max(a, b) >= 24 ? 0.7e12 : 1.5e12;
  return tc ? std::max(flops / 1.8e15, bytes / 4.5e12) : std::max(flops / 4.0e13, bytes / bw);
}

struct PlanOpts {
  uint64_t seed = 1;
  int trials = 16;
  int log2_cap = 26;
  int slices_min = 0;
  int slices_max = 64;
  double temperature = 0.5;
  int mode = 0;       // 0 greedy, 1 stem, 2 qubit split (sliced separator + fused stems)
  int objective = 0;  // 0 fewest multiply-adds, 1 least modeled GB300 time
  int slicing = 0;    // 0 index overhead of Eq. 1; 1 executed cost under tree-like reuse
  int branch_exchange = 0;  // 1: reorder consecutive contractions to shorten lifetimes
  int cluster_chains = 0;   // 1: fused chains may hold up to 2^15 entries on a CTA cluster
};

// One sliced index of a plan (slice bit t): its lifetime in the contraction order, the steps
// whose results depend on it, and its overheads at the plan's final slice set.
struct SliceStat {
  int first_step = -1, last_step = -1;  // first / last step with the index in an operand
  int dep_steps = 0;                    // steps whose subtree fixes the index
  double overhead = 1;                  // 2 C / C(without it): Eq. 1
  double reuse_overhead = 1;            // the same ratio of executed cost under tree-like reuse
  int post_steps = 0;                   // dependent steps after the lifetime: they run once
                                        // per value of the index, though it no longer appears
  double merge_saving = 0;              // fraction of the executed cost (under reuse) that
                                        // merging right after the lifetime would save
};

// Kernel classes of a compiled step.
enum StepKind {
  K_GENERIC = 0,   // tiled gather contraction (SIMT FP32), any shape
  K_SPLITK = 1,    // GEPDOT: same tiles, split over outer common indices + fixed-order reduce
  K_CHAIN = 2,     // fused chain of small absorptions into one big tensor (Sec. IV)
  K_TC = 3,        // tcgen05 complex GEMM, cp.async gathered tiles (fp16/bf16, FP32 in TMEM)
  K_TMA = 4,       // tcgen05 complex GEMM, TMA-loaded tiles (operands laid out [Kt | Mt/Nt | ...])
};

// Tile description of one pairwise contraction (all label ids are edge ids).
struct TileSpec {
  std::vector<int> Mt, Nt, Kt;   // tile labels
  std::vector<int> Mo, No, Ko;   // outer labels (grid / loop)
  int rm = 1, rn = 1;            // register micro-tile
  int kgroups = 1;               // intra-CTA split of the K tile
  int splitk = 1;                // CTAs along the outer K labels
  bool gepdot = false;           // few outputs, long K
  bool stream = false;           // long K loop over a thin operand: streamed through a cp.async ring
};

struct Step {
  int a, b, c;                    // tensor ids (A = the larger operand)
  int kind = K_GENERIC;
  TileSpec tile;
  // tensor-core variant for fp16/bf16 storage: 128 x 128 x 64 tiles; tc_tile.Kt[0..2]
  // sit at positions 0..2 of both operands
  bool tc_ok = false;
  TileSpec tc_tile;
  bool tc_swap = false;           // tensor-core rows come from b (b has more free labels)
  int tc_bn = 128, tc_bk = 64;    // tile width and K tile of the tensor-core kernel
};

// A fused chain (Sec. IV): consecutive absorptions of small tensors into one large
// tensor executed as one kernel that keeps a tile over the `inner` labels on chip.
struct Chain {
  std::vector<int> steps;         // step indices in order (link i's a = link i-1's c)
  std::vector<int> inner0;        // labels of the first big operand kept on chip
};

struct TensorInfo {
  std::vector<int> labels;        // storage order (position p = bit p)
  int producer = -1;              // step index, -1 for leaves
  int last_use = -1;              // step index of last consumer (root: n_steps)
  int64_t offset = -1;            // scalar offset in the arena (per instance), unfused program
  int64_t offset_fused = -1;      // ... in the fused program (-1: lives on chip inside a chain)
  int leaf = -1;                  // leaf index for leaf tensors
  bool on_chip = false;           // intermediate of a fused chain, never stored
  uint64_t dep = 0;               // sliced indices (slice-id bits) its values depend on
};

struct Plan {
  Network net;
  PlanOpts opts;
  std::vector<int> sliced;                 // edge ids; slice id bit t <-> sliced[t]
  std::vector<std::pair<int, int>> tree;   // SSA pairs over tensor ids (leaves first)
  std::vector<TensorInfo> tensors;         // leaves then intermediates (per-slice labels)
  std::vector<Step> steps;                 // compiled program (may fuse tree steps)
  int root = -1;
  double log2_flops_slice = 0, log2_flops_total = 0, overhead = 1;
  double log2_flops_executed = 0;  // all slices of one bitstring row under tree-like reuse
  double log2_flops_executed_merged = 0;  // ... with post-lifetime merging (computed by compile_plan)
  double model_seconds = 0;  // modeled GB300 time of one slice (step_model_seconds summed)
  int max_log2 = 0;
  int64_t arena_elems = 0;                 // per instance, in scalars, unfused program
  int64_t arena_elems_fused = 0;           // per instance, in scalars, fused program
  // fixed-leg bookkeeping for the leaf gather: for each leaf, positions of sliced legs
  // (with slice bit index) and closed output legs (with qubit)
  struct LegFix {
    int pos;     // position in the full leaf tensor
    int kind;    // 0 = slice bit, 1 = output bit
    int index;   // slice bit t, or qubit q
  };
  std::vector<std::vector<LegFix>> leaf_fix;
  std::vector<Chain> chains;               // fused chains (empty when compiled with fuse = false)
  std::vector<int> step_chain;             // per step: chain index or -1
  int n_gemm = 0, n_gepdot = 0, n_absorb = 0, n_fused = 0;
  double narrow_max = 0;
  bool fuse = true;
  uint64_t gate_version = 0;               // bumped whenever the gate matrices change
};

void plan_greedy(const Network& net, const PlanOpts& o, Plan& plan);
std::vector<SliceStat> slice_stats(const Plan& plan);
// (Re)compile the program of a plan whose tree and slices are set.
void compile_plan(Plan& plan, bool fuse);

void save_plan(const Plan& p, const std::string& path);
void load_plan(const std::string& path, Plan& p);

}  // namespace tnc
