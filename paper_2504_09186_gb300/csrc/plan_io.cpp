// Plan persistence.  Binary little-endian file:
//   "TNCPLAN4", n_qubits, n_gates, gates (arity, q0, q1, 16 complex128), open mask,
//   options, sliced edge ids, tree pairs, cost summary.
// Loading rebuilds the network from the stored circuit (the build is deterministic, so
// edge ids match) and recompiles the step program.
#include <cmath>
#include <cstring>
#include <fstream>

#include "host.h"

namespace tnc {

namespace {
const char kMagic[8] = {'T', 'N', 'C', 'P', 'L', 'A', 'N', '5'};

template <class T>
void put(std::ofstream& f, const T& v) {
  f.write(reinterpret_cast<const char*>(&v), sizeof(T));
}
template <class T>
T get(std::ifstream& f) {
  T v;
  f.read(reinterpret_cast<char*>(&v), sizeof(T));
  if (!f) fail(7, "plan file truncated");
  return v;
}
}  // namespace

void save_plan(const Plan& p, const std::string& path) {
  std::ofstream f(path, std::ios::binary | std::ios::trunc);
  if (!f) fail(7, "cannot open " + path + " for writing");
  f.write(kMagic, 8);
  const Circuit& c = p.net.circ;
  put<int32_t>(f, c.n);
  put<int64_t>(f, (int64_t)c.gates.size());
  for (const Gate& g : c.gates) {
    put<int32_t>(f, g.arity);
    put<int32_t>(f, g.q[0]);
    put<int32_t>(f, g.q[1]);
    for (int i = 0; i < 16; ++i) {
      put<double>(f, g.m[i].real());
      put<double>(f, g.m[i].imag());
    }
  }
  std::vector<uint8_t> mask(c.n, 0);
  for (int q : p.net.open_qubits) mask[q] = 1;
  for (uint8_t b : mask) put<uint8_t>(f, b);
  put<uint64_t>(f, p.opts.seed);
  put<int32_t>(f, p.opts.trials);
  put<int32_t>(f, p.opts.log2_cap);
  put<int32_t>(f, p.opts.slices_min);
  put<int32_t>(f, p.opts.slices_max);
  put<double>(f, p.opts.temperature);
  put<int32_t>(f, p.opts.mode);
  put<int32_t>(f, p.opts.objective);
  put<int32_t>(f, p.opts.slicing);
  put<int32_t>(f, p.opts.branch_exchange);
  put<int32_t>(f, p.opts.cluster_chains);
  put<int32_t>(f, (int32_t)p.sliced.size());
  for (int e : p.sliced) put<int32_t>(f, e);
  put<int32_t>(f, (int32_t)p.tree.size());
  for (auto& pr : p.tree) {
    put<int32_t>(f, pr.first);
    put<int32_t>(f, pr.second);
  }
  put<double>(f, p.log2_flops_slice);
  put<double>(f, p.log2_flops_total);
  put<double>(f, p.overhead);
  put<double>(f, p.log2_flops_executed);
  if (!f) fail(7, "write failed: " + path);
}

void load_plan(const std::string& path, Plan& p) {
  std::ifstream f(path, std::ios::binary);
  if (!f) fail(7, "cannot open " + path);
  char magic[8];
  f.read(magic, 8);
  if (!f || std::memcmp(magic, kMagic, 8) != 0) fail(7, "not a plan file: " + path);
  Circuit c;
  c.n = get<int32_t>(f);
  const int64_t ng = get<int64_t>(f);
  if (c.n < 1 || c.n > 64 || ng < 0 || ng > (int64_t(1) << 26)) fail(7, "corrupt plan header");
  c.gates.resize((size_t)ng);
  for (Gate& g : c.gates) {
    g.arity = get<int32_t>(f);
    g.q[0] = get<int32_t>(f);
    g.q[1] = get<int32_t>(f);
    if (g.arity < 1 || g.arity > 2) fail(7, "corrupt gate");
    for (int t = 0; t < g.arity; ++t)
      if (g.q[t] < 0 || g.q[t] >= c.n) fail(7, "corrupt gate qubit");
    for (int i = 0; i < 16; ++i) {
      double re = get<double>(f), im = get<double>(f);
      g.m[i] = cd(re, im);
    }
  }
  std::vector<uint8_t> mask(c.n);
  for (auto& b : mask) b = get<uint8_t>(f);
  Network net;
  build_network(c, mask, net);
  p = Plan();
  p.net = net;
  p.opts.seed = get<uint64_t>(f);
  p.opts.trials = get<int32_t>(f);
  p.opts.log2_cap = get<int32_t>(f);
  p.opts.slices_min = get<int32_t>(f);
  p.opts.slices_max = get<int32_t>(f);
  p.opts.temperature = get<double>(f);
  p.opts.mode = get<int32_t>(f);
  p.opts.objective = get<int32_t>(f);
  p.opts.slicing = get<int32_t>(f);
  p.opts.branch_exchange = get<int32_t>(f);
  p.opts.cluster_chains = get<int32_t>(f);
  if (p.opts.cluster_chains != 0 && p.opts.cluster_chains != 1) fail(7, "corrupt plan options");
  const int32_t ns = get<int32_t>(f);
  if (ns < 0 || ns > (int32_t)net.edges.size()) fail(7, "corrupt slice count");
  for (int i = 0; i < ns; ++i) {
    int e = get<int32_t>(f);
    if (e < 0 || e >= (int)net.edges.size()) fail(7, "corrupt sliced edge");
    p.sliced.push_back(e);
  }
  const int32_t nt = get<int32_t>(f);
  const int L = (int)net.leaves.size();
  if (nt != (L > 0 ? L - 1 : 0)) fail(7, "tree does not match the network");
  std::vector<char> used(2 * L, 0);
  for (int i = 0; i < nt; ++i) {
    int a = get<int32_t>(f), b = get<int32_t>(f);
    if (a < 0 || b < 0 || a >= L + i || b >= L + i || a == b || used[a] || used[b]) fail(7, "corrupt tree");
    used[a] = used[b] = 1;
    p.tree.emplace_back(a, b);
  }
  p.log2_flops_slice = get<double>(f);
  p.log2_flops_total = get<double>(f);
  p.overhead = get<double>(f);
  p.log2_flops_executed = get<double>(f);
  if (p.opts.slicing < 0 || p.opts.slicing > 1 || p.opts.branch_exchange < 0 || p.opts.branch_exchange > 1)
    fail(7, "corrupt plan options");
  compile_plan(p, true);
}

}  // namespace tnc
