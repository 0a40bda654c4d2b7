// Circuit -> tensor network (Sec. I; Sec. II-A).
//
// Every gate is first a tensor over wire segments: a segment of qubit q after j gates on
// q is one edge (label).  1-qubit gates are then multiplied into the next 2-qubit gate
// on their qubit (the previous one when none follows), so each leaf is one 2-qubit gate
// with its neighbouring 1-qubit gates; |0> inputs are fixed at once, closed outputs are
// kept as legs that the device fixes per bitstring, open outputs stay free.
#include <algorithm>
#include <map>
#include <string>
#include <numeric>

#include "host.h"

namespace tnc {

static int find_pos(const std::vector<int>& v, int x) {
  for (size_t i = 0; i < v.size(); ++i)
    if (v[i] == x) return (int)i;
  return -1;
}

SmallTensor small_fix(const SmallTensor& a, int label, int value) {
  int p = find_pos(a.labels, label);
  if (p < 0) fail(5, "small_fix: label not present");
  SmallTensor r;
  for (size_t i = 0; i < a.labels.size(); ++i)
    if ((int)i != p) r.labels.push_back(a.labels[i]);
  r.data.assign(size_t(1) << r.labels.size(), cd(0, 0));
  for (size_t idx = 0; idx < a.data.size(); ++idx) {
    if (((idx >> p) & 1) != (size_t)value) continue;
    size_t lo = idx & ((size_t(1) << p) - 1);
    size_t hi = idx >> (p + 1);
    r.data[lo | (hi << p)] = a.data[idx];
  }
  return r;
}

SmallTensor small_contract(const SmallTensor& a, const SmallTensor& b, const std::vector<int>& out) {
  std::vector<int> common;
  for (int x : a.labels)
    if (find_pos(b.labels, x) >= 0 && find_pos(out, x) < 0) common.push_back(x);
  for (int x : out) {
    bool in_a = find_pos(a.labels, x) >= 0, in_b = find_pos(b.labels, x) >= 0;
    if (!(in_a ^ in_b)) fail(5, "small_contract: output label must be free in exactly one operand");
  }
  if (a.labels.size() + b.labels.size() != out.size() + 2 * common.size())
    fail(5, "small_contract: labels do not partition");
  // per-label bit positions
  const int nc = (int)common.size();
  std::vector<int> pa_out(out.size(), -1), pb_out(out.size(), -1);
  for (size_t i = 0; i < out.size(); ++i) {
    pa_out[i] = find_pos(a.labels, out[i]);
    pb_out[i] = find_pos(b.labels, out[i]);
  }
  std::vector<int> pa_c(nc), pb_c(nc);
  for (int i = 0; i < nc; ++i) {
    pa_c[i] = find_pos(a.labels, common[i]);
    pb_c[i] = find_pos(b.labels, common[i]);
  }
  SmallTensor r;
  r.labels = out;
  r.data.assign(size_t(1) << out.size(), cd(0, 0));
  for (size_t o = 0; o < r.data.size(); ++o) {
    size_t ia = 0, ib = 0;
    for (size_t i = 0; i < out.size(); ++i) {
      size_t bit = (o >> i) & 1;
      if (pa_out[i] >= 0) ia |= bit << pa_out[i];
      else ib |= bit << pb_out[i];
    }
    cd acc(0, 0);
    for (size_t k = 0; k < (size_t(1) << nc); ++k) {
      size_t ja = ia, jb = ib;
      for (int i = 0; i < nc; ++i) {
        size_t bit = (k >> i) & 1;
        ja |= bit << pa_c[i];
        jb |= bit << pb_c[i];
      }
      acc += a.data[ja] * b.data[jb];
    }
    r.data[o] = acc;
  }
  return r;
}

// Free labels of a contraction, a's free labels first (in a's order), then b's.
static std::vector<int> free_labels(const std::vector<int>& a, const std::vector<int>& b) {
  std::vector<int> out;
  for (int x : a)
    if (find_pos(b, x) < 0) out.push_back(x);
  for (int x : b)
    if (find_pos(a, x) < 0) out.push_back(x);
  return out;
}

// Tensor of one gate over its legs [out legs..., in legs...]: flat bit s = out leg s
// (bit (arity-1-s) of the matrix row), bit arity+s = in leg s.
static SmallTensor gate_tensor(const Gate& g, const std::vector<int>& labels) {
  SmallTensor t;
  t.labels = labels;
  const int d = 1 << g.arity;
  t.data.assign(size_t(d) * d, cd(0, 0));
  for (int o = 0; o < d; ++o)
    for (int i = 0; i < d; ++i) {
      size_t idx = 0;
      for (int s = 0; s < g.arity; ++s) {
        idx |= size_t((o >> (g.arity - 1 - s)) & 1) << s;
        idx |= size_t((i >> (g.arity - 1 - s)) & 1) << (g.arity + s);
      }
      t.data[idx] = g.m[o * d + i];
    }
  return t;
}

// Leaf = contraction of its gates (circuit order), then |0> fixed on input legs.
static SmallTensor form_leaf(const Network& net, const Leaf& lf) {
  SmallTensor t = gate_tensor(net.circ.gates[lf.gates[0]], net.gate_labels[lf.gates[0]]);
  for (size_t m = 1; m < lf.gates.size(); ++m) {
    const SmallTensor u = gate_tensor(net.circ.gates[lf.gates[m]], net.gate_labels[lf.gates[m]]);
    t = small_contract(t, u, free_labels(t.labels, u.labels));
  }
  for (int e : std::vector<int>(t.labels))
    if (net.edges[e].kind == EDGE_INPUT) t = small_fix(t, e, 0);
  return t;
}

void update_gates(Network& net, const std::vector<Gate>& gates) {
  if (gates.size() != net.circ.gates.size()) fail(1, "update_gates: gate count differs");
  for (size_t g = 0; g < gates.size(); ++g) {
    const Gate& a = net.circ.gates[g];
    if (gates[g].arity != a.arity || gates[g].q[0] != a.q[0] || (a.arity == 2 && gates[g].q[1] != a.q[1]))
      fail(1, "update_gates: gate " + std::to_string(g) + " changes qubits or arity");
  }
  net.circ.gates = gates;
  for (Leaf& lf : net.leaves)
    if (!lf.gates.empty()) {
      SmallTensor t = form_leaf(net, lf);
      if (t.labels != lf.t.labels) fail(5, "update_gates: leaf labels changed");
      lf.t = t;
    }
}

void gate_envs_from_leaf_envs(const Network& net, const std::vector<SmallTensor>& leaf_env,
                              std::vector<std::vector<cd>>& out) {
  out.assign(net.circ.gates.size(), std::vector<cd>(16, cd(0, 0)));
  const SmallTensor e0{{-1}, {cd(1, 0), cd(0, 0)}};
  for (size_t li = 0; li < net.leaves.size(); ++li) {
    const Leaf& lf = net.leaves[li];
    for (size_t j = 0; j < lf.gates.size(); ++j) {
      const int gj = lf.gates[j];
      const std::vector<int>& mine = net.gate_labels[gj];
      SmallTensor t = leaf_env[li];
      for (size_t k = 0; k < lf.gates.size(); ++k) {
        if (k == j) continue;
        const int gk = lf.gates[k];
        SmallTensor u = gate_tensor(net.circ.gates[gk], net.gate_labels[gk]);
        // |0> on the other gate's fixed input legs
        for (int e : std::vector<int>(u.labels))
          if (net.edges[e].kind == EDGE_INPUT) u = small_fix(u, e, 0);
        std::vector<int> keep;
        for (int x : t.labels)
          if (std::find(u.labels.begin(), u.labels.end(), x) == u.labels.end() ||
              std::find(mine.begin(), mine.end(), x) != mine.end())
            keep.push_back(x);
        for (int x : u.labels)
          if (std::find(t.labels.begin(), t.labels.end(), x) == t.labels.end()) keep.push_back(x);
        t = small_contract(t, u, keep);
      }
      // env over the gate's own legs; fixed input legs carry |0>
      for (int x : mine) {
        if (std::find(t.labels.begin(), t.labels.end(), x) != t.labels.end()) continue;
        if (net.edges[x].kind != EDGE_INPUT) fail(5, "chain rule: missing gate leg");
        SmallTensor v = e0;
        v.labels = {x};
        std::vector<int> both = t.labels;
        both.push_back(x);
        t = small_contract(t, v, both);
      }
      if (t.labels.size() != mine.size()) fail(5, "chain rule: environment labels do not match the gate");
      const Gate& g = net.circ.gates[gj];
      const int d = 1 << g.arity;
      std::vector<int> pos(mine.size());
      for (size_t s = 0; s < mine.size(); ++s) pos[s] = find_pos(t.labels, mine[s]);
      for (int o = 0; o < d; ++o)
        for (int i = 0; i < d; ++i) {
          size_t idx = 0;
          for (int s = 0; s < g.arity; ++s) {
            idx |= size_t((o >> (g.arity - 1 - s)) & 1) << pos[s];
            idx |= size_t((i >> (g.arity - 1 - s)) & 1) << pos[g.arity + s];
          }
          out[gj][o * d + i] += t.data[idx];  // d x d row-major, as the gate matrices
        }
    }
  }
}

void build_network(const Circuit& c, const std::vector<uint8_t>& open_mask, Network& net) {
  const int n = c.n;
  net = Network();
  net.circ = c;
  // wire segments (q, j): edge ids
  std::vector<int> count(n, 0);
  for (const Gate& g : c.gates)
    for (int t = 0; t < g.arity; ++t) count[g.q[t]]++;
  std::vector<std::vector<int>> seg(n);
  for (int q = 0; q < n; ++q) {
    for (int j = 0; j <= count[q]; ++j) {
      Edge e;
      e.qubit = q;
      e.cut = j;
      e.kind = (j == count[q]) ? EDGE_OUTPUT : (j == 0 ? EDGE_INPUT : EDGE_INNER);
      e.open = (j == count[q]) && !open_mask.empty() && open_mask[q] != 0;
      seg[q].push_back((int)net.edges.size());
      net.edges.push_back(e);
    }
  }
  // per-gate legs: [out legs..., in legs...]
  std::vector<int> pos(n, 0);
  std::vector<std::vector<int>> gates_on(n);
  net.gate_labels.resize(c.gates.size());
  for (size_t gi = 0; gi < c.gates.size(); ++gi) {
    const Gate& g = c.gates[gi];
    std::vector<int>& labels = net.gate_labels[gi];
    for (int s = 0; s < g.arity; ++s) labels.push_back(seg[g.q[s]][pos[g.q[s]] + 1]);
    for (int s = 0; s < g.arity; ++s) labels.push_back(seg[g.q[s]][pos[g.q[s]]]);
    for (int s = 0; s < g.arity; ++s) {
      gates_on[g.q[s]].push_back((int)gi);
      pos[g.q[s]]++;
    }
  }
  // group gates into leaves: each 1-qubit gate joins the next 2-qubit gate on its qubit,
  // else the previous one, else (no 2-qubit gate on the qubit) the qubit's own chain
  std::vector<int> group(c.gates.size(), -1);
  for (size_t gi = 0; gi < c.gates.size(); ++gi)
    if (c.gates[gi].arity == 2) group[gi] = (int)gi;
  for (int q = 0; q < n; ++q) {
    const auto& L = gates_on[q];
    for (size_t p = 0; p < L.size(); ++p) {
      int gi = L[p];
      if (c.gates[gi].arity != 1) continue;
      int target = -1;
      for (size_t r = p + 1; r < L.size(); ++r)
        if (c.gates[L[r]].arity == 2) { target = L[r]; break; }
      if (target < 0)
        for (size_t r = p; r-- > 0;)
          if (c.gates[L[r]].arity == 2) { target = L[r]; break; }
      if (target < 0) target = L[0];  // 1-qubit-only wire: first gate names the group
      group[gi] = target;
    }
  }
  std::map<int, std::vector<int>> members;
  for (size_t gi = 0; gi < c.gates.size(); ++gi) members[group[gi]].push_back((int)gi);
  for (auto& kv : members) {
    Leaf leaf;
    leaf.gates = kv.second;  // circuit order
    leaf.t = form_leaf(net, leaf);
    net.leaves.push_back(leaf);
  }
  // qubits without any gate: a rank-1 |0> leaf on their single segment
  for (int q = 0; q < n; ++q) {
    if (count[q] != 0) continue;
    Leaf leaf;
    leaf.t.labels = {seg[q][0]};
    leaf.t.data = {cd(1, 0), cd(0, 0)};
    net.leaves.push_back(leaf);
  }
  net.out_edge.resize(n);
  for (int q = 0; q < n; ++q) {
    net.out_edge[q] = seg[q][count[q]];
    if (!open_mask.empty() && open_mask[q]) {
      net.open_qubits.push_back(q);
      net.open_edge.push_back(seg[q][count[q]]);
    }
  }
}

}  // namespace tnc
