// extern "C" entry points of the host-side calls (circuit, network, plan, errors).
// Device-side calls (context, amplitudes, contract, adjoint) are in exec.cu.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <string>

#include "../../include/tnc.h"
#include "capi_internal.h"
#include "host.h"

namespace tnc {

thread_local std::string g_last_error;

void fail(int32_t code, const std::string& msg) { throw Error{code, msg}; }

void set_error(const std::string& m) { g_last_error = m; }

}  // namespace tnc

using namespace tnc;

struct tnc_circuit_s {
  Circuit c;
};
struct tnc_network_s {
  Network n;
};

const char* tnc_last_error(void) { return g_last_error.c_str(); }

const char* tnc_version(void) { return "tnc-gb300 1.0 (sm_103a)"; }

tnc_status tnc_circuit_from_gates(int32_t n_qubits, int64_t n_gates, const int32_t* arity,
                                  const int32_t* qubits, const double* matrices, tnc_circuit* out) {
  return guarded([&] {
    if (!out) fail(TNC_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_qubits < 1 || n_qubits > 64) fail(TNC_E_INVALID_ARG, "n_qubits must be in [1, 64]");
    if (n_gates < 0) fail(TNC_E_INVALID_ARG, "n_gates < 0");
    if (n_gates > 0 && (!arity || !qubits || !matrices)) fail(TNC_E_INVALID_ARG, "NULL gate arrays");
    auto* c = new tnc_circuit_s();
    c->c.n = n_qubits;
    c->c.gates.resize((size_t)n_gates);
    for (int64_t g = 0; g < n_gates; ++g) {
      Gate& G = c->c.gates[(size_t)g];
      G.arity = arity[g];
      if (G.arity != 1 && G.arity != 2) {
        delete c;
        fail(TNC_E_INVALID_ARG, "gate " + std::to_string(g) + ": arity must be 1 or 2");
      }
      for (int t = 0; t < 2; ++t) G.q[t] = t < G.arity ? qubits[2 * g + t] : -1;
      for (int t = 0; t < G.arity; ++t)
        if (G.q[t] < 0 || G.q[t] >= n_qubits) {
          delete c;
          fail(TNC_E_INVALID_ARG, "gate " + std::to_string(g) + ": qubit out of range");
        }
      if (G.arity == 2 && G.q[0] == G.q[1]) {
        delete c;
        fail(TNC_E_INVALID_ARG, "gate " + std::to_string(g) + ": repeated qubit");
      }
      const int d = 1 << G.arity;
      for (int i = 0; i < 16; ++i) G.m[i] = 0;
      for (int i = 0; i < d * d; ++i) G.m[i] = cd(matrices[32 * g + 2 * i], matrices[32 * g + 2 * i + 1]);
    }
    *out = c;
  });
}

void tnc_circuit_destroy(tnc_circuit c) { delete c; }

namespace {
// splitmix64: the generator's one random stream (seed -> 64-bit draws)
struct Split64 {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return double(next() >> 11) * (1.0 / 9007199254740992.0); }  // [0, 1)
};
}  // namespace

tnc_status tnc_circuit_random_grid(int32_t rows, int32_t cols, int32_t cycles, uint64_t seed, int32_t fsim_mode,
                                   tnc_circuit* out) {
  return guarded([&] {
    if (!out) fail(TNC_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (rows < 1 || cols < 1 || int64_t(rows) * cols > 64) fail(TNC_E_INVALID_ARG, "grid must hold 1..64 qubits");
    if (cycles < 0) fail(TNC_E_INVALID_ARG, "cycles < 0");
    if (fsim_mode != 0 && fsim_mode != 1) fail(TNC_E_INVALID_ARG, "fsim_mode must be 0 (fixed) or 1 (uniform)");
    const int n = rows * cols;
    const double pi = 3.14159265358979323846, r2 = 0.70710678118654752440;
    // sqrt(X), sqrt(Y), sqrt(W) = (I - i P) / sqrt 2 with P = X, Y, (X + Y) / sqrt 2; U[out, in]
    const cd w = std::polar(1.0, 0.25 * pi);
    const cd one_q[3][4] = {{r2, cd(0, -r2), cd(0, -r2), r2},
                            {r2, -r2, r2, r2},
                            {r2, -r2 * w, r2 * std::conj(w), r2}};
    Split64 g1{seed}, g2{seed ^ 0xD1B54A32D192ED03ull};
    auto* c = new tnc_circuit_s();
    c->c.n = n;
    std::vector<int> prev(n, -1);
    for (int k = 0; k < cycles; ++k) {
      for (int q = 0; q < n; ++q) {
        // the first cycle draws from all three gates, later ones from the two that differ
        // from the qubit's previous gate (in index order)
        int pick;
        if (prev[q] < 0) {
          pick = (int)(g1.next() % 3);
        } else {
          const int j = (int)(g1.next() % 2);
          int others[2], m = 0;
          for (int t = 0; t < 3; ++t)
            if (t != prev[q]) others[m++] = t;
          pick = others[j];
        }
        prev[q] = pick;
        Gate G;
        G.arity = 1;
        G.q[0] = q;
        G.q[1] = -1;
        for (int i = 0; i < 16; ++i) G.m[i] = 0;
        for (int i = 0; i < 4; ++i) G.m[i] = one_q[pick][i];
        c->c.gates.push_back(G);
      }
      // fSim on coupler class A, B, C, D (cycle k mod 4) of the grid, lower qubit first
      const char cls = "ABCD"[k % 4];
      std::vector<std::pair<int, int>> pairs;
      if (cls == 'A' || cls == 'B') {
        for (int r = 0; r < rows; ++r)
          for (int col = cls == 'A' ? 0 : 1; col + 1 < cols; col += 2) pairs.emplace_back(r * cols + col, r * cols + col + 1);
      } else {
        for (int r = cls == 'C' ? 0 : 1; r + 1 < rows; r += 2)
          for (int col = 0; col < cols; ++col) pairs.emplace_back(r * cols + col, (r + 1) * cols + col);
      }
      for (auto& pq : pairs) {
        double theta = pi / 2, phi = pi / 6;
        if (fsim_mode == 1) {
          theta = pi * g2.uniform();
          phi = pi * g2.uniform();
        }
        // fSim(theta, phi) in the basis |q_a q_b>, q_a (the lower index) most significant
        Gate G;
        G.arity = 2;
        G.q[0] = pq.first;
        G.q[1] = pq.second;
        for (int i = 0; i < 16; ++i) G.m[i] = 0;
        G.m[0] = 1;
        G.m[5] = std::cos(theta);
        G.m[6] = cd(0, -std::sin(theta));
        G.m[9] = cd(0, -std::sin(theta));
        G.m[10] = std::cos(theta);
        G.m[15] = std::polar(1.0, -phi);
        c->c.gates.push_back(G);
      }
    }
    *out = c;
  });
}

tnc_status tnc_circuit_export(tnc_circuit c, int32_t* n_qubits, int64_t* n_gates, int32_t* arity, int32_t* qubits,
                              double* matrices, int64_t cap) {
  return guarded([&] {
    if (!c) fail(TNC_E_INVALID_ARG, "NULL circuit");
    const int64_t g = (int64_t)c->c.gates.size();
    if (n_qubits) *n_qubits = c->c.n;
    if (n_gates) *n_gates = g;
    if (!arity && !qubits && !matrices) return;  // size query
    if (cap < g) fail(TNC_E_INVALID_ARG, "cap below the number of gates");
    for (int64_t i = 0; i < g; ++i) {
      const Gate& G = c->c.gates[(size_t)i];
      if (arity) arity[i] = G.arity;
      if (qubits) {
        qubits[2 * i] = G.q[0];
        qubits[2 * i + 1] = G.arity == 2 ? G.q[1] : -1;
      }
      if (matrices) {
        const int d = 1 << G.arity;
        for (int j = 0; j < 32; ++j) matrices[32 * i + j] = 0;
        for (int j = 0; j < d * d; ++j) {
          matrices[32 * i + 2 * j] = G.m[j].real();
          matrices[32 * i + 2 * j + 1] = G.m[j].imag();
        }
      }
    }
  });
}

tnc_status tnc_network_build(tnc_circuit c, const uint8_t* open_mask, tnc_network* out) {
  return guarded([&] {
    if (!c || !out) fail(TNC_E_INVALID_ARG, "NULL argument");
    *out = nullptr;
    std::vector<uint8_t> mask;
    if (open_mask) mask.assign(open_mask, open_mask + c->c.n);
    auto* n = new tnc_network_s();
    try {
      build_network(c->c, mask, n->n);
    } catch (...) {
      delete n;
      throw;
    }
    *out = n;
  });
}

void tnc_network_destroy(tnc_network n) { delete n; }

tnc_status tnc_plan_greedy(tnc_network n, const tnc_plan_opts* opts, tnc_plan* out) {
  return guarded([&] {
    if (!n || !opts || !out) fail(TNC_E_INVALID_ARG, "NULL argument");
    *out = nullptr;
    PlanOpts o;
    o.seed = opts->seed;
    o.trials = opts->trials;
    o.log2_cap = opts->log2_cap;
    o.slices_min = opts->slices_min;
    o.slices_max = opts->slices_max;
    o.temperature = opts->temperature;
    o.mode = opts->mode;
    o.objective = opts->objective;
    o.slicing = opts->slicing;
    o.branch_exchange = opts->branch_exchange;
    o.cluster_chains = opts->cluster_chains;
    if (o.mode < 0 || o.mode > 2) fail(TNC_E_INVALID_ARG, "plan mode must be 0 (greedy), 1 (stem) or 2 (qubit split)");
    if (o.objective != 0 && o.objective != 1) fail(TNC_E_INVALID_ARG, "plan objective must be 0 or 1");
    if (o.slicing != 0 && o.slicing != 1) fail(TNC_E_INVALID_ARG, "plan slicing must be 0 (Eq. 1) or 1 (reuse)");
    if (o.branch_exchange != 0 && o.branch_exchange != 1) fail(TNC_E_INVALID_ARG, "branch_exchange must be 0 or 1");
    if (o.cluster_chains != 0 && o.cluster_chains != 1) fail(TNC_E_INVALID_ARG, "cluster_chains must be 0 or 1");
    auto* p = new tnc_plan_s();
    try {
      plan_greedy(n->n, o, p->p);
    } catch (...) {
      delete p;
      throw;
    }
    *out = p;
  });
}

void tnc_plan_destroy(tnc_plan p) {
  if (p) release_plan_device(p);
  delete p;
}

tnc_status tnc_plan_get_info(tnc_plan p, tnc_plan_info* info) {
  return guarded([&] {
    if (!p || !info) fail(TNC_E_INVALID_ARG, "NULL argument");
    const Plan& P = p->p;
    std::memset(info, 0, sizeof(*info));
    info->log2_flops_per_slice = P.log2_flops_slice;
    info->log2_total_flops = P.log2_flops_total;
    info->slicing_overhead = P.overhead;
    info->max_log2_size = P.max_log2;
    info->n_sliced = (int32_t)P.sliced.size();
    info->n_steps = (int32_t)P.tree.size();
    info->n_leaves = (int32_t)P.net.leaves.size();
    info->n_open = (int32_t)P.net.open_qubits.size();
    info->n_kernels = (int32_t)P.steps.size() + 3;
    info->n_gemm = P.n_gemm;
    info->n_gepdot = P.n_gepdot;
    info->n_absorb = P.n_absorb;
    info->n_fused = P.n_fused;
    info->narrow_max = P.narrow_max;
    info->model_seconds_per_slice = P.model_seconds;
    info->log2_executed_flops = P.log2_flops_executed;
    info->log2_executed_flops_merged = P.log2_flops_executed_merged;
  });
}

tnc_status tnc_plan_sliced_cuts(tnc_plan p, int32_t* qubit, int32_t* cut, int32_t cap) {
  return guarded([&] {
    if (!p || (!qubit && cap > 0) || (!cut && cap > 0)) fail(TNC_E_INVALID_ARG, "NULL argument");
    const Plan& P = p->p;
    if (cap < (int32_t)P.sliced.size()) fail(TNC_E_INVALID_ARG, "cap smaller than the number of sliced indices");
    for (size_t t = 0; t < P.sliced.size(); ++t) {
      qubit[t] = P.net.edges[P.sliced[t]].qubit;
      cut[t] = P.net.edges[P.sliced[t]].cut;
    }
  });
}

tnc_status tnc_plan_open_qubits(tnc_plan p, int32_t* qubits, int32_t cap) {
  return guarded([&] {
    if (!p) fail(TNC_E_INVALID_ARG, "NULL plan");
    const Plan& P = p->p;
    if (cap < (int32_t)P.net.open_qubits.size() || (!qubits && !P.net.open_qubits.empty()))
      fail(TNC_E_INVALID_ARG, "cap smaller than the number of open qubits");
    for (size_t t = 0; t < P.net.open_qubits.size(); ++t) qubits[t] = P.net.open_qubits[t];
  });
}

tnc_status tnc_plan_update_gates(tnc_plan p, int64_t n_gates, const double* matrices) {
  return guarded([&] {
    if (!p || (!matrices && n_gates > 0)) fail(TNC_E_INVALID_ARG, "NULL argument");
    Plan& P = p->p;
    if (n_gates != (int64_t)P.net.circ.gates.size()) fail(TNC_E_INVALID_ARG, "gate count differs from the plan's circuit");
    std::vector<Gate> gates = P.net.circ.gates;
    for (int64_t g = 0; g < n_gates; ++g) {
      const int d = 1 << gates[g].arity;
      for (int i = 0; i < 16; ++i) gates[g].m[i] = 0;
      for (int i = 0; i < d * d; ++i) gates[g].m[i] = cd(matrices[32 * g + 2 * i], matrices[32 * g + 2 * i + 1]);
    }
    update_gates(P.net, gates);
    P.gate_version++;
  });
}

tnc_status tnc_plan_save(tnc_plan p, const char* path) {
  return guarded([&] {
    if (!p || !path) fail(TNC_E_INVALID_ARG, "NULL argument");
    save_plan(p->p, path);
  });
}

tnc_status tnc_plan_load(const char* path, tnc_plan* out) {
  return guarded([&] {
    if (!path || !out) fail(TNC_E_INVALID_ARG, "NULL argument");
    *out = nullptr;
    auto* p = new tnc_plan_s();
    try {
      load_plan(path, p->p);
    } catch (...) {
      delete p;
      throw;
    }
    *out = p;
  });
}

namespace {
std::string jlist(const std::vector<int>& v) {
  std::string s = "[";
  for (size_t i = 0; i < v.size(); ++i) s += (i ? "," : "") + std::to_string(v[i]);
  return s + "]";
}
}  // namespace

tnc_status tnc_plan_slice_stats(tnc_plan p, int32_t* first_step, int32_t* last_step, int32_t* dep_steps,
                                double* overhead, double* reuse_overhead, int32_t* post_steps,
                                double* merge_saving, int32_t cap) {
  return guarded([&] {
    if (!p) fail(TNC_E_INVALID_ARG, "NULL plan");
    const auto st = slice_stats(p->p);
    if (cap < (int32_t)st.size()) fail(TNC_E_INVALID_ARG, "cap below the number of sliced indices");
    for (size_t j = 0; j < st.size(); ++j) {
      if (first_step) first_step[j] = st[j].first_step;
      if (last_step) last_step[j] = st[j].last_step;
      if (dep_steps) dep_steps[j] = st[j].dep_steps;
      if (overhead) overhead[j] = st[j].overhead;
      if (reuse_overhead) reuse_overhead[j] = st[j].reuse_overhead;
      if (post_steps) post_steps[j] = st[j].post_steps;
      if (merge_saving) merge_saving[j] = st[j].merge_saving;
    }
  });
}

tnc_status tnc_plan_describe(tnc_plan p, char* buf, int64_t cap, int64_t* len) {
  return guarded([&] {
    if (!p || !len) fail(TNC_E_INVALID_ARG, "NULL argument");
    const Plan& P = p->p;
    std::string s = "{\"n_qubits\":" + std::to_string(P.net.circ.n);
    s += ",\"edges\":[";
    for (size_t e = 0; e < P.net.edges.size(); ++e) {
      const Edge& E = P.net.edges[e];
      s += (e ? "," : "") + std::string("[") + std::to_string(E.qubit) + "," + std::to_string(E.cut) + "," +
           std::to_string(E.kind) + "," + (E.open ? "1" : "0") + "]";
    }
    s += "],\"leaves\":[";
    for (size_t i = 0; i < P.net.leaves.size(); ++i)
      s += (i ? "," : "") + std::string("{\"labels\":") + jlist(P.net.leaves[i].t.labels) +
           ",\"gates\":" + jlist(P.net.leaves[i].gates) + "}";
    s += "],\"sliced\":" + jlist(P.sliced) + ",\"tree\":[";
    for (size_t i = 0; i < P.tree.size(); ++i)
      s += (i ? "," : "") + std::string("[") + std::to_string(P.tree[i].first) + "," + std::to_string(P.tree[i].second) + "]";
    s += "],\"tensors\":[";
    for (size_t i = 0; i < P.tensors.size(); ++i)
      s += (i ? "," : "") + std::string("{\"labels\":") + jlist(P.tensors[i].labels) +
           ",\"offset\":" + std::to_string(P.tensors[i].offset) + "}";
    // fused chains: their steps, the first operand's on-chip labels and the largest on-chip
    // tile (log2 entries; above 12 the chain runs on a cluster of 2^(bits - 12) CTAs)
    s += "],\"chains\":[";
    for (size_t ci = 0; ci < P.chains.size(); ++ci) {
      const Chain& ch = P.chains[ci];
      std::vector<int> I = ch.inner0;
      size_t mx = I.size();
      for (int sidx : ch.steps) {
        const auto& a = P.tensors[P.steps[sidx].a].labels;
        const auto& b = P.tensors[P.steps[sidx].b].labels;
        std::vector<int> nI;
        for (int x : I)
          if (std::find(b.begin(), b.end(), x) == b.end()) nI.push_back(x);
        for (int x : b)
          if (std::find(a.begin(), a.end(), x) == a.end()) nI.push_back(x);
        I = nI;
        mx = std::max(mx, I.size());
      }
      s += (ci ? "," : "") + std::string("{\"steps\":") + jlist(ch.steps) + ",\"inner0\":" + jlist(ch.inner0) +
           ",\"tile_bits\":" + std::to_string(mx) + "}";
    }
    s += "],\"steps\":[";
    for (size_t i = 0; i < P.steps.size(); ++i) {
      const Step& S = P.steps[i];
      const TileSpec& t = S.tile;
      s += (i ? "," : "") + std::string("{\"a\":") + std::to_string(S.a) + ",\"b\":" + std::to_string(S.b) +
           ",\"c\":" + std::to_string(S.c) + ",\"kind\":" + std::to_string(S.kind) + ",\"Mt\":" + jlist(t.Mt) +
           ",\"Kt\":" + jlist(t.Kt) + ",\"Nt\":" + jlist(t.Nt) + ",\"Mo\":" + jlist(t.Mo) + ",\"Ko\":" + jlist(t.Ko) +
           ",\"No\":" + jlist(t.No) + ",\"splitk\":" + std::to_string(t.splitk) + ",\"rm\":" + std::to_string(t.rm) +
           ",\"rn\":" + std::to_string(t.rn) + ",\"kgroups\":" + std::to_string(t.kgroups) +
           ",\"tc\":" + std::to_string(S.tc_ok ? 1 : 0) + ",\"chain\":" +
           std::to_string(i < P.step_chain.size() ? P.step_chain[i] : -1);
      {
        // narrow rate 2 N_common / (N_A + N_B) of the step (per-slice labels)
        const auto& la = P.tensors[S.a].labels;
        const auto& lb = P.tensors[S.b].labels;
        int nk = 0;
        for (int x : la) nk += std::find(lb.begin(), lb.end(), x) != lb.end();
        char nb[48];
        std::snprintf(nb, sizeof nb, "%.17g", la.size() + lb.size() ? 2.0 * nk / double(la.size() + lb.size()) : 0.0);
        s += ",\"narrow\":" + std::string(nb);
      }
      if (S.tc_ok) {
        const TileSpec& u = S.tc_tile;
        s += ",\"tc_tile\":{\"swap\":" + std::to_string(S.tc_swap ? 1 : 0) + ",\"bn\":" + std::to_string(S.tc_bn) +
             ",\"bk\":" + std::to_string(S.tc_bk) + ",\"Mt\":" + jlist(u.Mt) + ",\"Kt\":" + jlist(u.Kt) +
             ",\"Nt\":" + jlist(u.Nt) + ",\"Mo\":" + jlist(u.Mo) + ",\"Ko\":" + jlist(u.Ko) + ",\"No\":" + jlist(u.No) +
             "}";
      }
      s += "}";
    }
    char num[64];
    std::snprintf(num, sizeof(num), "%.17g", P.log2_flops_slice);
    s += "],\"root\":" + std::to_string(P.root) + ",\"log2_flops_slice\":" + num;
    std::snprintf(num, sizeof(num), "%.17g", P.overhead);
    s += ",\"overhead\":" + std::string(num) + ",\"arena_scalars\":" + std::to_string(P.arena_elems) + "}";
    *len = (int64_t)s.size() + 1;
    if (buf && cap > 0) {
      const size_t n = std::min<size_t>((size_t)cap - 1, s.size());
      std::memcpy(buf, s.data(), n);
      buf[n] = 0;
    }
  });
}
