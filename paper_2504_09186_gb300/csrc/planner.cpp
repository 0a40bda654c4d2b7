// Seeded greedy contraction order and greedy slicing.
//
// Order: repeatedly contract the pair of tensors sharing an index that minimises
// size(out) - size(a) - size(b) (Sec. II-A: each contraction eliminates the shared
// edges), perturbed by seeded Gumbel noise so that independent trials explore
// different trees; the trial with the smallest total cost is kept.
//
// Slicing (Sec. II-A; Sec. III-A, Eq. 1): while some intermediate exceeds 2^cap entries,
// slice the index, among those of the oversized intermediates, whose index overhead
// O(a) = 2 C_a / C is smallest, C being the cost of one subtask before slicing a and
// C_a the cost after.  Indices of the lowest overhead are added afterwards until the
// requested minimum count is reached.  Cost = complex multiply-adds of one subtask,
// sum over steps of 2^|labels(a) U labels(b)|.
#include <algorithm>
#include <cmath>
#include <limits>
#include <map>
#include <set>

#include "host.h"

namespace tnc {

namespace {

struct Rng {
  uint64_t s;
  uint64_t next() {  // splitmix64
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
  double gumbel() { return -std::log(-std::log(uniform())); }
};

using LabelSet = std::vector<int>;  // sorted

LabelSet sym_diff(const LabelSet& a, const LabelSet& b) {
  LabelSet r;
  std::set_symmetric_difference(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(r));
  return r;
}
LabelSet set_union(const LabelSet& a, const LabelSet& b) {
  LabelSet r;
  std::set_union(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(r));
  return r;
}
size_t count_not_in(const LabelSet& a, const std::vector<char>& sliced) {
  size_t n = 0;
  for (int x : a) n += sliced[x] ? 0 : 1;
  return n;
}

struct Tree {
  std::vector<std::pair<int, int>> pairs;
  std::vector<LabelSet> sets;  // leaves then intermediates
};

// Greedy order.  Open labels occur in one tensor only, so the symmetric difference keeps them.
Tree greedy_tree(const std::vector<LabelSet>& leaves, int n_edges, Rng& rng, double temperature) {
  Tree t;
  t.sets = leaves;
  std::vector<char> alive(leaves.size(), 1);
  std::vector<std::vector<int>> owners(n_edges);
  for (size_t i = 0; i < leaves.size(); ++i)
    for (int e : leaves[i]) owners[e].push_back((int)i);
  size_t n_alive = leaves.size();
  while (n_alive > 1) {
    // candidate pairs sharing an edge
    std::vector<std::pair<int, int>> cand;
    for (int e = 0; e < n_edges; ++e) {
      auto& ow = owners[e];
      if (ow.size() == 2) cand.emplace_back(std::min(ow[0], ow[1]), std::max(ow[0], ow[1]));
    }
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    int bi = -1, bj = -1;
    if (cand.empty()) {
      // disconnected: outer product of the two smallest live tensors
      std::vector<std::pair<size_t, int>> live;
      for (size_t i = 0; i < t.sets.size(); ++i)
        if (alive[i]) live.emplace_back(t.sets[i].size(), (int)i);
      std::sort(live.begin(), live.end());
      bi = std::min(live[0].second, live[1].second);
      bj = std::max(live[0].second, live[1].second);
    } else {
      double best = std::numeric_limits<double>::infinity();
      for (auto& p : cand) {
        const LabelSet& A = t.sets[p.first];
        const LabelSet& B = t.sets[p.second];
        LabelSet o = sym_diff(A, B);
        double s = std::ldexp(1.0, (int)o.size()) - std::ldexp(1.0, (int)A.size()) - std::ldexp(1.0, (int)B.size());
        double score = (s >= 0 ? 1.0 : -1.0) * std::log2(1.0 + std::fabs(s));
        if (temperature > 0) score -= temperature * rng.gumbel();
        if (score < best) {
          best = score;
          bi = p.first;
          bj = p.second;
        }
      }
    }
    LabelSet o = sym_diff(t.sets[bi], t.sets[bj]);
    int id = (int)t.sets.size();
    for (int e : t.sets[bi]) {
      auto& ow = owners[e];
      ow.erase(std::remove(ow.begin(), ow.end(), bi), ow.end());
    }
    for (int e : t.sets[bj]) {
      auto& ow = owners[e];
      ow.erase(std::remove(ow.begin(), ow.end(), bj), ow.end());
    }
    for (int e : o) owners[e].push_back(id);
    alive[bi] = alive[bj] = 0;
    alive.push_back(1);
    t.sets.push_back(o);
    t.pairs.emplace_back(bi, bj);
    --n_alive;
  }
  return t;
}

// Stem order: one growing tensor absorbs, one at a time, the leaf sharing labels with it
// that keeps it smallest (Gumbel-perturbed; ties: more shared labels, lower id).  Leaves
// not connected to the stem are absorbed (outer product) when nothing else is left.
Tree stem_tree(const std::vector<LabelSet>& leaves, int n_edges, Rng& rng, double temperature, int start) {
  Tree t;
  t.sets = leaves;
  const int L = (int)leaves.size();
  std::vector<char> used(L, 0);
  std::vector<std::vector<int>> owners(n_edges);
  for (int i = 0; i < L; ++i)
    for (int e : leaves[i]) owners[e].push_back(i);
  int cur = start;
  used[start] = 1;
  for (int step = 1; step < L; ++step) {
    const LabelSet& S = t.sets[cur];
    std::vector<int> cand;
    for (int e : S)
      for (int o : owners[e])
        if (o < L && !used[o]) cand.push_back(o);
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    int pick = -1;
    if (cand.empty()) {
      size_t best = ~size_t(0);
      for (int i = 0; i < L; ++i)
        if (!used[i] && leaves[i].size() < best) best = leaves[i].size(), pick = i;
    } else {
      double best = std::numeric_limits<double>::infinity();
      for (int o : cand) {
        const LabelSet out = sym_diff(S, leaves[o]);
        LabelSet sh;
        std::set_intersection(S.begin(), S.end(), leaves[o].begin(), leaves[o].end(), std::back_inserter(sh));
        double score = (double)out.size() - 0.01 * (double)sh.size();
        if (temperature > 0) score -= temperature * rng.gumbel();
        if (score < best) best = score, pick = o;
      }
    }
    used[pick] = 1;
    t.pairs.emplace_back(cur, pick);
    t.sets.push_back(sym_diff(S, leaves[pick]));
    cur = (int)t.sets.size() - 1;
  }
  return t;
}

double tree_cost(const Tree& t, const std::vector<char>& sliced) {
  double c = 0;
  for (auto& p : t.pairs) {
    LabelSet u = set_union(t.sets[p.first], t.sets[p.second]);
    c += std::ldexp(1.0, (int)count_not_in(u, sliced));
  }
  return c;
}

int tree_max(const Tree& t, const std::vector<char>& sliced) {
  int m = 0;
  for (auto& s : t.sets) m = std::max(m, (int)count_not_in(s, sliced));
  return m;
}

// Number of sliced indices each tensor's subtree fixes (leaves: the sliced labels they
// hold; intermediates: the union over their operands), for any number of sliced indices.
std::vector<int> dep_counts(const Tree& t, const std::vector<int>& sliced_list) {
  const size_t n_leaves = t.sets.size() - t.pairs.size();
  const size_t words = (sliced_list.size() + 63) / 64;
  std::vector<std::vector<uint64_t>> dep(t.sets.size(), std::vector<uint64_t>(words, 0));
  for (size_t i = 0; i < n_leaves; ++i)
    for (size_t j = 0; j < sliced_list.size(); ++j)
      if (std::binary_search(t.sets[i].begin(), t.sets[i].end(), sliced_list[j])) dep[i][j / 64] |= uint64_t(1) << (j % 64);
  std::vector<int> cnt(t.sets.size(), 0);
  for (size_t i = 0; i < n_leaves; ++i)
    for (uint64_t w : dep[i]) cnt[i] += __builtin_popcountll(w);
  for (size_t k = 0; k < t.pairs.size(); ++k) {
    const auto& p = t.pairs[k];
    for (size_t w = 0; w < words; ++w) {
      dep[n_leaves + k][w] = dep[p.first][w] | dep[p.second][w];
      cnt[n_leaves + k] += __builtin_popcountll(dep[n_leaves + k][w]);
    }
  }
  return cnt;
}

// Modeled GB300 time of a call over all 2^s slices of one bitstring row: step_model_seconds
// of every step times the number of times it runs under tree-like reuse (Sec. III-B), one
// per assignment of the sliced indices its subtree fixes.
double model_time(const Tree& t, const std::vector<char>& sliced, const std::vector<int>& sliced_list) {
  const std::vector<int> dep = dep_counts(t, sliced_list);
  const size_t n_leaves = t.sets.size() - t.pairs.size();
  double tot = 0;
  for (size_t k = 0; k < t.pairs.size(); ++k) {
    const auto& p = t.pairs[k];
    const LabelSet& A = t.sets[p.first];
    const LabelSet& B = t.sets[p.second];
    const int a = (int)count_not_in(A, sliced), b = (int)count_not_in(B, sliced);
    const int u = (int)count_not_in(set_union(A, B), sliced);
    const int c = (int)count_not_in(sym_diff(A, B), sliced);
    tot += step_model_seconds(a, b, c, a + b - u) * std::ldexp(1.0, dep[n_leaves + k]);
  }
  return tot;
}

// Executed complex multiply-adds of all 2^s slices of one bitstring row under tree-like
// reuse (Sec. III-B): each step's per-slice cost times the assignments of the sliced indices
// its subtree fixes.  Lifetime-aware: an index costs only over the steps that depend on it.
double reuse_cost(const Tree& t, const std::vector<char>& sliced, const std::vector<int>& sliced_list) {
  const std::vector<int> dep = dep_counts(t, sliced_list);
  const size_t n_leaves = t.sets.size() - t.pairs.size();
  double tot = 0;
  for (size_t k = 0; k < t.pairs.size(); ++k) {
    const auto& p = t.pairs[k];
    const int u = (int)count_not_in(set_union(t.sets[p.first], t.sets[p.second]), sliced);
    tot += std::ldexp(1.0, u + dep[n_leaves + k]);
  }
  return tot;
}

// Branch exchange (Sec. III-C): when step k2 contracts the result of step k1 = (x, g1) with
// g2, the order of g1 and g2 may be exchanged -- k1 = (x, g2), k2 = (k1, g1) -- which leaves
// k2's result unchanged and moves g1's indices' lifetimes later.  Swaps that lower the cost
// (executed cost under reuse, or Eq. 1's when `reuse` is false) and keep every intermediate
// within the cap are kept, pass after pass until none helps (at most `passes`).
void branch_exchange(Tree& t, const std::vector<char>& sliced, const std::vector<int>& sliced_list, int log2_cap,
                     bool reuse, int passes) {
  const int L = (int)(t.sets.size() - t.pairs.size());
  auto cost = [&]() { return reuse ? reuse_cost(t, sliced, sliced_list) : tree_cost(t, sliced); };
  double cur = cost();
  for (int pass = 0; pass < passes; ++pass) {
    bool improved = false;
    for (int k2 = 0; k2 < (int)t.pairs.size(); ++k2) {
      for (int side = 0; side < 2; ++side) {
        auto& p2 = t.pairs[k2];
        const int n1 = side == 0 ? p2.first : p2.second;
        const int g2 = side == 0 ? p2.second : p2.first;
        if (n1 < L) continue;
        const int k1 = n1 - L;
        if (g2 >= L + k1) continue;  // g2 must exist before step k1
        auto& p1 = t.pairs[k1];
        for (int which = 0; which < 2; ++which) {
          const int g1 = which == 0 ? p1.second : p1.first;
          const int x = which == 0 ? p1.first : p1.second;
          const LabelSet new_n1 = sym_diff(t.sets[x], t.sets[g2]);
          if ((int)count_not_in(new_n1, sliced) > log2_cap) continue;
          const auto save1 = p1, save2 = p2;
          const LabelSet save_set = t.sets[n1];
          p1 = {x, g2};
          if (side == 0) p2 = {n1, g1};
          else p2 = {g1, n1};
          t.sets[n1] = new_n1;
          const double c = cost();
          if (c < cur * (1 - 1e-9)) {
            cur = c;
            improved = true;
            break;
          }
          p1 = save1;
          p2 = save2;
          t.sets[n1] = save_set;
        }
      }
    }
    if (!improved) break;
  }
}

// Contraction-level labels of each leaf: closed outputs are fixed per bitstring.
std::vector<LabelSet> contraction_leaves(const Network& net) {
  std::vector<LabelSet> leaves;
  for (const Leaf& l : net.leaves) {
    LabelSet s;
    for (int e : l.t.labels)
      if (!(net.edges[e].kind == EDGE_OUTPUT && !net.edges[e].open)) s.push_back(e);
    std::sort(s.begin(), s.end());
    leaves.push_back(s);
  }
  return leaves;
}

// ------------------------------------------------------------------ qubit split (mode 2)
//
// Slicing a separator (Sec. II-A: a sliced index is fixed in every tensor holding it, so
// slicing every index between two parts of the network makes them independent subtasks).
// For a circuit network the cheapest balanced separator of the *qubits* is taken: the
// qubits are bisected so that few 2-qubit gates straddle the two sides, every leaf goes to
// one side, and the indices joining leaves on different sides are sliced.  Each side is
// then contracted by one stem in circuit order (the stem picture of Sec. II-A / III-C),
// which absorbs fused blocks of leaves: a block gathers consecutive leaves acting on at
// most `fuse` qubits and is contracted first as a small branch, so that each absorption is
// one large GEMM (K, N = 2^inputs, 2^outputs of the block) instead of a run of 2-qubit ones.

// Balanced bisection of n qubits minimising the weight of the pairs split: Fiduccia-
// Mattheyses passes (move the unlocked qubit of largest gain that keeps both sides within
// [n - max_side, max_side], keep the best prefix of moves) from a seeded random start.
std::vector<char> bisect_qubits(int n, const std::vector<std::vector<double>>& w, int max_side, Rng& rng,
                                double* cut_out) {
  std::vector<char> side(n, 0);
  std::vector<int> perm(n);
  for (int i = 0; i < n; ++i) perm[i] = i;
  for (int i = n - 1; i > 0; --i) std::swap(perm[i], perm[rng.next() % (uint64_t)(i + 1)]);
  for (int i = 0; i < n / 2; ++i) side[perm[i]] = 1;
  const int lo = n - max_side, hi = max_side;
  for (int pass = 0; pass < 32; ++pass) {
    std::vector<double> gain(n, 0.0);
    for (int q = 0; q < n; ++q)
      for (int r = 0; r < n; ++r)
        if (w[q][r] != 0) gain[q] += side[r] != side[q] ? w[q][r] : -w[q][r];
    std::vector<char> locked(n, 0);
    int n1 = 0;
    for (int q = 0; q < n; ++q) n1 += side[q];
    std::vector<int> moves;
    double cur = 0, best = 0;
    size_t best_len = 0;
    std::vector<double> tie(n);
    for (int q = 0; q < n; ++q) tie[q] = rng.uniform();
    for (int it = 0; it < n; ++it) {
      int pick = -1;
      for (int q = 0; q < n; ++q) {
        if (locked[q]) continue;
        const int m1 = n1 + (side[q] ? -1 : 1);
        if (m1 < lo || m1 > hi) continue;
        if (pick < 0 || gain[q] > gain[pick] + 1e-12 || (std::fabs(gain[q] - gain[pick]) <= 1e-12 && tie[q] < tie[pick]))
          pick = q;
      }
      if (pick < 0) break;
      locked[pick] = 1;
      cur += gain[pick];
      n1 += side[pick] ? -1 : 1;
      side[pick] ^= 1;
      moves.push_back(pick);
      for (int r = 0; r < n; ++r)
        if (w[pick][r] != 0 && !locked[r]) gain[r] += side[r] == side[pick] ? -2 * w[pick][r] : 2 * w[pick][r];
      if (cur > best + 1e-9) best = cur, best_len = moves.size();
    }
    for (size_t i = best_len; i < moves.size(); ++i) side[moves[i]] ^= 1;
    if (best <= 1e-9) break;
  }
  double cut = 0;
  for (int q = 0; q < n; ++q)
    for (int r = q + 1; r < n; ++r)
      if (side[q] != side[r]) cut += w[q][r];
  if (cut_out) *cut_out = cut;
  return side;
}

// One side's stem: `ids` are its leaves in circuit order, `lq[i]` the qubits of leaf i's
// unsliced labels.  Blocks are formed greedily: start at the earliest leaf not absorbed,
// then add, among the leaves next in line on a qubit of the block (and next in line on all
// of their own qubits), the one that adds the fewest new qubits while the block stays within
// `fuse` qubits.  Appends the pairs to t and returns the stem's tensor id (-1 if no leaf).
int fused_stem(const std::vector<int>& ids, const std::vector<std::vector<int>>& lq, int n_qubits, int fuse,
               Tree& t) {
  if (ids.empty()) return -1;
  std::vector<std::vector<int>> queue(n_qubits);
  for (int i : ids)
    for (int q : lq[i]) queue[q].push_back(i);
  std::vector<size_t> head(n_qubits, 0);
  std::map<int, char> done;
  auto at_head = [&](int l) {
    for (int q : lq[l])
      if (head[q] >= queue[q].size() || queue[q][head[q]] != l) return false;
    return true;
  };
  auto pop = [&](int l) {
    for (int q : lq[l]) ++head[q];
    done[l] = 1;
  };
  auto add_qubits = [](std::vector<int>& Q, const std::vector<int>& more) {
    for (int r : more)
      if (std::find(Q.begin(), Q.end(), r) == Q.end()) Q.push_back(r);
  };
  // blocks in the order the stem absorbs them: their leaves and qubits
  std::vector<std::vector<int>> blocks;
  std::vector<std::vector<int>> bq;
  size_t next = 0;
  while (true) {
    while (next < ids.size() && done.count(ids[next])) ++next;
    if (next >= ids.size()) break;
    const int first = ids[next];
    std::vector<int> Q = lq[first];
    pop(first);
    std::vector<int> block{first};
    while (true) {
      int pick = -1;
      size_t pick_new = 0;
      for (int q : Q) {
        if (head[q] >= queue[q].size()) continue;
        const int l = queue[q][head[q]];
        if (!at_head(l)) continue;
        size_t add = 0;
        for (int r : lq[l]) add += std::find(Q.begin(), Q.end(), r) == Q.end();
        if (Q.size() + add > (size_t)fuse) continue;
        if (pick < 0 || add < pick_new || (add == pick_new && l < pick)) pick = l, pick_new = add;
      }
      if (pick < 0) break;
      add_qubits(Q, lq[pick]);
      pop(pick);
      block.push_back(pick);
    }
    blocks.push_back(block);
    bq.push_back(Q);
  }
  // consecutive blocks whose qubits together stay within `fuse` become one branch: the stem
  // absorbs them one after the other, so contracting them first changes nothing but the
  // number (and the width) of the large absorptions
  std::vector<std::vector<int>> merged{blocks[0]};
  std::vector<std::vector<int>> mq{bq[0]};
  for (size_t b = 1; b < blocks.size(); ++b) {
    std::vector<int> u = mq.back();
    add_qubits(u, bq[b]);
    if (u.size() <= (size_t)fuse) {
      merged.back().insert(merged.back().end(), blocks[b].begin(), blocks[b].end());
      mq.back() = u;
    } else {
      merged.push_back(blocks[b]);
      mq.push_back(bq[b]);
    }
  }
  auto join = [&](int x, int y) {
    if (x < 0) return y;
    t.pairs.emplace_back(x, y);
    t.sets.push_back(sym_diff(t.sets[x], t.sets[y]));
    return (int)t.sets.size() - 1;
  };
  int stem = -1;
  for (const auto& blk : merged) {
    int branch = -1;
    for (int l : blk) branch = join(branch, l);
    stem = join(stem, branch);
  }
  return stem;
}

// The qubit-split tree of one bisection: returns false when a side is empty.
bool split_tree(const Network& net, const std::vector<LabelSet>& leaves, const std::vector<char>& qside,
                int fuse, Tree& t, std::vector<int>& sliced) {
  const int L = (int)leaves.size();
  const int n = net.circ.n;
  std::vector<std::vector<int>> owners(net.edges.size());
  for (int i = 0; i < L; ++i)
    for (int e : leaves[i]) owners[e].push_back(i);
  // leaves on one side follow their qubits; straddling leaves take the side that leaves
  // fewer of their indices crossing (ties: the side of their first qubit)
  std::vector<int> lside(L, -1);
  std::vector<std::vector<int>> qs(L);
  for (int i = 0; i < L; ++i) {
    for (int e : leaves[i]) {
      const int q = net.edges[e].qubit;
      if (std::find(qs[i].begin(), qs[i].end(), q) == qs[i].end()) qs[i].push_back(q);
    }
    int c0 = 0, c1 = 0;
    for (int q : qs[i]) (qside[q] ? c1 : c0)++;
    if (c1 == 0) lside[i] = 0;
    else if (c0 == 0) lside[i] = 1;
  }
  for (int i = 0; i < L; ++i) {
    if (lside[i] >= 0) continue;
    int cross[2] = {0, 0};
    for (int s = 0; s < 2; ++s)
      for (int e : leaves[i]) {
        if (owners[e].size() != 2) continue;
        const int o = owners[e][0] == i ? owners[e][1] : owners[e][0];
        const int os = lside[o] >= 0 ? lside[o] : qside[net.edges[e].qubit];
        cross[s] += os != s;
      }
    lside[i] = cross[0] < cross[1] ? 0 : cross[1] < cross[0] ? 1 : (qs[i].empty() ? 0 : qside[qs[i][0]]);
  }
  int count[2] = {0, 0};
  for (int i = 0; i < L; ++i) count[lside[i]]++;
  if (count[0] == 0 || count[1] == 0) return false;
  std::vector<char> sl(net.edges.size(), 0);
  sliced.clear();
  for (size_t e = 0; e < owners.size(); ++e)
    if (owners[e].size() == 2 && lside[owners[e][0]] != lside[owners[e][1]]) {
      sl[e] = 1;
      sliced.push_back((int)e);
    }
  // qubits of each leaf's unsliced labels drive the fusion
  std::vector<std::vector<int>> lq(L);
  for (int i = 0; i < L; ++i)
    for (int e : leaves[i]) {
      if (sl[e]) continue;
      const int q = net.edges[e].qubit;
      if (std::find(lq[i].begin(), lq[i].end(), q) == lq[i].end()) lq[i].push_back(q);
    }
  t = Tree();
  t.sets = leaves;
  // sliced labels stay in the sets (cost functions skip them); the order is per side
  int root[2];
  for (int s = 0; s < 2; ++s) {
    std::vector<int> ids;
    for (int i = 0; i < L; ++i)
      if (lside[i] == s) ids.push_back(i);
    root[s] = fused_stem(ids, lq, n, fuse, t);
  }
  t.pairs.emplace_back(root[0], root[1]);
  t.sets.push_back(sym_diff(t.sets[root[0]], t.sets[root[1]]));
  return true;
}

}  // namespace

std::vector<SliceStat> slice_stats(const Plan& plan) {
  Tree t;
  t.sets = contraction_leaves(plan.net);
  const int L = (int)t.sets.size();
  for (auto& p : plan.tree) {
    t.pairs.push_back(p);
    t.sets.push_back(sym_diff(t.sets[p.first], t.sets[p.second]));
  }
  std::vector<char> sl(plan.net.edges.size(), 0);
  for (int e : plan.sliced) sl[e] = 1;
  const double c_all = tree_cost(t, sl), r_all = reuse_cost(t, sl, plan.sliced);
  std::vector<SliceStat> out(plan.sliced.size());
  for (size_t j = 0; j < plan.sliced.size(); ++j) {
    const int e = plan.sliced[j];
    SliceStat& st = out[j];
    std::vector<char> dep(t.sets.size(), 0);
    for (int i = 0; i < L; ++i) dep[i] = std::binary_search(t.sets[i].begin(), t.sets[i].end(), e) ? 1 : 0;
    for (size_t k = 0; k < t.pairs.size(); ++k) {
      const auto& p = t.pairs[k];
      const bool in_op = std::binary_search(t.sets[p.first].begin(), t.sets[p.first].end(), e) ||
                         std::binary_search(t.sets[p.second].begin(), t.sets[p.second].end(), e);
      if (in_op) {
        if (st.first_step < 0) st.first_step = (int)k;
        st.last_step = (int)k;
      }
      dep[L + k] = dep[p.first] | dep[p.second];
      st.dep_steps += dep[L + k];
    }
    // post-lifetime steps: they depend on e without containing it.  Summing over e's two
    // values right after its last step (Sec. III-B post-lifetime merging) would run each of
    // them once per assignment of the other sliced indices: half its executed cost saved.
    {
      const std::vector<int> dm = dep_counts(t, plan.sliced);
      double saved = 0;
      for (size_t k = 0; k < t.pairs.size(); ++k) {
        const auto& p = t.pairs[k];
        if ((int)k > st.last_step && dep[L + k]) {
          ++st.post_steps;
          const int u = (int)count_not_in(set_union(t.sets[p.first], t.sets[p.second]), sl);
          saved += 0.5 * std::ldexp(1.0, u + dm[L + k]);
        }
      }
      st.merge_saving = saved / r_all;
    }
    std::vector<int> rest;
    for (int x : plan.sliced)
      if (x != e) rest.push_back(x);
    sl[e] = 0;
    st.overhead = 2.0 * c_all / tree_cost(t, sl);
    st.reuse_overhead = r_all / reuse_cost(t, sl, rest);
    sl[e] = 1;
  }
  return out;
}

void plan_greedy(const Network& net, const PlanOpts& o, Plan& plan) {
  if (o.trials < 1 || o.log2_cap < 1 || o.log2_cap > 34 || o.slices_min < 0 || o.slices_max < 0)
    fail(1, "plan_greedy: bad options");
  const int n_edges = (int)net.edges.size();
  if (o.slicing < 0 || o.slicing > 1 || o.branch_exchange < 0 || o.branch_exchange > 1)
    fail(1, "plan_greedy: bad options");
  std::vector<LabelSet> leaves = contraction_leaves(net);
  if (leaves.empty()) fail(5, "plan_greedy: empty network");
  std::vector<char> is_open(n_edges, 0);
  for (int e : net.open_edge) is_open[e] = 1;

  struct Best {
    Tree tree;
    std::vector<int> sliced;
    double total = std::numeric_limits<double>::infinity();
    double score = std::numeric_limits<double>::infinity();
    double per_slice = 0, unsliced = 0;
    bool within_max = false;
  } best;

  // One candidate tree, with the indices already sliced (a separator, mode 2): slice while
  // an intermediate exceeds the cap, release separator indices the cap still admits, add
  // indices up to slices_min, then compare it with the best so far.
  auto consider = [&](Tree& t, std::vector<int> sliced) {
    std::vector<char> sl(n_edges, 0);
    for (int e : sliced) sl[e] = 1;
    const double c0 = tree_cost(t, std::vector<char>(n_edges, 0));
    double cur = tree_cost(t, sl);
    auto try_slice = [&](bool only_oversized) -> int {
      // candidates: labels of oversized tensors (or every inner label)
      std::set<int> cand;
      if (only_oversized) {
        for (auto& s : t.sets)
          if ((int)count_not_in(s, sl) > o.log2_cap)
            for (int e : s)
              if (!sl[e] && !is_open[e]) cand.insert(e);
      } else {
        for (auto& s : t.sets)
          for (int e : s)
            if (!sl[e] && !is_open[e]) cand.insert(e);
      }
      int pick = -1;
      double pick_cost = 0;
      int pick_over = -1;
      const double rcur = o.slicing == 1 ? reuse_cost(t, sl, sliced) : 0.0;
      for (int e : cand) {
        sl[e] = 1;
        double ov;
        if (o.slicing == 1) {
          // lifetime-aware: the executed cost under tree-like reuse grows by this factor
          std::vector<int> with = sliced;
          with.push_back(e);
          ov = reuse_cost(t, sl, with) / rcur;
        } else {
          // index overhead O(e) = 2 C_e / C (Eq. 1)
          ov = 2.0 * tree_cost(t, sl) / cur;
        }
        int over = 0;
        for (auto& s : t.sets) over += (int)count_not_in(s, sl) > o.log2_cap;
        sl[e] = 0;
        // ties: fewer oversized tensors left
        if (pick < 0 || ov < pick_cost * (1 - 1e-12) || (std::fabs(ov - pick_cost) <= 1e-12 * pick_cost && over < pick_over)) {
          pick = e;
          pick_cost = ov;
          pick_over = over;
        }
      }
      return pick;
    };
    while (tree_max(t, sl) > o.log2_cap) {
      int e = try_slice(true);
      if (e < 0) return;
      sl[e] = 1;
      sliced.push_back(e);
      cur = tree_cost(t, sl);
    }
    // release sliced indices while every intermediate stays within the cap and the total
    // cost 2^s * C does not grow (the separator of mode 2 may leave room under the cap)
    while (!sliced.empty() && (int)sliced.size() > o.slices_min) {
      int pick = -1;
      double pick_cost = 0;
      for (size_t j = 0; j < sliced.size(); ++j) {
        const int e = sliced[j];
        sl[e] = 0;
        if (tree_max(t, sl) <= o.log2_cap) {
          const double c = tree_cost(t, sl);
          if (c <= 2.0 * cur * (1 + 1e-12) && (pick < 0 || c < pick_cost)) pick = (int)j, pick_cost = c;
        }
        sl[e] = 1;
      }
      if (pick < 0) break;
      sl[sliced[pick]] = 0;
      sliced.erase(sliced.begin() + pick);
      cur = pick_cost;
    }
    while ((int)sliced.size() < o.slices_min) {
      int e = try_slice(false);
      if (e < 0) break;
      sl[e] = 1;
      sliced.push_back(e);
      cur = tree_cost(t, sl);
    }
    const double total = std::ldexp(cur, (int)sliced.size());
    // objective 0 with the lifetime-aware slicer: executed multiply-adds under reuse
    const double score =
        o.objective == 1 ? model_time(t, sl, sliced) : (o.slicing == 1 ? reuse_cost(t, sl, sliced) : total);
    const bool within = (int)sliced.size() <= o.slices_max;
    bool better;
    if (within != best.within_max) better = within;
    else better = score < best.score * (1 - 1e-12);
    if (better) {
      best.tree = t;
      best.sliced = sliced;
      best.total = total;
      best.score = score;
      best.per_slice = cur;
      best.unsliced = c0;
      best.within_max = within;
    }
  };

  // mode 2: qubit weights = 2-qubit leaves joining each pair of qubits
  const int nq = net.circ.n;
  std::vector<std::vector<double>> qw;
  if (o.mode == 2) {
    qw.assign(nq, std::vector<double>(nq, 0.0));
    for (const LabelSet& l : leaves) {
      std::vector<int> qs;
      for (int e : l)
        if (std::find(qs.begin(), qs.end(), net.edges[e].qubit) == qs.end()) qs.push_back(net.edges[e].qubit);
      for (size_t i = 0; i < qs.size(); ++i)
        for (size_t j = i + 1; j < qs.size(); ++j) qw[qs[i]][qs[j]] += 1, qw[qs[j]][qs[i]] += 1;
    }
  }
  for (int trial = 0; trial < o.trials; ++trial) {
    Rng rng{o.seed * 0x100000001B3ull + 0x9E3779B97F4A7C15ull * (uint64_t)(trial + 1)};
    if (leaves.size() == 1) {
      Tree t{{}, leaves};
      consider(t, {});
    } else if (o.mode == 2) {
      if (nq < 2) fail(1, "plan_greedy: mode 2 needs at least two qubits");
      // both sides within the cap when the circuit allows it
      const int max_side = std::min(nq - 1, std::max((nq + 1) / 2, std::min(o.log2_cap, nq - 1)));
      const std::vector<char> qside = bisect_qubits(nq, qw, max_side, rng, nullptr);
      for (int fuse : {2, 4, 6, 8, 10}) {
        Tree t;
        std::vector<int> sep;
        if (split_tree(net, leaves, qside, fuse, t, sep)) consider(t, sep);
      }
    } else {
      Tree t = o.mode == 1 ? stem_tree(leaves, n_edges, rng, trial == 0 ? 0.0 : o.temperature,
                                       (int)(rng.next() % leaves.size()))
                           : greedy_tree(leaves, n_edges, rng, trial == 0 ? 0.0 : o.temperature);
      consider(t, {});
    }
  }
  if (!std::isfinite(best.total)) fail(5, "plan_greedy: no trial met the size cap");
  if (o.branch_exchange) {
    // on the kept trial, with its slice set
    std::vector<char> sl(n_edges, 0);
    for (int e : best.sliced) sl[e] = 1;
    branch_exchange(best.tree, sl, best.sliced, o.log2_cap, o.slicing == 1, 8);
    best.per_slice = tree_cost(best.tree, sl);
    best.total = std::ldexp(best.per_slice, (int)best.sliced.size());
    best.unsliced = tree_cost(best.tree, std::vector<char>(n_edges, 0));
  }

  plan = Plan();
  plan.net = net;
  plan.opts = o;
  plan.sliced = best.sliced;
  plan.tree = best.tree.pairs;
  plan.log2_flops_slice = std::log2(best.per_slice);
  plan.log2_flops_total = std::log2(best.total);
  plan.overhead = best.total / best.unsliced;
  {
    std::vector<char> sl(n_edges, 0);
    for (int e : best.sliced) sl[e] = 1;
    plan.log2_flops_executed = std::log2(reuse_cost(best.tree, sl, best.sliced));
  }
  compile_plan(plan, true);
}

}  // namespace tnc
