// Step compiler: turns a tree + slice set into the per-step program the device runs.
//
// For each pairwise contraction C = A * B (Sec. II-A) it fixes
//  * operand roles: the larger tensor is A and keeps its index order in C ("large
//    tensors stay at the multiplier position", Sec. V-A); B's free indices take the
//    positions A's contracted indices vacate, the rest go on top;
//  * tiles: sets of indices each CTA keeps on chip.  Because every index has dimension
//    2, an operand's tile is a sub-tensor over a set of its indices; choosing the tile
//    sets to contain each operand's lowest positions makes every load and store a run
//    of contiguous memory, so the permutation to the M x K x N view costs no extra
//    pass (the permutation is folded into the loads, Sec. V-A);
//  * the class: split over the common indices when M*N is small and K large (the
//    GEPDOT of Sec. II-A / Sec. V-B), fused on-chip chains of absorptions of small
//    tensors into one large one (Sec. IV), or the generic tiled contraction;
//  * device memory: every tensor gets an arena offset, reused once its last consumer ran.
#include <algorithm>
#include <cmath>
#include <map>
#include <set>

#include "host.h"

namespace tnc {

namespace {

int find_pos(const std::vector<int>& v, int x) {
  for (size_t i = 0; i < v.size(); ++i)
    if (v[i] == x) return (int)i;
  return -1;
}

bool contains(const std::vector<int>& v, int x) { return find_pos(v, x) >= 0; }

// C's storage order: A's free labels keep their positions' order; B's free labels
// fill the slots of A's common labels (in B's order), the remainder is appended.
std::vector<int> output_layout(const std::vector<int>& la, const std::vector<int>& lb) {
  std::vector<int> bfree;
  for (int x : lb)
    if (!contains(la, x)) bfree.push_back(x);
  std::vector<int> out;
  size_t nb = 0;
  for (int x : la) {
    if (!contains(lb, x)) out.push_back(x);
    else if (nb < bfree.size()) out.push_back(bfree[nb++]);
  }
  while (nb < bfree.size()) out.push_back(bfree[nb++]);
  return out;
}

// Lowest `k` labels of a layout.
std::vector<int> low(const std::vector<int>& l, int k) {
  return std::vector<int>(l.begin(), l.begin() + std::min<size_t>(l.size(), (size_t)k));
}

void add_unique(std::vector<int>& dst, int x) {
  if (!contains(dst, x)) dst.push_back(x);
}

// Tile limits (log2 entries): operand tiles <= 2^11, output tile <= 2^12.
constexpr int TILE_AB = 11;
constexpr int TILE_C = 12;

// Largest output tile (log2) that 256 threads cover with micro-tiles of up to 8 x 4.
int max_out_bits(int mt, int nt) { return 8 + std::min(3, mt) + std::min(2, nt); }

// Choose a tile for the generic / split-K kernels.
TileSpec choose_tile(const std::vector<int>& la, const std::vector<int>& lb, const std::vector<int>& lc,
                     int n_inst_hint, int& kind_out) {
  std::vector<int> M, K, N;
  for (int x : la) (contains(lb, x) ? K : M).push_back(x);
  for (int x : lb)
    if (!contains(la, x)) N.push_back(x);
  const int m = (int)M.size(), k = (int)K.size(), n = (int)N.size();
  TileSpec t;
  // GEPDOT steps (few outputs, long K) and the other streamed steps below are bound by memory:
  // operand tiles of 2^12 entries double the bytes each CTA has in flight per K step
  const bool gepdot = (m + n <= 10) && (k >= 12);
  // memory-bound long K loops (GEPDOTs, and at most 4 rows or columns): each loaded entry
  // feeds at most 4 multiply-adds, so they stream their tiles (k_stream)
  const bool stream = gepdot || (k >= 12 && std::min(m, n) <= 2);
  const int tile_ab = stream ? TILE_AB + 1 : TILE_AB;
  // GEMM-shaped steps on the SIMT kernel (the complex64 path): 128 x 64 output tiles with
  // 8 x 4 micro-tiles, 32 complex multiply-adds per 12 shared-memory loads
  const bool wide_out = !stream && k + n > 6 && m >= 7 && n >= 6 && k >= 5;
  const int tile_c = wide_out ? TILE_C + 1 : TILE_C;
  auto fits = [tile_ab, tile_c](const std::vector<int>& Mt, const std::vector<int>& Kt, const std::vector<int>& Nt) {
    const int mt = (int)Mt.size(), kt = (int)Kt.size(), nt = (int)Nt.size();
    return mt + kt <= tile_ab && kt + nt <= tile_ab && mt + nt <= tile_c && mt + nt <= max_out_bits(mt, nt);
  };
  // labels each tile must hold so that loads and stores run over contiguous memory
  for (int need = 4; need >= 0; --need) {
    std::vector<int> Mt, Kt, Nt;
    for (int x : low(la, need)) {
      if (contains(K, x)) add_unique(Kt, x);
      else add_unique(Mt, x);
    }
    for (int x : low(lb, need)) {
      if (contains(K, x)) add_unique(Kt, x);
      else add_unique(Nt, x);
    }
    for (int x : low(lc, need)) {
      if (contains(M, x)) add_unique(Mt, x);
      else add_unique(Nt, x);
    }
    if (!fits(Mt, Kt, Nt)) continue;
    t.Mt = Mt;
    t.Kt = Kt;
    t.Nt = Nt;
    break;
  }
  // grow the tiles by class, one label at a time while the limits hold
  auto grow = [&](std::vector<int>& tile, const std::vector<int>& pool, int target) {
    for (int x : pool) {
      if ((int)tile.size() >= target) break;
      if (contains(tile, x)) continue;
      tile.push_back(x);
      if (!fits(t.Mt, t.Kt, t.Nt)) {
        tile.pop_back();
        break;
      }
    }
  };
  // common labels by position, alternating between A and B, so that the K tile extends the
  // contiguous low runs of both operands (with K in A's order only, B's loads could be
  // short runs)
  std::vector<int> Kab;
  {
    std::vector<int> KB;
    for (int x : lb)
      if (contains(K, x)) KB.push_back(x);
    for (size_t i = 0; i < K.size(); ++i) {
      add_unique(Kab, K[i]);
      add_unique(Kab, KB[i]);
    }
  }
  if (gepdot) {
    grow(t.Mt, M, m);
    grow(t.Nt, N, n);
    grow(t.Kt, Kab, k);
  } else if (stream) {
    // a long K loop over a thin operand: all of the thin side, then A's labels in A's order
    // from its lowest position while they fit, so each tile row of A is one long run
    grow(t.Nt, N, n);
    for (int x : la) {
      if (contains(t.Mt, x) || contains(t.Kt, x)) continue;
      std::vector<int>& v = contains(K, x) ? t.Kt : t.Mt;
      v.push_back(x);
      if (!fits(t.Mt, t.Kt, t.Nt)) {
        v.pop_back();
        break;
      }
    }
  } else if (k + n <= 6) {
    // absorption of a small tensor: all of B on chip, a wide slice of A
    grow(t.Kt, Kab, k);
    grow(t.Nt, N, n);
    grow(t.Mt, M, std::min(m, 9));
  } else {
    grow(t.Mt, M, std::min(m, wide_out ? 7 : 6));
    grow(t.Nt, N, std::min(n, 6));
    grow(t.Kt, Kab, std::min(k, 5));
  }
  // canonical orders: M and K by A position, N by B position
  auto order_by = [](std::vector<int>& v, const std::vector<int>& layout) {
    std::sort(v.begin(), v.end(), [&](int x, int y) { return find_pos(layout, x) < find_pos(layout, y); });
  };
  order_by(t.Mt, la);
  order_by(t.Kt, la);
  order_by(t.Nt, lb);
  for (int x : M)
    if (!contains(t.Mt, x)) t.Mo.push_back(x);
  for (int x : K)
    if (!contains(t.Kt, x)) t.Ko.push_back(x);
  for (int x : N)
    if (!contains(t.Nt, x)) t.No.push_back(x);
  // micro-tile (up to 4 x 4 outputs per thread) and intra-CTA K groups, 256 threads
  const int mt = (int)t.Mt.size(), nt = (int)t.Nt.size(), kt = (int)t.Kt.size();
  const int out_bits = mt + nt;
  int lrm = 0, lrn = 0;
  if (stream) {
    // few outputs per K step: every thread takes the largest micro-tile (up to 4 x 4) over
    // its own k values (8 shared-memory loads per 16 complex multiply-adds), the K groups are
    // summed once at the end
    lrm = std::min(2, mt);
    lrn = std::min(2, nt);
  }
  while (out_bits - lrm - lrn > 8) {
    if (lrm <= lrn && lrm < 2 && lrm < mt) ++lrm;
    else if (lrn < 2 && lrn < nt) ++lrn;
    else if (lrm < 3 && lrm < mt) ++lrm;
    else break;
  }
  if (out_bits - lrm - lrn > 8) fail(5, "compile: output tile too large");
  t.rm = 1 << lrm;
  t.rn = 1 << lrn;
  const int threads_out = 1 << (out_bits - lrm - lrn);
  int kg = 256 / threads_out;
  kg = std::min(kg, 1 << kt);
  t.kgroups = std::max(1, kg);
  // split over the outer common labels for GEPDOT-shaped steps whose tiles leave SMs idle:
  // one wave of two CTAs per SM (the streaming kernel's occupancy), each with at least four
  // K steps for its cp.async ring.  Any count: CTA y takes the outer K steps
  // [y KO / splitk, (y + 1) KO / splitk)
  t.splitk = 1;
  const int ko = (int)t.Ko.size();
  if (gepdot && ko > 0) {
    const int64_t tiles = (int64_t(1) << (t.Mo.size() + t.No.size())) * std::max(1, n_inst_hint);
    const int64_t slots = 2 * 152;
    int64_t s = tiles >= slots ? 1 : (slots + tiles - 1) / tiles;
    s = std::min<int64_t>(s, (int64_t(1) << ko) / 4);
    t.splitk = (int)std::max<int64_t>(1, s);
  }
  t.gepdot = gepdot;
  t.stream = stream;
  kind_out = t.splitk > 1 ? K_SPLITK : K_GENERIC;
  return t;
}

// Tensor-core tile: 7 row labels from the operand with more free labels (A after an
// optional swap), 6 or 7 column labels (BN = 64 / 128), 4 or 5 K labels (BK = 16 / 32)
// whose first three are the k3 labels at positions 0..2 of both operands.  Returns false
// if the step does not qualify.
bool choose_tc_tile(const std::vector<int>& la0, const std::vector<int>& lb0, const std::vector<int>& lc,
                    const std::vector<int>& k3, TileSpec& t, bool& swap, int& bn, int& bk) {
  std::vector<int> M, K, N;
  for (int x : la0) (contains(lb0, x) ? K : M).push_back(x);
  for (int x : lb0)
    if (!contains(la0, x)) N.push_back(x);
  swap = N.size() > M.size();
  const std::vector<int>& la = swap ? lb0 : la0;
  const std::vector<int>& lb = swap ? la0 : lb0;
  if (swap) std::swap(M, N);
  if (M.size() < 7 || N.size() < 6 || K.size() < 4 || k3.size() != 3) return false;
  for (int j = 0; j < 3; ++j)
    if (la.size() < 3 || lb.size() < 3 || la[j] != k3[j] || lb[j] != k3[j]) return false;
  bn = N.size() >= 7 ? 128 : 64;
  bk = K.size() >= 5 ? 32 : 16;
  const size_t nt = bn == 128 ? 7 : 6, kt = bk == 32 ? 5 : 4;
  t = TileSpec();
  t.Kt = k3;
  for (int x : la) {  // further K labels by A position
    if (t.Kt.size() >= kt) break;
    if (contains(K, x) && !contains(t.Kt, x)) t.Kt.push_back(x);
  }
  for (int x : lc) {  // C's lowest labels first, so stores are runs
    if (contains(M, x) && t.Mt.size() < 7) t.Mt.push_back(x);
    else if (contains(N, x) && t.Nt.size() < nt) t.Nt.push_back(x);
    if (t.Mt.size() + t.Nt.size() >= 3) break;
  }
  for (int x : la)
    if (contains(M, x) && !contains(t.Mt, x) && t.Mt.size() < 7) t.Mt.push_back(x);
  for (int x : lb)
    if (contains(N, x) && !contains(t.Nt, x) && t.Nt.size() < nt) t.Nt.push_back(x);
  // C's three lowest positions must be tile labels
  for (int j = 0; j < 3; ++j)
    if (!contains(t.Mt, lc[j]) && !contains(t.Nt, lc[j])) return false;
  for (int x : M)
    if (!contains(t.Mt, x)) t.Mo.push_back(x);
  for (int x : K)
    if (!contains(t.Kt, x)) t.Ko.push_back(x);
  for (int x : N)
    if (!contains(t.Nt, x)) t.No.push_back(x);
  if (t.Mo.size() + t.No.size() > 30 || t.Ko.size() > 24) return false;
  return true;
}

}  // namespace

bool tc_tile_for(const std::vector<int>& la, const std::vector<int>& lb, const std::vector<int>& lc, TileSpec& t,
                 bool& swap, int& bn, int& bk) {
  if (la.size() < 3 || lb.size() < 3) return false;
  std::vector<int> k3(la.begin(), la.begin() + 3);
  return choose_tc_tile(la, lb, lc, k3, t, swap, bn, bk);
}

TileSpec tile_for(const std::vector<int>& la, const std::vector<int>& lb, const std::vector<int>& lc, int n_inst,
                  int& kind) {
  return choose_tile(la, lb, lc, n_inst, kind);
}

void compile_plan(Plan& plan, bool fuse) {
  const Network& net = plan.net;
  const int L = (int)net.leaves.size();
  plan.fuse = fuse;
  std::vector<char> sliced(net.edges.size(), 0);
  for (int e : plan.sliced) sliced[e] = 1;
  std::map<int, int> slice_bit;
  for (size_t t = 0; t < plan.sliced.size(); ++t) slice_bit[plan.sliced[t]] = (int)t;

  plan.tensors.clear();
  plan.leaf_fix.assign(L, {});
  for (int i = 0; i < L; ++i) {
    TensorInfo ti;
    ti.leaf = i;
    const auto& labs = net.leaves[i].t.labels;
    for (size_t p = 0; p < labs.size(); ++p) {
      int e = labs[p];
      const Edge& ed = net.edges[e];
      if (ed.kind == EDGE_OUTPUT && !ed.open) {
        plan.leaf_fix[i].push_back({(int)p, 1, ed.qubit});
      } else if (sliced[e]) {
        plan.leaf_fix[i].push_back({(int)p, 0, slice_bit[e]});
        if (slice_bit[e] < 64) ti.dep |= uint64_t(1) << slice_bit[e];
      } else {
        ti.labels.push_back(e);
      }
    }
    plan.tensors.push_back(ti);
  }
  // Tensor-core steps, decided on label sets from the root down: a step qualifies when both
  // operands are intermediates, M >= 2^7 rows (the larger operand A), N >= 2^5 columns and
  // K >= 2^4.  Its tile is Kt (4 or 5 common labels), Mt (7 of A's free labels) and Nt (5, 6,
  // 7 or 8 of B's), and it requires its operands' layouts to start with Kt then Mt (A) / Nt (B):
  // every operand tile is then one contiguous block, a plain box for the tensor memory
  // accelerator.  Mt / Nt include the first three labels its own consumer requires of its
  // output, so the output tile covers the output's lowest positions (contiguous stores).
  const int n_leaves = L;
  const int n_tree = (int)plan.tree.size();
  std::vector<std::vector<int>> sets(L);
  for (int i = 0; i < L; ++i) {
    sets[i] = plan.tensors[i].labels;
    std::sort(sets[i].begin(), sets[i].end());
  }
  for (int s = 0; s < n_tree; ++s) {
    const auto& A = sets[plan.tree[s].first];
    const auto& B = sets[plan.tree[s].second];
    std::vector<int> U;
    std::set_symmetric_difference(A.begin(), A.end(), B.begin(), B.end(), std::back_inserter(U));
    sets.push_back(U);
  }
  struct TcDec {
    bool ok = false;
    int bn = 128, bk = 32;
    int rows = -1;  // operand whose free labels are the tile rows (TMEM lanes)
    TileSpec t;
  };
  std::vector<TcDec> dec(n_tree);
  std::vector<std::vector<int>> req(L + n_tree);  // required leading labels of each intermediate
  // Which operand of intermediate t's producer contributes label x (0: the tree node's first,
  // 1: its second), and whether that producer can take the labels from that operand as its
  // tile columns: from the smaller operand as is, from the larger one by swapping roles,
  // which needs 7 row labels from the other side (the role rule below).
  auto side_of = [&](int t, int x) { return contains(sets[plan.tree[t - n_leaves].first], x) ? 0 : 1; };
  auto columns_ok = [&](int t, int sd) {
    const auto& P0 = sets[plan.tree[t - n_leaves].first];
    const auto& P1 = sets[plan.tree[t - n_leaves].second];
    const int larger = P1.size() > P0.size() ? 1 : 0;
    if (sd != larger) return true;
    std::vector<int> Kp;
    std::set_intersection(P0.begin(), P0.end(), P1.begin(), P1.end(), std::back_inserter(Kp));
    const size_t free_larger = (larger ? P1.size() : P0.size()) - Kp.size();
    const size_t free_smaller = (larger ? P0.size() : P1.size()) - Kp.size();
    return free_smaller >= 7 && free_larger >= 6;
  };
  for (int s = n_tree - 1; s >= 0; --s) {
    int a = plan.tree[s].first, b = plan.tree[s].second;
    if (sets[b].size() > sets[a].size()) std::swap(a, b);  // same roles as the layouts below
    const auto& A = sets[a];
    const auto& B = sets[b];
    std::vector<int> K, M, N;
    std::set_intersection(A.begin(), A.end(), B.begin(), B.end(), std::back_inserter(K));
    std::set_difference(A.begin(), A.end(), B.begin(), B.end(), std::back_inserter(M));
    std::set_difference(B.begin(), B.end(), A.begin(), A.end(), std::back_inserter(N));
    const std::vector<int>& rq = req[n_leaves + s];
    // roles: the result's leading labels (its consumer's requirement) should be tile
    // columns, so that each thread's TMEM row holds runs of consecutive result entries and
    // the epilogue can store them directly; swap rows and columns when most of the first
    // three are free labels of the larger operand
    {
      int in_m = 0, in_n = 0;
      for (size_t j = 0; j < rq.size() && j < 3; ++j) in_m += contains(M, rq[j]), in_n += contains(N, rq[j]);
      if (in_m > in_n && N.size() >= 7 && M.size() >= 6) {
        std::swap(a, b);
        std::swap(M, N);
      }
    }
    if (a < n_leaves || b < n_leaves || M.size() < 7 || N.size() < 5 || K.size() < 4) continue;
    TcDec d;
    d.ok = true;
    d.rows = a;
    d.bk = K.size() >= 5 ? 32 : 16;
    // 256-wide tiles take a whole SM (all TMEM) and leave the epilogue exposed; with at
    // most 8 K tiles the epilogue weighs, and 128-wide tiles run on the persistent kernel,
    // which overlaps it with the next tile
    const size_t kt0 = d.bk == 32 ? 5 : 4;
    d.bn = (N.size() >= 8 && K.size() > kt0 + 3) ? 256 : (N.size() >= 7 ? 128 : (N.size() >= 6 ? 64 : 32));
    const size_t kt = d.bk == 32 ? 5 : 4, nt = d.bn == 256 ? 8 : (d.bn == 128 ? 7 : (d.bn == 64 ? 6 : 5));
    // K-tile order: Kt[0..3] become the lowest positions of both operands, i.e. of both
    // producers' results.  A producer stores its tiles straight from registers (direct
    // epilogue) when its result's positions 0..2 are tile columns and position 3 a tile row:
    // three labels from one of its operands, the fourth from the other.  Take such labels
    // for both producers where K allows it, else for the larger operand's producer.
    std::vector<int> Kord = K;
    {
      int best = -1;
      std::vector<int> pick;
      for (int both = 1; both >= 0 && best < 0; --both)
        for (int sa = 0; sa < 2; ++sa)
          for (int sb = 0; sb < 2; ++sb) {
            if (!both && sb == 1) continue;
            std::vector<int> g, opp;
            for (int x : K) {
              const int xa = side_of(a, x), xb = side_of(b, x);
              if (xa == sa && (!both || xb == sb)) g.push_back(x);
              else if (xa != sa && (!both || xb != sb)) opp.push_back(x);
            }
            if (g.size() < 3 || opp.empty()) continue;
            const int score = (columns_ok(a, sa) ? 1 : 0) + (both && columns_ok(b, sb) ? 1 : 0);
            if (score > best) {
              best = score;
              pick = {g[0], g[1], g[2], opp[0]};
            }
          }
      if (best >= 0) {
        Kord = pick;
        for (int x : K)
          if (!contains(pick, x)) Kord.push_back(x);
      }
    }
    d.t.Kt.assign(Kord.begin(), Kord.begin() + kt);
    // the result's leading labels first, in their order: the lowest result positions are
    // then the lowest canonical column / row bits (runs per thread, adjacent rows per warp)
    for (size_t j = 0; j < rq.size(); ++j) {
      if (contains(M, rq[j]) && d.t.Mt.size() < 7) d.t.Mt.push_back(rq[j]);
      else if (contains(N, rq[j]) && d.t.Nt.size() < nt) d.t.Nt.push_back(rq[j]);
    }
    for (int x : M)
      if (d.t.Mt.size() < 7 && !contains(d.t.Mt, x)) d.t.Mt.push_back(x);
    for (int x : N)
      if (d.t.Nt.size() < nt && !contains(d.t.Nt, x)) d.t.Nt.push_back(x);
    for (int x : M)
      if (!contains(d.t.Mt, x)) d.t.Mo.push_back(x);
    for (int x : N)
      if (!contains(d.t.Nt, x)) d.t.No.push_back(x);
    for (int x : Kord)
      if (!contains(d.t.Kt, x)) d.t.Ko.push_back(x);
    if (d.t.Mt.size() != 7 || d.t.Nt.size() != nt || d.t.Mo.size() + d.t.No.size() > 30 || d.t.Ko.size() > 24) continue;
    req[a] = d.t.Kt;
    req[a].insert(req[a].end(), d.t.Mt.begin(), d.t.Mt.end());
    req[b] = d.t.Kt;
    req[b].insert(req[b].end(), d.t.Nt.begin(), d.t.Nt.end());
    dec[s] = d;
  }
  // intermediates
  plan.steps.clear();
  plan.n_gemm = plan.n_gepdot = plan.n_absorb = plan.n_fused = 0;
  plan.model_seconds = 0;
  plan.narrow_max = 0;
  plan.max_log2 = 0;
  for (auto& ti : plan.tensors) plan.max_log2 = std::max(plan.max_log2, (int)ti.labels.size());
  for (size_t s = 0; s < plan.tree.size(); ++s) {
    int a = plan.tree[s].first, b = plan.tree[s].second;
    if (plan.tensors[b].labels.size() > plan.tensors[a].labels.size()) std::swap(a, b);
    TensorInfo ci;
    ci.labels = output_layout(plan.tensors[a].labels, plan.tensors[b].labels);
    const int cid = (int)plan.tensors.size();
    std::vector<int> lead = req[cid];
    if (lead.empty() && dec[s].ok) {
      // a tensor-core step whose consumer is not one: its own tile labels lead -- three tile
      // columns, a tile row, then the rest of the tile -- so its epilogue stores straight from
      // registers in runs as long as the tile
      const TileSpec& t = dec[s].t;
      lead = {t.Nt[0], t.Nt[1], t.Nt[2], t.Mt[0]};
      lead.insert(lead.end(), t.Nt.begin() + 3, t.Nt.end());
      lead.insert(lead.end(), t.Mt.begin() + 1, t.Mt.end());
    }
    if (!lead.empty()) {
      // the leading labels in order (the consumer's tensor-core tile labels, or the step's
      // own); the rest keep their order
      std::vector<int> rest;
      for (int x : ci.labels)
        if (!contains(lead, x)) rest.push_back(x);
      ci.labels = lead;
      ci.labels.insert(ci.labels.end(), rest.begin(), rest.end());
    }
    ci.producer = (int)s;
    // tree-like reuse (Sec. III-B): a result depends on the sliced indices its subtree fixes
    ci.dep = plan.tensors[a].dep | plan.tensors[b].dep;
    plan.max_log2 = std::max(plan.max_log2, (int)ci.labels.size());
    Step st;
    st.a = a;
    st.b = b;
    st.c = (int)plan.tensors.size();
    plan.tensors.push_back(ci);
    plan.steps.push_back(st);
  }
  plan.root = plan.tree.empty() ? 0 : (int)plan.tensors.size() - 1;
  // executed complex multiply-adds of all slices of one row under tree-like reuse with
  // post-lifetime merging (Sec. III-B), the executor's rule: the step whose two operands both
  // depend on a sliced index sums its result over that index (except the root step), and
  // later steps no longer depend on it
  {
    std::vector<uint64_t> md(plan.tensors.size(), 0);
    for (size_t i = 0; i < plan.tensors.size(); ++i) md[i] = plan.tensors[i].dep;
    double ex = 0;
    for (size_t s = 0; s < plan.steps.size(); ++s) {
      const Step& st = plan.steps[s];
      const uint64_t full = md[st.a] | md[st.b];
      std::vector<int> u = plan.tensors[st.a].labels;
      for (int x : plan.tensors[st.b].labels)
        if (!contains(u, x)) u.push_back(x);
      ex += std::ldexp(1.0, (int)u.size() + __builtin_popcountll(full));
      const uint64_t m = s + 1 < plan.steps.size() ? (md[st.a] & md[st.b]) : 0;
      md[st.c] = full & ~m;
    }
    plan.log2_flops_executed_merged = plan.steps.empty() ? 0.0 : std::log2(ex);
  }
  // classify + tiles
  for (size_t s = 0; s < plan.steps.size(); ++s) {
    Step& st = plan.steps[s];
    const auto& la = plan.tensors[st.a].labels;
    const auto& lb = plan.tensors[st.b].labels;
    const auto& lc = plan.tensors[st.c].labels;
    int kind = K_GENERIC;
    // split sizing of the SIMT steps assumes every slice of the plan in flight, at most 2^12
    st.tile = choose_tile(la, lb, lc, 1 << std::min<int>((int)plan.sliced.size(), 12), kind);
    st.kind = kind;
    st.tc_ok = dec[s].ok;
    if (st.tc_ok) {
      st.tc_tile = dec[s].t;
      st.tc_swap = dec[s].rows != st.a;  // rows from b when the roles were swapped
      st.tc_bn = dec[s].bn;
      st.tc_bk = dec[s].bk;
      // the layouts honour the requirement: operands lead with Kt + Mt / Kt + Nt
      const auto& lr = st.tc_swap ? lb : la;
      const auto& lcol = st.tc_swap ? la : lb;
      const size_t kt = st.tc_tile.Kt.size();
      for (size_t j = 0; j < kt; ++j)
        if (lr[j] != st.tc_tile.Kt[j] || lcol[j] != st.tc_tile.Kt[j]) fail(5, "compile: tensor-core K labels not leading");
      for (size_t j = 0; j < st.tc_tile.Mt.size(); ++j)
        if (lr[kt + j] != st.tc_tile.Mt[j]) fail(5, "compile: tensor-core M labels not leading");
      for (size_t j = 0; j < st.tc_tile.Nt.size(); ++j)
        if (lcol[kt + j] != st.tc_tile.Nt[j]) fail(5, "compile: tensor-core N labels not leading");
    }
    int nk = 0;
    for (int x : la) nk += contains(lb, x);
    int nm = (int)la.size() - nk, nn = (int)lb.size() - nk;
    if (!la.empty() || !lb.empty()) {
      double narrow = (la.size() + lb.size()) ? 2.0 * nk / double(la.size() + lb.size()) : 0;
      plan.narrow_max = std::max(plan.narrow_max, narrow);
    }
    if (nm + nn <= 8 && nk >= 12) plan.n_gepdot++;
    else if (nk + nn <= 6) plan.n_absorb++;
    else plan.n_gemm++;
    // per slice, averaged over a call on every slice with tree-like reuse (a step runs once
    // per assignment of the sliced indices its result depends on)
    plan.model_seconds += step_model_seconds((int)la.size(), (int)lb.size(), (int)lc.size(), nk) *
                          std::ldexp(1.0, __builtin_popcountll(plan.tensors[st.c].dep) - (int)plan.sliced.size());
  }
  // fused chains (Sec. IV): follow the big operand through consecutive absorptions of
  // small tensors (rank <= 6) while the on-chip label set stays within 2^15 entries (a
  // tile above 2^12 is spread over a thread-block cluster of up to 8 CTAs).  The
  // first big operand keeps on chip its four lowest positions (contiguous loads) and every
  // label the chain contracts; labels brought in by the small tensors join it; the chain's
  // result must have its three lowest positions on chip (contiguous stores).  A fused
  // section of n links saves 2(n-1) passes over the big tensor.
  plan.chains.clear();
  plan.step_chain.assign(plan.steps.size(), -1);
  if (fuse) {
    auto is_link = [&](size_t j) {
      const Step& st = plan.steps[j];
      return st.kind == K_GENERIC && !st.tc_ok && plan.tensors[st.b].labels.size() <= 6 &&
             plan.tensors[st.a].labels.size() >= 10;
    };
    // 2^12 entries per CTA (the chain kernel's buffers), times up to 2^3 CTAs per cluster
    // when the plan allows cluster-cooperative chains
    constexpr size_t kTileBitsCta = 12;
    const size_t kInnerMax = kTileBitsCta + (plan.opts.cluster_chains ? 3 : 0);
    for (size_t i = 0; i < plan.steps.size(); ++i) {
      if (plan.step_chain[i] >= 0 || !is_link(i)) continue;
      const std::vector<int>& A0 = plan.tensors[plan.steps[i].a].labels;
      std::vector<int> inner0(A0.begin(), A0.begin() + std::min<size_t>(4, A0.size()));
      std::vector<size_t> links;
      std::vector<int> best_inner;
      size_t best_len = 0;
      for (size_t j = i; j < plan.steps.size(); ++j) {
        if (!is_link(j) || plan.step_chain[j] >= 0) break;
        if (j > i && plan.steps[j].a != plan.steps[j - 1].c) break;
        // tentative inner set with this link's contracted labels of A0 added
        std::vector<int> cand = inner0;
        const auto& la = plan.tensors[plan.steps[j].a].labels;
        const auto& lb = plan.tensors[plan.steps[j].b].labels;
        for (int x : la)
          if (contains(lb, x) && contains(A0, x)) add_unique(cand, x);
        // simulate the on-chip sets
        std::vector<int> I = cand;
        size_t mx = I.size();
        bool ok = true;
        for (size_t l = i; l <= j && ok; ++l) {
          const auto& a = plan.tensors[plan.steps[l].a].labels;
          const auto& b = plan.tensors[plan.steps[l].b].labels;
          std::vector<int> nI;
          for (int x : I)
            if (!contains(b, x)) nI.push_back(x);
          for (int x : b)
            if (!contains(a, x)) nI.push_back(x);
          for (int x : b)
            if (contains(a, x) && !contains(I, x)) ok = false;  // contracted label not on chip
          I = nI;
          mx = std::max(mx, I.size());
        }
        if (!ok || mx > kInnerMax) break;
        inner0 = cand;
        links.push_back(j);
        // the result's lowest positions must be on chip
        const auto& lc = plan.tensors[plan.steps[j].c].labels;
        bool store_ok = true;
        for (size_t q = 0; q < std::min<size_t>(3, lc.size()); ++q) store_ok = store_ok && contains(I, lc[q]);
        if (store_ok && links.size() >= 2) {
          best_len = links.size();
          best_inner = inner0;
        }
      }
      if (best_len >= 2) {
        // widen the on-chip set with A0's untouched low-position labels while every tile of
        // the chain stays within 2^12 entries, or within the chain's own largest tile when
        // that is larger (larger tiles amortize each CTA's setup; a wider tile would only
        // spread the chain over more CTAs)
        auto max_tile = [&](const std::vector<int>& in0) {
          std::vector<int> I = in0;
          size_t mx = I.size();
          for (size_t l = 0; l < best_len; ++l) {
            const auto& a = plan.tensors[plan.steps[links[l]].a].labels;
            const auto& b = plan.tensors[plan.steps[links[l]].b].labels;
            std::vector<int> nI;
            for (int x : I)
              if (!contains(b, x)) nI.push_back(x);
            for (int x : b)
              if (!contains(a, x)) nI.push_back(x);
            I = nI;
            mx = std::max(mx, I.size());
          }
          return mx;
        };
        const size_t widen_to = std::max<size_t>(kTileBitsCta, max_tile(best_inner));
        for (int x : A0) {
          if (contains(best_inner, x)) continue;
          best_inner.push_back(x);
          if (max_tile(best_inner) > widen_to) {
            best_inner.pop_back();
            break;
          }
        }
        Chain ch;
        ch.steps.assign(links.begin(), links.begin() + best_len);
        ch.inner0 = best_inner;
        for (int sidx : ch.steps) plan.step_chain[sidx] = (int)plan.chains.size();
        plan.n_fused += (int)best_len;
        plan.chains.push_back(ch);
      }
    }
  }
  // liveness + arena (first fit over a sorted free list, per instance, in complex elements;
  // planar storage takes 2 * 2^rank scalars, so offsets are kept in scalars)
  for (auto& ti : plan.tensors) ti.last_use = -1;
  for (size_t s = 0; s < plan.steps.size(); ++s) {
    plan.tensors[plan.steps[s].a].last_use = (int)s;
    plan.tensors[plan.steps[s].b].last_use = (int)s;
  }
  plan.tensors[plan.root].last_use = (int)plan.steps.size();
  std::vector<std::pair<int64_t, int64_t>> freelist;  // (offset, size) in scalars
  int64_t top = 0;
  auto alloc = [&](int64_t size) -> int64_t {
    // align to 64 scalars (>= 128 B for every precision)
    size = (size + 63) & ~int64_t(63);
    for (size_t i = 0; i < freelist.size(); ++i) {
      if (freelist[i].second >= size) {
        int64_t off = freelist[i].first;
        freelist[i].first += size;
        freelist[i].second -= size;
        if (freelist[i].second == 0) freelist.erase(freelist.begin() + i);
        return off;
      }
    }
    int64_t off = top;
    top += size;
    return off;
  };
  auto release = [&](int64_t off, int64_t size) {
    size = (size + 63) & ~int64_t(63);
    freelist.emplace_back(off, size);
    std::sort(freelist.begin(), freelist.end());
    std::vector<std::pair<int64_t, int64_t>> merged;
    for (auto& f : freelist) {
      if (!merged.empty() && merged.back().first + merged.back().second == f.first) merged.back().second += f.second;
      else merged.push_back(f);
    }
    freelist.swap(merged);
  };
  auto scalars = [](const TensorInfo& t) { return int64_t(2) << t.labels.size(); };
  for (int i = 0; i < L; ++i) plan.tensors[i].offset = alloc(scalars(plan.tensors[i]));
  for (size_t s = 0; s < plan.steps.size(); ++s) {
    Step& st = plan.steps[s];
    // the output may not overlap its inputs: allocate before releasing them
    plan.tensors[st.c].offset = alloc(scalars(plan.tensors[st.c]));
    for (int opnd : {st.a, st.b})
      if (plan.tensors[opnd].last_use == (int)s) release(plan.tensors[opnd].offset, scalars(plan.tensors[opnd]));
  }
  plan.arena_elems = top;  // scalars per instance

  // fused program: a chain runs at its last link, so its inputs (the first large operand
  // and every small one) stay allocated until its result is; its intermediates take no memory
  for (auto& ti : plan.tensors) ti.offset_fused = -1;
  if (plan.chains.empty()) {
    for (auto& ti : plan.tensors) ti.offset_fused = ti.offset;
    plan.arena_elems_fused = plan.arena_elems;
    return;
  }
  std::vector<std::vector<int>> unit_in, unit_out;  // execution units in order
  for (size_t s = 0; s < plan.steps.size(); ++s) {
    const int ci = plan.step_chain[s];
    if (ci < 0) {
      unit_in.push_back({plan.steps[s].a, plan.steps[s].b});
      unit_out.push_back({plan.steps[s].c});
      continue;
    }
    const Chain& ch = plan.chains[ci];
    if ((int)s != ch.steps.back()) continue;
    std::vector<int> ins = {plan.steps[ch.steps.front()].a};
    for (int sidx : ch.steps) ins.push_back(plan.steps[sidx].b);
    unit_in.push_back(ins);
    unit_out.push_back({plan.steps[ch.steps.back()].c});
  }
  std::vector<int> last_unit(plan.tensors.size(), -1);
  for (size_t u = 0; u < unit_in.size(); ++u)
    for (int t : unit_in[u]) last_unit[t] = (int)u;
  last_unit[plan.root] = (int)unit_in.size();
  freelist.clear();
  top = 0;
  for (int i = 0; i < L; ++i) plan.tensors[i].offset_fused = alloc(scalars(plan.tensors[i]));
  for (size_t u = 0; u < unit_in.size(); ++u) {
    for (int t : unit_out[u]) plan.tensors[t].offset_fused = alloc(scalars(plan.tensors[t]));
    for (int t : unit_in[u])
      if (last_unit[t] == (int)u) release(plan.tensors[t].offset_fused, scalars(plan.tensors[t]));
  }
  plan.arena_elems_fused = top;
}

}  // namespace tnc
