// Host construction of the cluster tree, directions, block tree and the
// (cluster, direction) work lists of the compression.
//
// Floating-point decisions (split coordinate, admissibility, nearest
// direction) are computed in IEEE double with the operation order written
// here and no contraction (built with -ffp-contract=off), so that another
// implementation evaluating the same formulas in the same order reaches the
// same integer decisions.  The nearest-direction searches and the two sides'
// work lists run on several host threads; each result is written by one
// thread only, so the output does not depend on the thread count.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <new>
#include <stdexcept>
#include <thread>

#include "dh2_internal.h"

namespace dh2 {

namespace {

// f(i) for i in [0, n) on up to 16 host threads, contiguous ranges of at
// least `grain` indices (each f(i) writes only its own outputs, so the result
// does not depend on the split).
template <typename F>
void parallel_for(int64_t n, F f, int64_t grain = 256) {
  const int64_t hw = std::max<int64_t>(1, (int64_t)std::thread::hardware_concurrency());
  const int64_t nt = std::min<int64_t>({hw, (int64_t)16, std::max<int64_t>(1, n / grain)});
  if (nt <= 1) {
    for (int64_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::vector<std::thread> th;
  th.reserve((size_t)nt);
  for (int64_t k = 0; k < nt; ++k)
    th.emplace_back([&, k] {
      const int64_t lo = n * k / nt, hi = n * (k + 1) / nt;
      for (int64_t i = lo; i < hi; ++i) f(i);
    });
  for (auto& t : th) t.join();
}

// Section 3: midpoints of an m x m subdivision of each face of [-1,1]^3
// (face order +x,-x,+y,-y,+z,-z, squares row-major), projected to the sphere.
void cube_directions(int m, std::vector<double>& out) {
  out.clear();
  out.reserve((size_t)6 * m * m * 3);
  for (int face = 0; face < 6; ++face) {
    const int ax = face / 2;
    const double sgn = (face % 2 == 0) ? 1.0 : -1.0;
    int o0 = -1, o1 = -1;
    for (int d = 0; d < 3; ++d)
      if (d != ax) { if (o0 < 0) o0 = d; else o1 = d; }
    for (int a = 0; a < m; ++a) {
      const double u = -1.0 + (2.0 * a + 1.0) / m;
      for (int b = 0; b < m; ++b) {
        const double v = -1.0 + (2.0 * b + 1.0) / m;
        double p[3] = {0.0, 0.0, 0.0};
        p[ax] = sgn;
        p[o0] = u;
        p[o1] = v;
        const double nrm = std::sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
        out.push_back(p[0] / nrm);
        out.push_back(p[1] / nrm);
        out.push_back(p[2] / nrm);
      }
    }
  }
}

// argmin_j |u - D_j|^2, lowest j on ties.
int32_t nearest(const double* u, const std::vector<double>& D) {
  const size_t nd = D.size() / 3;
  int32_t best = 0;
  double bd = 0.0;
  for (size_t j = 0; j < nd; ++j) {
    const double d0 = u[0] - D[3 * j + 0];
    const double d1 = u[1] - D[3 * j + 1];
    const double d2 = u[2] - D[3 * j + 2];
    const double dd = d0 * d0 + d1 * d1 + d2 * d2;
    if (j == 0 || dd < bd) { bd = dd; best = (int32_t)j; }
  }
  return best;
}

double box_dist(const double* lo_t, const double* hi_t, const double* lo_s, const double* hi_s) {
  double acc = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double g = std::max(0.0, std::max(lo_s[a] - hi_t[a], lo_t[a] - hi_s[a]));
    acc = acc + g * g;
  }
  return std::sqrt(acc);
}

struct Builder {
  Tree& tr;
  const double* pts;
  int64_t offset = 0;
  explicit Builder(Tree& t, const double* p) : tr(t), pts(p) {}

  // Def. 1 by bisection; clusters numbered in pre-order, sons' index sets
  // contiguous in the permuted order.
  int32_t make(std::vector<int64_t>& idx, int32_t lvl, int32_t parent) {
    const int32_t cid = (int32_t)tr.start.size();
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) { lo[a] = pts[3 * idx[0] + a]; hi[a] = lo[a]; }
    for (size_t i = 1; i < idx.size(); ++i)
      for (int a = 0; a < 3; ++a) {
        const double v = pts[3 * idx[i] + a];
        if (v < lo[a]) lo[a] = v;
        if (v > hi[a]) hi[a] = v;
      }
    tr.start.push_back((int32_t)offset);
    tr.size.push_back((int32_t)idx.size());
    tr.level.push_back(lvl);
    tr.parent.push_back(parent);
    tr.son0.push_back(-1);
    tr.son1.push_back(-1);
    for (int a = 0; a < 3; ++a) {
      tr.lo.push_back(lo[a]);
      tr.hi.push_back(hi[a]);
      tr.center.push_back((lo[a] + hi[a]) * 0.5);
    }
    const double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
    tr.diam.push_back(std::sqrt(dx * dx + dy * dy + dz * dz));

    bool split = false;
    std::vector<int64_t> first, second;
    if ((int64_t)idx.size() > tr.params.leaf_size) {
      const double ext[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
      int ax = 0;
      for (int a = 1; a < 3; ++a)
        if (ext[a] > ext[ax]) ax = a;
      const double mid = (lo[ax] + hi[ax]) * 0.5;
      for (int64_t i : idx) (pts[3 * i + ax] <= mid ? first : second).push_back(i);
      split = !first.empty() && !second.empty();
    }
    if (split) {
      idx.clear();
      idx.shrink_to_fit();
      const int32_t s1 = make(first, lvl + 1, cid);
      const int32_t s2 = make(second, lvl + 1, cid);
      tr.son0[cid] = s1;
      tr.son1[cid] = s2;
    } else {
      for (size_t i = 0; i < idx.size(); ++i) tr.perm[offset + i] = idx[i];
      offset += (int64_t)idx.size();
      tr.max_leaf = std::max<int32_t>(tr.max_leaf, (int32_t)idx.size());
    }
    return cid;
  }

  // Def. 2 by the standard recursion with Eqs. (adm_standard), (adm_parabolic),
  // appending the leaves to `out` in depth-first order.  Below depth `cut`
  // the subtrees are not entered: their (t, s) pairs are appended to `defer`
  // and a placeholder (adm = -1, cb = index in defer) marks their place.
  void blocks(int32_t t, int32_t s, std::vector<Block>& out, int depth, int cut,
              std::vector<std::pair<int32_t, int32_t>>* defer) const {
    const double md = std::max(tr.diam[t], tr.diam[s]);
    const double d = box_dist(&tr.lo[3 * t], &tr.hi[3 * t], &tr.lo[3 * s], &tr.hi[3 * s]);
    const double eta2 = tr.params.eta2, kappa = tr.params.kappa;
    const bool adm = d > 0.0 && md <= eta2 * d && kappa * (md * md) <= eta2 * d;
    if (adm) {
      out.push_back({t, s, 1, -1});
    } else if (tr.is_leaf(t) || tr.is_leaf(s)) {
      out.push_back({t, s, 0, -1});
    } else if (defer && depth >= cut) {
      out.push_back({t, s, -1, (int32_t)defer->size()});
      defer->push_back({t, s});
    } else {
      const int32_t ts[2] = {tr.son0[t], tr.son1[t]};
      const int32_t ss[2] = {tr.son0[s], tr.son1[s]};
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) blocks(ts[i], ss[j], out, depth + 1, cut, defer);
    }
  }
};

void build_side(Tree& tr, int side) {
  Side& S = tr.side[side];
  const int32_t nc = tr.nclusters();
  auto width = [&](int32_t b) -> int64_t {
    const Block& B = tr.blocks[b];
    return side == kSideRow ? tr.size[B.s] : tr.size[B.t];
  };
  auto other_start = [&](int32_t b) -> int32_t {
    const Block& B = tr.blocks[b];
    return side == kSideRow ? tr.start[B.s] : tr.start[B.t];
  };
  // own admissible blocks per cluster and direction, ordered by the other
  // cluster's start: one sorted array with a range per cluster (clusters at
  // one level have distinct starts, so the order has no ties)
  struct OwnE {
    int32_t r, c, os, b;
  };
  std::vector<OwnE> ownv;
  for (int32_t b = 0; b < (int32_t)tr.blocks.size(); ++b) {
    const Block& B = tr.blocks[b];
    if (!B.adm) continue;
    ownv.push_back({side == kSideRow ? B.t : B.s, B.cb, other_start(b), b});
  }
  std::sort(ownv.begin(), ownv.end(), [](const OwnE& x, const OwnE& y) {
    if (x.r != y.r) return x.r < y.r;
    if (x.c != y.c) return x.c < y.c;
    return x.os < y.os;
  });
  std::vector<int64_t> own_ptr(nc + 1, 0);
  for (const OwnE& e : ownv) ++own_ptr[e.r + 1];
  for (int32_t r = 0; r < nc; ++r) own_ptr[r + 1] += own_ptr[r];

  // used pairs, top-down (pre-order numbering puts fathers first).  Column
  // order of (t, c): own blocks, then for each father pair (father, c_p) with
  // sd(c_p) = c in ascending c_p the father's columns -- so every father pair
  // is one contiguous column range of each of its son pairs.
  std::vector<Pair> tmp;
  std::vector<std::vector<std::pair<int32_t, int64_t>>> pair_of(nc);  // per cluster: (direction, pair), ascending
  std::vector<std::pair<int32_t, int64_t>> segs;                      // (son direction, father pair)
  std::vector<int32_t> used;
  for (int32_t r = 0; r < nc; ++r) {
    segs.clear();
    const int32_t par = tr.parent[r];
    if (par >= 0)
      for (const auto& kv : pair_of[par]) segs.push_back({tr.sd_of(tr.level[par], kv.first), kv.second});
    // by son direction; the father pairs of one direction stay in ascending c_p
    std::stable_sort(segs.begin(), segs.end(),
                     [](const std::pair<int32_t, int64_t>& x, const std::pair<int32_t, int64_t>& y) {
                       return x.first < y.first;
                     });
    used.clear();
    for (int64_t i = own_ptr[r]; i < own_ptr[r + 1]; ++i) used.push_back(ownv[i].c);
    for (const auto& sg : segs) used.push_back(sg.first);
    std::sort(used.begin(), used.end());
    used.erase(std::unique(used.begin(), used.end()), used.end());
    int64_t oi = own_ptr[r];
    size_t si = 0;
    for (const int32_t c : used) {
      Pair P;
      P.cluster = r;
      P.dir = c;
      P.level = tr.level[r];
      P.leaf = tr.is_leaf(r) ? 1 : 0;
      int64_t off = 0;
      for (; oi < own_ptr[r + 1] && ownv[oi].c == c; ++oi) {
        P.own.push_back(ownv[oi].b);
        off += width(ownv[oi].b);
      }
      for (; si < segs.size() && segs[si].first == c; ++si) {
        P.parents.push_back({segs[si].second, off});
        off += tmp[segs[si].second].ncols;
      }
      P.ncols = off;
      pair_of[r].push_back({c, (int64_t)tmp.size()});
      tmp.push_back(std::move(P));
    }
  }
  auto pair_at = [&](int32_t r, int32_t c) -> int64_t {
    const auto& v = pair_of[r];
    const auto it = std::lower_bound(v.begin(), v.end(), std::make_pair(c, (int64_t)INT64_MIN));
    if (it == v.end() || it->first != c) throw std::logic_error("son pair not used");
    return it->second;
  };
  // son links
  for (int64_t p = 0; p < (int64_t)tmp.size(); ++p) {
    Pair& P = tmp[p];
    if (P.leaf) continue;
    const int32_t cs = tr.sd_of(P.level, P.dir);
    const int32_t sons[2] = {tr.son0[P.cluster], tr.son1[P.cluster]};
    for (int j = 0; j < 2; ++j) {
      const int64_t q = pair_at(sons[j], cs);
      P.son_pair[j] = q;
      bool found = false;
      for (auto& seg : tmp[q].parents)
        if (seg.first == p) { P.son_off[j] = seg.second; found = true; }
      if (!found) throw std::logic_error("son pair without the father segment");
    }
  }
  // final order: level descending; in a level leaf pairs first
  std::vector<int64_t> order(tmp.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int64_t)i;
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    if (tmp[a].level != tmp[b].level) return tmp[a].level > tmp[b].level;
    return tmp[a].leaf > tmp[b].leaf;
  });
  std::vector<int64_t> newid(tmp.size());
  for (size_t i = 0; i < order.size(); ++i) newid[order[i]] = (int64_t)i;
  S.pairs.clear();
  S.pairs.reserve(tmp.size());
  for (int64_t o : order) {
    Pair P = std::move(tmp[o]);
    for (auto& seg : P.parents) seg.first = newid[seg.first];
    for (int j = 0; j < 2; ++j)
      if (P.son_pair[j] >= 0) P.son_pair[j] = newid[P.son_pair[j]];
    S.pairs.push_back(std::move(P));
  }
  S.leaf_pairs.clear();
  S.nonleaf_by_level.assign(tr.depth + 1, {});
  S.ncols_total = 0;
  for (int64_t p = 0; p < (int64_t)S.pairs.size(); ++p) {
    S.ncols_total += S.pairs[p].ncols;
    if (S.pairs[p].leaf) S.leaf_pairs.push_back(p);
    else S.nonleaf_by_level[S.pairs[p].level].push_back(p);
  }
  // block -> pair and offset in the pair's own range
  S.block_pair.assign(tr.blocks.size(), -1);
  S.block_off.assign(tr.blocks.size(), 0);
  for (int64_t p = 0; p < (int64_t)S.pairs.size(); ++p) {
    int64_t off = 0;
    for (int32_t b : S.pairs[p].own) {
      S.block_pair[b] = p;
      S.block_off[b] = off;
      off += width(b);
    }
  }
  // leaf column maps: one segment per block, the father segments expanded
  // recursively (the per-column entries are written on the device)
  S.leaf_colmap_off.assign(S.pairs.size() + 1, 0);
  S.seg_dst.clear();
  S.seg_col0.clear();
  S.seg_w.clear();
  S.seg_blk.clear();
  int64_t pos = 0;
  std::function<void(int64_t)> emit = [&](int64_t p) {
    const Pair& P = S.pairs[p];
    for (int32_t b : P.own) {
      const int64_t w = width(b);
      S.seg_dst.push_back(pos);
      S.seg_col0.push_back(other_start(b));
      S.seg_w.push_back((int32_t)w);
      S.seg_blk.push_back(b);
      pos += w;
    }
    for (auto& seg : P.parents) emit(seg.first);
  };
  S.seg_begin.assign(S.pairs.size() + 1, 0);
  for (int64_t p = 0; p < (int64_t)S.pairs.size(); ++p) {
    S.leaf_colmap_off[p] = pos;
    S.seg_begin[p] = (int64_t)S.seg_dst.size();
    if (S.pairs[p].leaf) emit(p);
  }
  S.leaf_colmap_off[S.pairs.size()] = pos;
  S.seg_begin[S.pairs.size()] = (int64_t)S.seg_dst.size();
  S.nleafcols = pos;
}

}  // namespace

int32_t Tree::sd_of(int32_t lvl, int32_t c) {
  int32_t& v = sd[lvl][c];
  if (v == -2) v = nearest(&dirs[lvl][3 * (size_t)c], dirs[lvl + 1]);
  return v;
}

dh2_status build_tree(const double* pts, int64_t n, const dh2_tree_params& p, Tree& tr) {
  if (!pts || n <= 0 || n > (int64_t)INT32_MAX / 2 || p.leaf_size < 1 || !(p.kappa >= 0.0) ||
      !(p.eta1 > 0.0) || !(p.eta2 > 0.0) || (p.dir_rule != 0 && p.dir_rule != 1))
    return DH2_EINVAL;
  for (int64_t i = 0; i < 3 * n; ++i)
    if (!std::isfinite(pts[i])) return DH2_EINVAL;
  tr = Tree();
  tr.n = n;
  tr.params = p;
  tr.perm.assign(n, 0);
  Builder B(tr, pts);
  {
    std::vector<int64_t> idx(n);
    for (int64_t i = 0; i < n; ++i) idx[i] = i;
    B.make(idx, 0, -1);
  }
  tr.depth = 0;
  for (int32_t l : tr.level) tr.depth = std::max(tr.depth, l);
  tr.delta.assign(tr.depth + 1, 0.0);
  for (int32_t t = 0; t < tr.nclusters(); ++t)
    if (tr.diam[t] > tr.delta[tr.level[t]]) tr.delta[tr.level[t]] = tr.diam[t];
  tr.dirs.resize(tr.depth + 1);
  tr.sd.resize(tr.depth + 1);
  for (int32_t l = 0; l <= tr.depth; ++l) {
    if (p.dir_rule == 1 && p.kappa * tr.delta[l] <= p.eta1) {
      tr.dirs[l].assign(3, 0.0);
    } else {
      const double x = std::sqrt(2.0) * p.kappa * tr.delta[l] / p.eta1;
      const double mc = std::ceil(x);
      if (!(mc <= 4096.0)) return DH2_EUNSUPPORTED;
      const int m = std::max(1, (int)mc);
      cube_directions(m, tr.dirs[l]);
    }
    tr.sd[l].assign(tr.dirs[l].size() / 3, l < tr.depth ? -2 : -1);
  }
  {
    // the block tree to depth 3, then its subtrees on several threads, spliced
    // back in depth-first order
    std::vector<Block> top;
    std::vector<std::pair<int32_t, int32_t>> defer;
    B.blocks(0, 0, top, 0, 3, &defer);
    std::vector<std::vector<Block>> sub(defer.size());
    parallel_for(
        (int64_t)defer.size(),
        [&](int64_t k) { B.blocks(defer[k].first, defer[k].second, sub[k], 0, 0, nullptr); }, 1);
    tr.blocks.clear();
    for (const Block& b : top) {
      if (b.adm >= 0) tr.blocks.push_back(b);
      else tr.blocks.insert(tr.blocks.end(), sub[b.cb].begin(), sub[b.cb].end());
    }
  }
  // block directions c_b: nearest direction to (m_t - m_s)/|m_t - m_s|
  double adm_entries = 0.0;
  for (Block& b : tr.blocks) {
    if (!b.adm) continue;
    ++tr.nadm;
    adm_entries += (double)tr.size[b.t] * (double)tr.size[b.s];
  }
  parallel_for((int64_t)tr.blocks.size(), [&](int64_t i) {
    Block& b = tr.blocks[i];
    if (!b.adm) return;
    double dv[3];
    for (int a = 0; a < 3; ++a) dv[a] = tr.center[3 * b.t + a] - tr.center[3 * b.s + a];
    const double nd = std::sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    const double u[3] = {dv[0] / nd, dv[1] / nd, dv[2] / nd};
    b.cb = nearest(u, tr.dirs[tr.level[b.t]]);
  });
  tr.adm_fraction = adm_entries / ((double)n * (double)n);
  // son maps of every direction a pair can take, level by level from the
  // root (a level's directions: its blocks' c_b and the son directions of the
  // level above), so that the two sides below read them concurrently
  {
    std::vector<std::vector<char>> used(tr.depth + 1);
    for (int32_t l = 0; l <= tr.depth; ++l) used[l].assign(tr.dirs[l].size() / 3, 0);
    for (const Block& b : tr.blocks)
      if (b.adm) used[tr.level[b.t]][b.cb] = 1;
    for (int32_t l = 0; l < tr.depth; ++l) {
      std::vector<int32_t> cs;
      for (int32_t c = 0; c < (int32_t)used[l].size(); ++c)
        if (used[l][c]) cs.push_back(c);
      parallel_for((int64_t)cs.size(), [&](int64_t i) {
        tr.sd[l][cs[i]] = nearest(&tr.dirs[l][3 * (size_t)cs[i]], tr.dirs[l + 1]);
      });
      for (int32_t c : cs) used[l + 1][tr.sd[l][c]] = 1;
    }
  }
  std::thread col([&] { build_side(tr, kSideCol); });
  build_side(tr, kSideRow);
  col.join();
  return DH2_OK;
}

}  // namespace dh2
