// C ABI of the library: tree queries, device upload of the work lists, the
// level schedule of the compression, matrix-vector product, error, export.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include <cstdio>

#include "dh2_check.cuh"
#include "dh2_internal.h"
#include "dh2_kernels.cuh"
#include "dh2_ops.cuh"

using namespace dh2;

#define DH2_CUDA_TRY(x)                   \
  do {                                    \
    if ((x) != cudaSuccess) {             \
      cudaGetLastError();                 \
      return DH2_ECUDA;                   \
    }                                     \
  } while (0)

namespace dh2 {

constexpr int kLeafClasses = 5;
inline bool mode_f32(int mode) { return mode != DH2_MODE_FP64; }  // complex64 data, FP32 kernels
inline bool mode_mixed(int mode) { return mode == DH2_MODE_MIXED_BF16X3; }
inline int leaf_class(int m) { return m <= 32 ? 0 : m <= 40 ? 1 : m <= 48 ? 2 : m <= 64 ? 3 : 4; }

// The process's tuning table (dh2_tuning_set, dh2_autotune): read once by each
// compression when it prepares its launches.
std::mutex g_tune_mu;
TuneTable g_tune = {{32, 32, 32, 32, 32}, {1, 1, 1, 1}, 0, 0, 1024};
TuneTable tune_current() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return g_tune;
}
bool tune_valid(const dh2_tuning& t) {
  for (int c = 0; c < 5; ++c) {
    const int v = t.jacobi_tpp[c];
    if (v != 4 && v != 8 && v != 16 && v != 32) return false;
  }
  for (int c = 0; c < 4; ++c)
    if (t.jacobi_narrow[c] < 0 || t.jacobi_narrow[c] > 2) return false;
  return t.rq_ctas_per_sm >= 0 && t.rq_ctas_per_sm <= 4 && (t.rq_tensor == 0 || t.rq_tensor == 1) &&
         (t.level_seg_cols == 0 || (t.level_seg_cols >= 256 && t.level_seg_cols <= 8192 && t.level_seg_cols % 64 == 0));
}
TuneTable to_table(const dh2_tuning& t) {
  TuneTable x{};
  for (int c = 0; c < 5; ++c) x.jacobi_tpp[c] = t.jacobi_tpp[c];
  for (int c = 0; c < 4; ++c) x.jacobi_narrow[c] = t.jacobi_narrow[c];
  x.rq_ctas_per_sm = t.rq_ctas_per_sm;
  x.rq_tensor = t.rq_tensor;
  x.level_seg_cols = t.level_seg_cols;
  return x;
}
dh2_tuning from_table(const TuneTable& x) {
  dh2_tuning t{};
  for (int c = 0; c < 5; ++c) t.jacobi_tpp[c] = x.jacobi_tpp[c];
  for (int c = 0; c < 4; ++c) t.jacobi_narrow[c] = x.jacobi_narrow[c];
  t.rq_ctas_per_sm = x.rq_ctas_per_sm;
  t.rq_tensor = x.rq_tensor;
  t.level_seg_cols = x.level_seg_cols;
  return t;
}

// Device copy of a tree's work lists (one arena, uploaded on first use).
struct Tree::Dev {
  void* arena = nullptr;
  // clusters
  int32_t *cstart, *csize, *clevel;
  // per side, per pair
  int32_t *cluster[2], *leaf[2], *start[2], *m[2], *ncols[2], *son[2], *sonoff[2], *level[2], *kcap[2],
      *rowcap[2];
  int64_t *cmoff[2], *Roff[2], *Qoff[2], *Xoff[2], *hoff[2];
  int64_t* gram_off[2];  // mixed modes: leaf Gram matrix offsets
  int32_t *gcol[2], *gblk[2];
  int64_t* seg_dst[2];  // column-map segments (expanded into gcol/gblk on upload)
  int64_t* seg_begin[2];  // per pair: first segment
  int32_t *seg_col0[2], *seg_w[2], *seg_blk[2];
  int32_t* iota[2];        // 0..npairs-1
  int32_t* leaf_list[2];   // leaf pair ids
  // blocks
  int32_t *bt, *bs, *badm, *bpair[2], *boff_row;
  int64_t *near_off, *Soff, *bmax_off;
  int32_t *adm_list, *inadm_list;
  int64_t* norm_pieces;  // admissible blocks' norms pass: b << 32 | 32-row slab << 16 | column group
  int64_t* norm_pbegin;  // per admissible block (adm_list order) its first piece; nadm + 1 entries
  int64_t nnorm_pieces = 0;
  // matvec lists (row side; the column side's serve the adjoint product)
  int64_t *own_ptr, *par_ptr;
  int32_t *own_blk, *par_pair, *par_son;
  int64_t *own_ptr_c, *par_ptr_c;
  int32_t *own_blk_c, *par_pair_c, *par_son_c;
  // launch orders: leaf launch (both sides) then non-leaf per level
  uint32_t* codes;
  // R tiles in the same order: code << 32 | first column, 32 columns each
  int64_t* tiles;
  // host-side sizes
  int64_t npairs[2] = {0, 0}, nleaf[2] = {0, 0};
  int64_t R_elems[2] = {0, 0}, Q_elems[2] = {0, 0}, X_elems[2] = {0, 0}, h_elems[2] = {0, 0};
  int64_t gram_elems = 0;  // both sides together
  int64_t S_elems = 0, near_elems = 0, bmax_elems = 0;
  int64_t nadm = 0, ninadm = 0;
  int64_t nleaf_codes = 0;
  // leaf codes grouped by size class (rows <= 32, <= 40, <= 48, <= 64, more), each
  // group costliest first; the pair kernel's CTA is sized to the class
  int64_t leaf_class_begin[kLeafClasses + 1] = {};
  int32_t leaf_class_maxm[kLeafClasses] = {};
  std::vector<int64_t> nl_code_begin, nl_code_count;    // per level
  int64_t nleaf_tiles = 0;
  int64_t leaf_tile_class_begin[kLeafClasses + 1] = {};  // leaf tiles of each size class
  std::vector<int64_t> nl_tile_begin, nl_tile_count;    // per level
  std::vector<int32_t> nl_rowcap_max;                   // per level
  std::vector<int64_t> lvl_begin[2], lvl_nl_begin[2], lvl_end[2];
  int32_t max_leaf = 0;
  std::vector<int32_t> kcap_h[2], rowcap_h[2];
  std::vector<int64_t> Qoff_h[2], Soff_h;
};

}  // namespace dh2

struct dh2_matrix {
  dh2_tree* tree = nullptr;
  int device = 0;
  int mode = 0;
  dh2_dtype dtype = DH2_C64;
  size_t es = 8;  // bytes per complex element
  cudaStream_t stream = nullptr;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  void* R[2] = {nullptr, nullptr};
  void* Q[2] = {nullptr, nullptr};
  void* X[2] = {nullptr, nullptr};
  void* colw[2] = {nullptr, nullptr};  // per column-map entry 1/omega (FP32 or FP64)
  double* sig[2] = {nullptr, nullptr};
  int32_t* rank[2] = {nullptr, nullptr};
  void* S = nullptr;
  void* near = nullptr;
  double* invw = nullptr;
  double* bnorm2 = nullptr;  // per block |G_b|_F^2 (admissible blocks)
  double* eps2 = nullptr;
  double* zpow = nullptr;
  uint32_t* status = nullptr;
  double* acc = nullptr;
  const void* G = nullptr;
  int64_t ld = 0;
  int nearfield_copy = 1;
  bool v_expanded = false;
  std::vector<double> eps2_h, zpow_h;
  float phase_ms[6] = {0, 0, 0, 0, 0, 0};
  float leaf_split_ms[2] = {0, 0};  // mixed modes, device input: leaf Gram launches, leaf factor launches
  int32_t launches = 0;  // kernels launched by the last compression (shared by a batch)
  int32_t class_launches[DH2_KC_COUNT] = {};  // the same launches by kernel class
  void* gram = nullptr;  // mixed modes with keep_gram: the leaf Gram matrices (double-float complex)
  // matrix-free mode
  int gen = 0;
  double* pts = nullptr;  // device, permuted order
  double kappa = 0.0, diag = 0.0;
  std::vector<double> pts_h;
  double* nrm = nullptr;  // device normals after the points (double layer), or NULL
};

namespace {

template <typename V>
size_t bytes_of(const std::vector<V>& v) {
  return v.size() * sizeof(V);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Every device allocation of the library goes through dev_malloc /
// dev_malloc_async, so that a test can make the n-th one fail as if the device
// were out of memory (dh2_debug_fail_alloc): 0 = off, k > 0 = the k-th
// allocation from now is refused.
std::atomic<int> g_fail_alloc{0};

bool alloc_refused() {
  int k = g_fail_alloc.load();
  while (k > 0)
    if (g_fail_alloc.compare_exchange_weak(k, k - 1)) return k == 1;
  return false;
}

cudaError_t dev_malloc(void** p, size_t bytes) {
  if (alloc_refused()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t st) {
  if (alloc_refused()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocAsync(p, bytes, st);
}

// Capacities: leaf rank <= min(rows, #F); non-leaf rank <= min(k_cap(t1c') +
// k_cap(t2c'), #F, 128).  Offsets of R (k_cap x #F), Q ([E1;E2] rowcap x k_cap)
// and of the expanded non-leaf bases (#t x k_cap) follow.
dh2_status upload_tree(Tree& tr) {
  for (int sd = 0; sd < 2; ++sd)
    if (tr.side[sd].pairs.size() > kCodePairMask) return DH2_EUNSUPPORTED;
  if (tr.blocks.size() >= (size_t(1) << 26)) return DH2_EUNSUPPORTED;
  Tree::Dev* D = new (std::nothrow) Tree::Dev();
  if (!D) return DH2_ENOMEM;
  const int32_t nc = tr.nclusters();
  struct Buf {
    const void* src;
    size_t bytes;
    void** dst;
  };
  std::vector<Buf> bufs;
  // keep host arrays alive until the copy
  std::vector<std::vector<int32_t>> i32;
  std::vector<std::vector<int64_t>> i64;
  i32.reserve(64);
  i64.reserve(32);
  auto add32 = [&](std::vector<int32_t>&& v, int32_t** dst) {
    i32.push_back(std::move(v));
    bufs.push_back({i32.back().data(), bytes_of(i32.back()), (void**)dst});
  };
  auto add64 = [&](std::vector<int64_t>&& v, int64_t** dst) {
    i64.push_back(std::move(v));
    bufs.push_back({i64.back().data(), bytes_of(i64.back()), (void**)dst});
  };
  add32(std::vector<int32_t>(tr.start), &D->cstart);
  add32(std::vector<int32_t>(tr.size), &D->csize);
  add32(std::vector<int32_t>(tr.level), &D->clevel);
  D->max_leaf = tr.max_leaf;

  for (int sd = 0; sd < 2; ++sd) {
    Side& S = tr.side[sd];
    const int64_t np = (int64_t)S.pairs.size();
    D->npairs[sd] = np;
    std::vector<int32_t> cl(np), lf(np), st(np), mm(np), nco(np), son(2 * np, -1), soff(2 * np, 0), lv(np),
        kc(np), rc(np), io(np);
    std::vector<int64_t> cmo(np), ro(np), qo(np), xo(np, 0), ho(np), go(np, 0);
    int64_t R_e = 0, Q_e = 0, X_e = 0, h_e = 0;
    for (int64_t p = 0; p < np; ++p) {  // sons before fathers (level descending)
      const Pair& P = S.pairs[p];
      cl[p] = P.cluster;
      lf[p] = P.leaf;
      st[p] = tr.start[P.cluster];
      mm[p] = tr.size[P.cluster];
      nco[p] = (int32_t)P.ncols;
      lv[p] = P.level;
      io[p] = (int32_t)p;
      cmo[p] = S.leaf_colmap_off[p];
      if (P.leaf) {
        rc[p] = tr.size[P.cluster];
        kc[p] = (int32_t)std::min<int64_t>(rc[p], P.ncols);
        const int64_t mpd = (rc[p] + 7) & ~7;  // Gram matrix: mp x mp
        go[p] = D->gram_elems;
        D->gram_elems += mpd * mpd;
      } else {
        for (int j = 0; j < 2; ++j) {
          son[2 * p + j] = (int32_t)P.son_pair[j];
          soff[2 * p + j] = (int32_t)P.son_off[j];
        }
        rc[p] = std::min(kc[P.son_pair[0]] + kc[P.son_pair[1]], kPmaxF32);
        kc[p] = (int32_t)std::min<int64_t>(rc[p], P.ncols);
        xo[p] = X_e;
        X_e += (int64_t)tr.size[P.cluster] * kc[p];
      }
      ro[p] = R_e;
      R_e += (int64_t)kc[p] * P.ncols;
      qo[p] = Q_e;
      Q_e += (int64_t)rc[p] * kc[p];
      ho[p] = h_e;
      h_e += kc[p];
    }
    D->R_elems[sd] = R_e;
    D->Q_elems[sd] = Q_e;
    D->X_elems[sd] = X_e;
    D->h_elems[sd] = h_e;
    D->kcap_h[sd] = kc;
    D->rowcap_h[sd] = rc;
    D->Qoff_h[sd] = qo;
    D->nleaf[sd] = (int64_t)S.leaf_pairs.size();
    std::vector<int32_t> ll(S.leaf_pairs.begin(), S.leaf_pairs.end());
    // level ranges
    D->lvl_begin[sd].assign(tr.depth + 1, 0);
    D->lvl_nl_begin[sd].assign(tr.depth + 1, 0);
    D->lvl_end[sd].assign(tr.depth + 1, 0);
    for (int l = 0; l <= tr.depth; ++l) {
      int64_t b = -1, nb = -1, e = -1;
      for (int64_t p = 0; p < np; ++p)
        if (S.pairs[p].level == l) {
          if (b < 0) b = p;
          if (!S.pairs[p].leaf && nb < 0) nb = p;
          e = p + 1;
        }
      if (b < 0) b = e = nb = 0;
      if (nb < 0) nb = e;
      D->lvl_begin[sd][l] = b;
      D->lvl_nl_begin[sd][l] = nb;
      D->lvl_end[sd][l] = e;
    }
    add32(std::move(cl), &D->cluster[sd]);
    add32(std::move(lf), &D->leaf[sd]);
    add32(std::move(st), &D->start[sd]);
    add32(std::move(mm), &D->m[sd]);
    add32(std::move(nco), &D->ncols[sd]);
    add32(std::move(son), &D->son[sd]);
    add32(std::move(soff), &D->sonoff[sd]);
    add32(std::move(lv), &D->level[sd]);
    add32(std::vector<int32_t>(D->kcap_h[sd]), &D->kcap[sd]);
    add32(std::vector<int32_t>(D->rowcap_h[sd]), &D->rowcap[sd]);
    add32(std::move(io), &D->iota[sd]);
    add32(std::move(ll), &D->leaf_list[sd]);
    add64(std::move(cmo), &D->cmoff[sd]);
    add64(std::move(ro), &D->Roff[sd]);
    add64(std::move(qo), &D->Qoff[sd]);
    add64(std::move(xo), &D->Xoff[sd]);
    add64(std::move(ho), &D->hoff[sd]);
    add64(std::move(go), &D->gram_off[sd]);
    // column maps: allocated here, expanded from the segments after the upload
    bufs.push_back({nullptr, 4 * (size_t)S.nleafcols, (void**)&D->gcol[sd]});
    bufs.push_back({nullptr, 4 * (size_t)S.nleafcols, (void**)&D->gblk[sd]});
    add64(std::vector<int64_t>(S.seg_dst), &D->seg_dst[sd]);
    add32(std::vector<int32_t>(S.seg_col0), &D->seg_col0[sd]);
    add32(std::vector<int32_t>(S.seg_w), &D->seg_w[sd]);
    add32(std::vector<int32_t>(S.seg_blk), &D->seg_blk[sd]);
    add64(std::vector<int64_t>(S.seg_begin), &D->seg_begin[sd]);
  }
  // blocks
  const int64_t nb = (int64_t)tr.blocks.size();
  std::vector<int32_t> bt(nb), bs(nb), ba(nb), bpr(nb), bpc(nb), bo(nb), adm, inadm;
  std::vector<int64_t> noff(nb, 0), soffs(nb, 0), mxoff(nb, -1);
  int64_t S_e = 0, N_e = 0, MX_e = 0;
  for (int64_t b = 0; b < nb; ++b) {
    const Block& B = tr.blocks[b];
    bt[b] = B.t;
    bs[b] = B.s;
    ba[b] = B.adm;
    bpr[b] = (int32_t)tr.side[0].block_pair[b];
    bpc[b] = (int32_t)tr.side[1].block_pair[b];
    bo[b] = (int32_t)tr.side[0].block_off[b];
    if (B.adm) {
      adm.push_back((int32_t)b);
      soffs[b] = S_e;
      S_e += (int64_t)D->kcap_h[0][bpr[b]] * D->kcap_h[1][bpc[b]];
      mxoff[b] = MX_e;  // mixed modes: largest |re|, |im| of each row, then of each column
      MX_e += (int64_t)tr.size[B.t] + tr.size[B.s];
    } else {
      inadm.push_back((int32_t)b);
      noff[b] = N_e;
      N_e += (int64_t)tr.size[B.t] * tr.size[B.s];
    }
  }
  D->S_elems = S_e;
  D->near_elems = N_e;
  D->bmax_elems = MX_e;
  D->nadm = (int64_t)adm.size();
  D->ninadm = (int64_t)inadm.size();
  D->Soff_h = soffs;
  add32(std::move(bt), &D->bt);
  add32(std::move(bs), &D->bs);
  add32(std::move(ba), &D->badm);
  add32(std::move(bpr), &D->bpair[0]);
  add32(std::move(bpc), &D->bpair[1]);
  add32(std::move(bo), &D->boff_row);
  add64(std::move(noff), &D->near_off);
  add64(std::move(soffs), &D->Soff);
  add64(std::move(mxoff), &D->bmax_off);
  {
    std::vector<int64_t> pcs, pbeg;
    for (int32_t b : adm) {
      pbeg.push_back((int64_t)pcs.size());
      const Block& B = tr.blocks[b];
      const int64_t nsl = ((int64_t)tr.size[B.t] + 31) / 32, ngr = ((int64_t)tr.size[B.s] + kNormCols - 1) / kNormCols;
      for (int64_t sl = 0; sl < nsl; ++sl)
        for (int64_t g = 0; g < ngr; ++g) pcs.push_back((int64_t)(((uint64_t)b << 32) | ((uint64_t)sl << 16) | (uint64_t)g));
    }
    pbeg.push_back((int64_t)pcs.size());
    D->nnorm_pieces = (int64_t)pcs.size();
    add64(std::move(pcs), &D->norm_pieces);
    add64(std::move(pbeg), &D->norm_pbegin);
  }
  add32(std::move(adm), &D->adm_list);
  add32(std::move(inadm), &D->inadm_list);
  // matvec lists: own blocks and father pairs per pair, row side (the
  // product) and column side (the adjoint product)
  for (int sd = 0; sd < 2; ++sd) {
    Side& S = tr.side[sd];
    const int64_t np = (int64_t)S.pairs.size();
    std::vector<int64_t> optr(np + 1, 0), pptr(np + 1, 0);
    std::vector<int32_t> oblk, ppair, pson;
    for (int64_t p = 0; p < np; ++p) {
      for (int32_t b : S.pairs[p].own) oblk.push_back(b);
      optr[p + 1] = (int64_t)oblk.size();
      for (auto& seg : S.pairs[p].parents) {
        const int64_t fp = seg.first;
        ppair.push_back((int32_t)fp);
        pson.push_back(S.pairs[fp].son_pair[0] == p ? 0 : 1);
      }
      pptr[p + 1] = (int64_t)ppair.size();
    }
    add64(std::move(optr), sd == 0 ? &D->own_ptr : &D->own_ptr_c);
    add64(std::move(pptr), sd == 0 ? &D->par_ptr : &D->par_ptr_c);
    add32(std::move(oblk), sd == 0 ? &D->own_blk : &D->own_blk_c);
    add32(std::move(ppair), sd == 0 ? &D->par_pair : &D->par_pair_c);
    add32(std::move(pson), sd == 0 ? &D->par_son : &D->par_son_c);
  }
  // launch codes: all leaf pairs of both sides by size class, costliest first
  // within a class; then non-leaf pairs per level
  {
    struct LC {
      int cls;
      double cost;
      int32_t code;
      int m;
    };
    std::vector<LC> lc;
    for (int sd = 0; sd < 2; ++sd)
      for (int64_t p : tr.side[sd].leaf_pairs) {
        const int m = tr.size[tr.side[sd].pairs[p].cluster];
        lc.push_back({leaf_class(m), (double)m * m * (double)tr.side[sd].pairs[p].ncols,
                      (int32_t)((sd << kCodeSideShift) | (int32_t)p), m});
      }
    std::stable_sort(lc.begin(), lc.end(), [](const LC& a, const LC& b) {
      return a.cls != b.cls ? a.cls < b.cls : a.cost > b.cost;
    });
    std::vector<int32_t> codes;
    for (size_t i = 0; i < lc.size(); ++i) {
      codes.push_back(lc[i].code);
      D->leaf_class_maxm[lc[i].cls] = std::max(D->leaf_class_maxm[lc[i].cls], (int32_t)lc[i].m);
      D->leaf_class_begin[lc[i].cls + 1] = (int64_t)i + 1;
    }
    for (int c = 1; c <= kLeafClasses; ++c)
      D->leaf_class_begin[c] = std::max(D->leaf_class_begin[c], D->leaf_class_begin[c - 1]);
    D->nleaf_codes = (int64_t)codes.size();
    D->nl_code_begin.assign(tr.depth + 1, 0);
    D->nl_code_count.assign(tr.depth + 1, 0);
    D->nl_rowcap_max.assign(tr.depth + 1, 0);
    for (int l = tr.depth; l >= 0; --l) {
      D->nl_code_begin[l] = (int64_t)codes.size();
      for (int sd = 0; sd < 2; ++sd)
        for (int64_t p : tr.side[sd].nonleaf_by_level[l]) {
          codes.push_back((int32_t)((sd << kCodeSideShift) | (int32_t)p));
          D->nl_rowcap_max[l] = std::max(D->nl_rowcap_max[l], D->rowcap_h[sd][p]);
        }
      D->nl_code_count[l] = (int64_t)codes.size() - D->nl_code_begin[l];
    }
    // R tiles of 32 columns per pair, in the order of the codes
    std::vector<int64_t> tiles;
    auto add_tiles = [&](int32_t code) {
      const int sd = (code >> kCodeSideShift) & 1;
      const int64_t p = code & (int32_t)kCodePairMask;
      const int64_t nc = tr.side[sd].pairs[p].ncols;
      for (int64_t j0 = 0; j0 < nc; j0 += kRTile) tiles.push_back((int64_t)(((uint64_t)(uint32_t)code << 32) | (uint64_t)j0));
    };
    for (int c = 0; c < kLeafClasses; ++c) {
      D->leaf_tile_class_begin[c] = (int64_t)tiles.size();
      for (int64_t i = D->leaf_class_begin[c]; i < D->leaf_class_begin[c + 1]; ++i) add_tiles(codes[i]);
    }
    D->nleaf_tiles = (int64_t)tiles.size();
    D->leaf_tile_class_begin[kLeafClasses] = D->nleaf_tiles;
    D->nl_tile_begin.assign(tr.depth + 1, 0);
    D->nl_tile_count.assign(tr.depth + 1, 0);
    for (int l = tr.depth; l >= 0; --l) {
      D->nl_tile_begin[l] = (int64_t)tiles.size();
      for (int64_t i = 0; i < D->nl_code_count[l]; ++i) add_tiles(codes[D->nl_code_begin[l] + i]);
      D->nl_tile_count[l] = (int64_t)tiles.size() - D->nl_tile_begin[l];
    }
    add32(std::move(codes), (int32_t**)&D->codes);
    add64(std::move(tiles), &D->tiles);
  }
  size_t total = 0;
  for (auto& b : bufs) total += align256(std::max<size_t>(b.bytes, 4));
  if (dev_malloc(&D->arena, total) != cudaSuccess) {
    cudaGetLastError();
    delete D;
    return DH2_ENOMEM;
  }
  size_t off = 0;
  for (auto& b : bufs) {
    *b.dst = (char*)D->arena + off;
    if (b.bytes && b.src && cudaMemcpy(*b.dst, b.src, b.bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(D->arena);
      delete D;
      return DH2_ECUDA;
    }
    off += align256(std::max<size_t>(b.bytes, 4));
  }
  for (int sd = 0; sd < 2; ++sd)
    launch_colmap_expand(D->seg_dst[sd], D->seg_col0[sd], D->seg_w[sd], D->seg_blk[sd],
                         (int64_t)tr.side[sd].seg_dst.size(), D->gcol[sd], D->gblk[sd], nullptr);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    cudaFree(D->arena);
    delete D;
    return DH2_ECUDA;
  }
  tr.dev = D;
  return DH2_OK;
}

dh2_status ensure_device(Tree& tr, int dev) {
  if (tr.dev) return tr.dev_id == dev ? DH2_OK : DH2_EINVAL;
  const dh2_status s = upload_tree(tr);
  if (s == DH2_OK) tr.dev_id = dev;
  return s;
}

void set_pool_threshold(int dev) {
  static int done[64] = {0};
  if (dev < 0 || dev >= 64 || done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  done[dev] = 1;
}

template <typename T>
SideView<T> side_view(const Tree& tr, const dh2_matrix* M, int sd) {
  const Tree::Dev* D = tr.dev;
  SideView<T> v;
  v.cluster = D->cluster[sd];
  v.leaf = D->leaf[sd];
  v.son = D->son[sd];
  v.rowcap = D->rowcap[sd];
  v.kcap = D->kcap[sd];
  v.Roff = D->Roff[sd];
  v.Qoff = D->Qoff[sd];
  v.Xoff = D->Xoff[sd];
  v.cstart = D->cstart;
  v.csize = D->csize;
  v.rank = M->rank[sd];
  v.side = sd;
  v.R = (C2<T>*)M->R[sd];
  v.Q = (C2<T>*)M->Q[sd];
  v.X = (C2<T>*)M->X[sd];
  return v;
}

int even_up(int x) { return x + (x & 1); }

#ifdef DH2_CHECK
#define DH2_PHASE_SYNC(name)                                                                        \
  do {                                                                                              \
    const cudaError_t e_ = cudaStreamSynchronize(st);                                               \
    if (e_ != cudaSuccess) {                                                                        \
      std::fprintf(stderr, "dh2: launch '%s' failed: %s\n", name, cudaGetErrorString(e_));           \
      return DH2_ECUDA;                                                                             \
    }                                                                                               \
  } while (0)
#else
#define DH2_PHASE_SYNC(name) \
  do {                       \
  } while (0)
#endif

template <typename T>
void fill_args(dh2_matrix* M, const dh2_compress_params& cp, PairArgs<T>& pa, NormsArgs<T>& na) {
  Tree& tr = M->tree->tr;
  Tree::Dev* D = tr.dev;
  na.G = (const C2<T>*)M->G;
  na.ld = M->ld;
  na.bt = D->bt;
  na.bs = D->bs;
  na.badm = D->badm;
  na.cstart = D->cstart;
  na.csize = D->csize;
  na.clevel = D->clevel;
  na.zpow = M->zpow;
  na.invw = M->invw;
  na.near = (C2<T>*)M->near;
  na.near_off = D->near_off;
  na.copy = M->nearfield_copy;
  na.pts = M->pts;
  na.nrm = M->nrm;
  na.kappa = M->kappa;
  na.diag = M->diag;
  na.gen = M->gen;
  na.bmax = nullptr;  // set by run_compress in the mixed modes
  na.bmax_off = D->bmax_off;
  na.bnorm2 = M->bnorm2;
  for (int sd = 0; sd < 2; ++sd) {
    pa.start[sd] = D->start[sd];
    pa.m[sd] = D->m[sd];
    pa.ncols[sd] = D->ncols[sd];
    pa.cmoff[sd] = D->cmoff[sd];
    pa.gcol[sd] = D->gcol[sd];
    pa.gblk[sd] = D->gblk[sd];
    pa.colw[sd] = (const T*)M->colw[sd];
    pa.son[sd] = D->son[sd];
    pa.sonoff[sd] = D->sonoff[sd];
    pa.level[sd] = D->level[sd];
    pa.kcap[sd] = D->kcap[sd];
    pa.rowcap[sd] = D->rowcap[sd];
    pa.Roff[sd] = D->Roff[sd];
    pa.Qoff[sd] = D->Qoff[sd];
    pa.R[sd] = (C2<T>*)M->R[sd];
    pa.Q[sd] = (C2<T>*)M->Q[sd];
    pa.sig[sd] = M->sig[sd];
    pa.rank[sd] = M->rank[sd];
  }
  pa.G = (const C2<T>*)M->G;
  pa.ld = M->ld;
  pa.invw = M->invw;
  pa.eps2 = M->eps2;
  pa.H = nullptr;  // set by run_compress in the mixed modes
  pa.L4 = nullptr;
  for (int sd = 0; sd < 2; ++sd) {
    pa.hoff[sd] = D->gram_off[sd];
    pa.rank_ovr[sd] = nullptr;  // set by run_compress when ranks are given
  }
  pa.max_sweeps = cp.max_sweeps > 0 ? cp.max_sweeps : 30;
  const TuneTable tt = tune_current();
  for (int c = 0; c < 5; ++c) pa.jacobi_tpp[c] = tt.jacobi_tpp[c];
  pa.seg_off[0] = pa.seg_off[1] = nullptr;  // set by run_compress when wide pairs are split
  pa.seg_buf = nullptr;
  pa.seg_cols = 0;
  pa.status = M->status;
  pa.pts = M->pts;
  pa.nrm = M->nrm;
  pa.kappa = M->kappa;
  pa.diag = M->diag;
  pa.gen = M->gen;
}

// Panel plan of a tree for a host-resident G (see PanelPlan).
#ifndef DH2_HOST_PANELS
#define DH2_HOST_PANELS 4  // column panels of a host-resident G
#endif

void make_panel_plan(const Tree& tr, PanelPlan& pp) {
  // few panels: each panel's leaf lists must still fill the GPU (a launch of
  // a few hundred pairs leaves most SMs idle in its last wave)
  constexpr int kPanels = DH2_HOST_PANELS;
  const int64_t n = tr.n;
  int32_t lmin = INT32_MAX;
  for (const Block& B : tr.blocks)
    if (B.adm) lmin = std::min(lmin, tr.level[B.t]);
  // atoms: clusters of level lmin and leaves above it, in increasing start
  // order (pre-order with the first son first)
  std::vector<int32_t> atoms;
  if (lmin == INT32_MAX) {
    atoms.push_back(0);
  } else {
    std::vector<int32_t> stack{0};
    while (!stack.empty()) {
      const int32_t c = stack.back();
      stack.pop_back();
      if (tr.level[c] >= lmin || tr.is_leaf(c)) {
        atoms.push_back(c);
      } else {
        stack.push_back(tr.son1[c]);
        stack.push_back(tr.son0[c]);
      }
    }
  }
  const int64_t target = (n + kPanels - 1) / kPanels;
  auto assign = [&](bool one_panel) -> bool {
    pp.col.assign(1, 0);
    if (!one_panel) {
      int64_t acc = 0;
      for (int32_t a : atoms) {
        acc += tr.size[a];
        const int64_t end = (int64_t)tr.start[a] + tr.size[a];
        if (acc >= target && end < n) {
          pp.col.push_back(end);
          acc = 0;
        }
      }
    }
    pp.col.push_back(n);
    const int K = (int)pp.col.size() - 1;
    auto panel_of = [&](int64_t j) {
      return (int)(std::upper_bound(pp.col.begin(), pp.col.end(), j) - pp.col.begin()) - 1;
    };
    pp.blk.assign(K, {});
    pp.blk_rest.clear();
    for (size_t b = 0; b < tr.blocks.size(); ++b) {
      const Block& B = tr.blocks[b];
      const int k0 = panel_of(tr.start[B.s]), k1 = panel_of((int64_t)tr.start[B.s] + tr.size[B.s] - 1);
      if (k0 == k1) pp.blk[k0].push_back((uint32_t)b);
      else if (B.adm) return false;  // not expected by construction
      else pp.blk_rest.push_back((uint32_t)b);
    }
    struct E {
      double cost;
      uint32_t code;
    };
    std::vector<std::vector<std::vector<E>>> cl(K, std::vector<std::vector<E>>(kLeafClasses));
    std::vector<std::vector<std::vector<E>>> rl(K, std::vector<std::vector<E>>(kLeafClasses));
    // row basis: the last panel a pair reads (its own blocks' column clusters
    // and, recursively, its father pairs')
    const Side& S0 = tr.side[kSideRow];
    std::vector<int> lastp(S0.pairs.size(), -1);
    std::function<int(int64_t)> last = [&](int64_t p) -> int {
      if (lastp[p] >= 0) return lastp[p];
      int m = 0;
      for (int32_t b : S0.pairs[p].own) {
        const Block& B = tr.blocks[b];
        m = std::max(m, panel_of((int64_t)tr.start[B.s] + tr.size[B.s] - 1));
      }
      for (const auto& seg : S0.pairs[p].parents) m = std::max(m, last(seg.first));
      return lastp[p] = m;
    };
    for (int sd = 0; sd < 2; ++sd)
      for (int64_t p : tr.side[sd].leaf_pairs) {
        const int32_t c = tr.side[sd].pairs[p].cluster;
        const int m = tr.size[c];
        const E e{(double)m * m * (double)tr.side[sd].pairs[p].ncols,
                  (uint32_t)((sd << kCodeSideShift) | (int32_t)p)};
        if (sd == kSideCol) cl[panel_of(tr.start[c])][leaf_class(m)].push_back(e);
        else rl[last(p)][leaf_class(m)].push_back(e);
      }
    auto codes = [](std::vector<E>& v) {
      std::stable_sort(v.begin(), v.end(), [](const E& a, const E& b) { return a.cost > b.cost; });
      std::vector<uint32_t> out;
      out.reserve(v.size());
      for (const E& e : v) out.push_back(e.code);
      return out;
    };
    pp.col_leaf.assign(K, std::vector<std::vector<uint32_t>>(kLeafClasses));
    pp.row_leaf.assign(K, std::vector<std::vector<uint32_t>>(kLeafClasses));
    for (int k = 0; k < K; ++k)
      for (int c = 0; c < kLeafClasses; ++c) {
        pp.col_leaf[k][c] = codes(cl[k][c]);
        pp.row_leaf[k][c] = codes(rl[k][c]);
      }
    return true;
  };
  if (!assign(false)) assign(true);
}

// G in host memory (dh2_compress_host): copied panel by panel into the
// staging buffer (the matrix's G, ld = n).
struct HostStage {
  const void* G_host;
  int64_t ld;   // leading dimension of G_host, elements
  size_t elem;  // bytes per element
  const PanelPlan* plan;
};

// A compression captured into a CUDA graph (dh2_plan): the graph, the scratch
// it works in, and a function that writes new matrix pointers into the
// device copies of the kernels' argument blocks before a replay.
struct PlanState {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  void* scratch = nullptr;
  bool ok_launch = true;
  std::function<cudaError_t(const void* const* G, cudaStream_t st)> set_inputs;
};

// The compression of one or several independent problems: each phase is one
// launch over every problem (block norms, leaf factors, one launch per level
// for the non-leaf steps), then expansion and projection per problem.
template <typename T>
dh2_status run_compress(std::vector<dh2_matrix*>& Ms, const dh2_compress_params& cp, cudaStream_t st,
                        const HostStage* hs = nullptr, PlanState* plan = nullptr) {
#if defined(DH2_CHECK) || defined(DH2_PROFILE)
  if (plan) return DH2_EUNSUPPORTED;  // these builds synchronise inside the schedule
#endif
  if (plan && hs) return DH2_EINVAL;
  bool any_gen = false;  // entries generated in the kernels (matrix-free mode)
  for (const dh2_matrix* M : Ms) any_gen = any_gen || M->gen != 0;
  const int nprob = (int)Ms.size();
  const int pmax = sizeof(T) == 4 ? kPmaxF32 : kPmaxF64;
  std::vector<PairArgs<T>> pas(nprob);
  std::vector<NormsArgs<T>> nas(nprob);
  for (int i = 0; i < nprob; ++i) fill_args<T>(Ms[i], cp, pas[i], nas[i]);
  // launch codes: cached in the tree for one problem, merged for a batch
  std::vector<uint32_t> leaf_codes, norm_codes;
  std::vector<std::vector<uint32_t>> nl_codes;
  int maxdepth = 0, P_leaf = 2;
  std::vector<int> P_level;
  for (dh2_matrix* M : Ms) maxdepth = std::max(maxdepth, M->tree->tr.depth);
  nl_codes.resize(maxdepth + 1);
  P_level.assign(maxdepth + 1, 2);
  for (int i = 0; i < nprob; ++i) {
    const Tree::Dev* D = Ms[i]->tree->tr.dev;
    P_leaf = std::max(P_leaf, even_up(std::max(2, D->max_leaf)));
    for (int l = 0; l <= Ms[i]->tree->tr.depth; ++l)
      if (D->nl_code_count[l]) P_level[l] = std::max(P_level[l], even_up(std::min(pmax, D->nl_rowcap_max[l])));
  }
  const uint32_t* d_leaf = nullptr;
  const uint32_t* d_norm = nullptr;
  std::vector<const uint32_t*> d_nl(maxdepth + 1, nullptr);
  std::vector<int64_t> n_nl(maxdepth + 1, 0);
  int64_t n_leaf = 0, n_norm = 0, n_norm_adm = 0;
  const uint32_t* d_norm_adm = nullptr;   // the admissible blocks' codes
  const uint32_t* d_norm_near = nullptr;  // the nearfield blocks' codes
  const uint64_t* d_pieces = nullptr;     // the admissible blocks' norms pass in pieces
  const int64_t* d_pbegin = nullptr;      // per admissible code its first piece
  int64_t n_pieces = 0;
  std::vector<uint64_t> pieces;
  std::vector<int64_t> pbegin;
  // R tiles (code << 32 | first column) in the order of the codes
  const uint64_t* d_ltiles = nullptr;
  std::vector<const uint64_t*> d_nltiles(maxdepth + 1, nullptr);
  std::vector<int64_t> n_nltiles(maxdepth + 1, 0);
  int64_t n_ltiles = 0;
  std::vector<uint64_t> leaf_tiles;
  // leaf launches per size class: code ranges and largest row count
  int64_t cls_begin[kLeafClasses + 1] = {};
  int cls_maxm[kLeafClasses] = {};
  int64_t tile_cls_begin[kLeafClasses + 1] = {};
  std::vector<std::vector<uint64_t>> nl_tiles(maxdepth + 1);
  size_t args_bytes = align256(sizeof(PairArgs<T>) * nprob) + align256(sizeof(NormsArgs<T>) * nprob);
  size_t codes_bytes = 0;
  if (nprob > 1) {
    struct LC {
      int cls;
      double cost;
      uint32_t code;
      int m;
    };
    std::vector<LC> lc;
    for (int i = 0; i < nprob; ++i) {
      const Tree& tr = Ms[i]->tree->tr;
      for (int sd = 0; sd < 2; ++sd)
        for (int64_t p : tr.side[sd].leaf_pairs) {
          const int m = tr.size[tr.side[sd].pairs[p].cluster];
          lc.push_back({leaf_class(m), (double)m * m * (double)tr.side[sd].pairs[p].ncols,
                        ((uint32_t)i << kCodeProbShift) | ((uint32_t)sd << kCodeSideShift) | (uint32_t)p, m});
        }
      for (int l = tr.depth; l >= 0; --l)
        for (int sd = 0; sd < 2; ++sd)
          for (int64_t p : tr.side[sd].nonleaf_by_level[l])
            nl_codes[l].push_back(((uint32_t)i << kCodeProbShift) | ((uint32_t)sd << kCodeSideShift) | (uint32_t)p);
      for (size_t b = 0; b < tr.blocks.size(); ++b)
        if (tr.blocks[b].adm) norm_codes.push_back(((uint32_t)i << 26) | (uint32_t)b);
    }
    n_norm_adm = (int64_t)norm_codes.size();  // admissible blocks first, then the nearfield blocks
    for (int i = 0; i < nprob; ++i) {
      const Tree& tr = Ms[i]->tree->tr;
      for (size_t b = 0; b < tr.blocks.size(); ++b)
        if (!tr.blocks[b].adm) norm_codes.push_back(((uint32_t)i << 26) | (uint32_t)b);
    }
    for (int64_t q = 0; q < n_norm_adm; ++q) {
      pbegin.push_back((int64_t)pieces.size());
      const uint32_t code = norm_codes[q];
      const Tree& tr = Ms[code >> 26]->tree->tr;
      const Block& B = tr.blocks[code & ((1u << 26) - 1u)];
      const uint64_t nsl = ((uint64_t)tr.size[B.t] + 31) / 32, ngr = ((uint64_t)tr.size[B.s] + kNormCols - 1) / kNormCols;
      for (uint64_t sl = 0; sl < nsl; ++sl)
        for (uint64_t g = 0; g < ngr; ++g) pieces.push_back(((uint64_t)code << 32) | (sl << 16) | g);
    }
    pbegin.push_back((int64_t)pieces.size());
    std::stable_sort(lc.begin(), lc.end(), [](const LC& a, const LC& b) {
      return a.cls != b.cls ? a.cls < b.cls : a.cost > b.cost;
    });
    for (size_t i = 0; i < lc.size(); ++i) {
      leaf_codes.push_back(lc[i].code);
      cls_maxm[lc[i].cls] = std::max(cls_maxm[lc[i].cls], lc[i].m);
      cls_begin[lc[i].cls + 1] = (int64_t)i + 1;
    }
    for (int c = 1; c <= kLeafClasses; ++c) cls_begin[c] = std::max(cls_begin[c], cls_begin[c - 1]);
    auto tiles_of = [&](const std::vector<uint32_t>& codes, std::vector<uint64_t>& out) {
      for (uint32_t c : codes) {
        const Tree& tr = Ms[c >> kCodeProbShift]->tree->tr;
        const int64_t nc = tr.side[(c >> kCodeSideShift) & 1u].pairs[c & kCodePairMask].ncols;
        for (int64_t j0 = 0; j0 < nc; j0 += kRTile) out.push_back(((uint64_t)c << 32) | (uint64_t)j0);
      }
    };
    for (int c = 0; c < kLeafClasses; ++c) {
      tile_cls_begin[c] = (int64_t)leaf_tiles.size();
      const std::vector<uint32_t> seg(leaf_codes.begin() + cls_begin[c], leaf_codes.begin() + cls_begin[c + 1]);
      tiles_of(seg, leaf_tiles);
    }
    tile_cls_begin[kLeafClasses] = (int64_t)leaf_tiles.size();
    for (int l = 0; l <= maxdepth; ++l) tiles_of(nl_codes[l], nl_tiles[l]);
    codes_bytes = align256(4 * leaf_codes.size()) + align256(4 * norm_codes.size()) + align256(8 * leaf_tiles.size()) +
                  align256(8 * pieces.size()) + align256(8 * pbegin.size());
    for (int l = 0; l <= maxdepth; ++l)
      codes_bytes += align256(4 * nl_codes[l].size()) + align256(8 * nl_tiles[l].size());
  }
  // per level: the non-leaf codes sorted into row-count classes
  int64_t nl_max = 0;
  for (int l = 0; l <= maxdepth; ++l) nl_max = std::max(nl_max, (int64_t)nl_codes[l].size());
  for (dh2_matrix* M : Ms)
    for (int l = 0; l <= M->tree->tr.depth; ++l) nl_max = std::max(nl_max, M->tree->tr.dev->nl_code_count[l]);
  const size_t cls_bytes = align256(4 * 4 * (size_t)std::max<int64_t>(nl_max, 1)) + align256(16 * (maxdepth + 1));
  // host-input schedule: the plan's launch lists (blocks per panel, the blocks
  // across panels, column-basis leaves per panel and class, row-basis leaves
  // per class) with their R tiles, uploaded behind the other lists
  struct HList {
    const std::vector<uint32_t>* codes = nullptr;
    std::vector<uint64_t> tiles;
    const uint32_t* d_codes = nullptr;
    const uint64_t* d_tiles = nullptr;
  };
  std::vector<HList> hl;
  size_t host_bytes = 0;
  int hK = 0;
  if (hs) {
    const PanelPlan& pl = *hs->plan;
    const Tree& tr = Ms[0]->tree->tr;
    hK = (int)pl.col.size() - 1;
    // lists: blocks per panel, blocks across panels, then per panel the
    // column-basis and the row-basis leaves per class
    hl.resize((size_t)hK + 1 + (size_t)2 * hK * kLeafClasses);
    for (int k = 0; k < hK; ++k) hl[k].codes = &pl.blk[k];
    hl[hK].codes = &pl.blk_rest;
    for (int k = 0; k < 2 * hK; ++k)
      for (int c = 0; c < kLeafClasses; ++c) {
        HList& L = hl[(size_t)hK + 1 + (size_t)k * kLeafClasses + c];
        L.codes = k < hK ? &pl.col_leaf[k][c] : &pl.row_leaf[k - hK][c];
        for (uint32_t code : *L.codes) {
          const int64_t nc = tr.side[(code >> kCodeSideShift) & 1u].pairs[code & kCodePairMask].ncols;
          for (int64_t j0 = 0; j0 < nc; j0 += kRTile) L.tiles.push_back(((uint64_t)code << 32) | (uint64_t)j0);
        }
      }
    for (const HList& L : hl) host_bytes += align256(4 * L.codes->size()) + align256(8 * L.tiles.size());
  }
  // mixed modes: the leaf Gram matrices (double-float, mp x mp per leaf pair)
  // and the window sums of the pairs with more than one window, per problem
  const bool mixed = mode_mixed(cp.mode);
  std::vector<size_t> gram_h_off(nprob, 0), gram_l_off(nprob, 0), gram_m_off(nprob, 0);
  size_t gram_bytes = 0;
  if (mixed) {
    gram_bytes = align256(sizeof(GramArgs) * nprob);
    for (int i = 0; i < nprob; ++i) {
      const Tree::Dev* D = Ms[i]->tree->tr.dev;
      gram_h_off[i] = gram_bytes;
      if (!Ms[i]->gram) gram_bytes += align256(sizeof(float4) * (size_t)D->gram_elems);  // else kept by the matrix
      gram_l_off[i] = gram_bytes;  // Cholesky factors: over H, or beside the kept Gram matrices
      if (Ms[i]->gram) gram_bytes += align256(sizeof(float4) * (size_t)D->gram_elems);
      gram_m_off[i] = gram_bytes;
      gram_bytes += align256(sizeof(float) * (size_t)D->bmax_elems);
    }
  }
  // ranks given instead of the truncation rule (one problem only)
  size_t ovr_bytes = 0;
  if (nprob == 1)
    for (int sd = 0; sd < 2; ++sd)
      if (cp.rank_override[sd]) ovr_bytes += align256(4 * (size_t)Ms[0]->tree->tr.dev->npairs[sd]);
  // the norms pass's partial sums, one per piece
  int64_t n_pieces_all = nprob > 1 ? (int64_t)pieces.size() : Ms[0]->tree->tr.dev->nnorm_pieces;
  const size_t part_bytes = align256(8 * (size_t)std::max<int64_t>(n_pieces_all, 1));
  // non-leaf pairs wider than twice the tuning table's segment width are
  // factored by column segments: per level the segment entries (code << 32 |
  // segment), per problem and side each pair's slot in the segment buffer
  // (p x p per segment, p at most the pair's row capacity)
  const int seg_cols = tune_current().level_seg_cols;
  std::vector<std::vector<uint64_t>> seg_lists(maxdepth + 1);
  std::vector<std::vector<int64_t>> seg_off_h((size_t)nprob * 2);
  int64_t seg_elems = 0;
  if (seg_cols > 0)
    for (int i = 0; i < nprob; ++i) {
      const Tree& tr = Ms[i]->tree->tr;
      const Tree::Dev* D = tr.dev;
      for (int sd = 0; sd < 2; ++sd) {
        std::vector<int64_t>& so = seg_off_h[(size_t)i * 2 + sd];
        so.assign(tr.side[sd].pairs.size(), -1);
        for (int l = tr.depth; l >= 0; --l)
          for (int64_t p : tr.side[sd].nonleaf_by_level[l]) {
            const int64_t nc = tr.side[sd].pairs[p].ncols;
            if (nc <= 2 * (int64_t)seg_cols) continue;
            const int64_t nseg = (nc + seg_cols - 1) / seg_cols, rc = D->rowcap_h[sd][p];
            so[p] = seg_elems;
            seg_elems += nseg * rc * rc;
            const uint32_t code = ((uint32_t)i << kCodeProbShift) | ((uint32_t)sd << kCodeSideShift) | (uint32_t)p;
            for (int64_t s = 0; s < nseg; ++s) seg_lists[l].push_back(((uint64_t)code << 32) | (uint64_t)s);
          }
      }
    }
  size_t seg_bytes = 0;
  if (seg_elems > 0) {
    seg_bytes += align256(sizeof(C2<T>) * (size_t)seg_elems);
    for (const auto& v : seg_off_h) seg_bytes += align256(8 * std::max<size_t>(v.size(), 1));
    for (const auto& v : seg_lists) seg_bytes += 5 * align256(8 * v.size()) + align256(16);  // list, 4 classes, counts
  }
  void* scratch = nullptr;
  if (dev_malloc_async(&scratch, args_bytes + codes_bytes + cls_bytes + host_bytes + gram_bytes + ovr_bytes +
                                     part_bytes + seg_bytes + 256,
                       st) != cudaSuccess) {
    cudaGetLastError();
    return DH2_ENOMEM;
  }
  char* const gram_base = (char*)scratch + args_bytes + codes_bytes + cls_bytes + host_bytes;
  char* const ovr_base = gram_base + gram_bytes;
  double* const d_partial = (double*)(ovr_base + ovr_bytes);
  cudaError_t ce_ovr = cudaSuccess;
  if (ovr_bytes) {
    char* op = ovr_base;
    for (int sd = 0; sd < 2; ++sd)
      if (cp.rank_override[sd]) {
        const int64_t np = Ms[0]->tree->tr.dev->npairs[sd];
        if (ce_ovr == cudaSuccess)
          ce_ovr = cudaMemcpyAsync(op, cp.rank_override[sd], 4 * (size_t)np, cudaMemcpyHostToDevice, st);
        pas[0].rank_ovr[sd] = (const int32_t*)op;
        op += align256(4 * (size_t)np);
      }
  }
  // the segment buffer, slots, lists and class lists
  std::vector<const uint64_t*> d_seg(maxdepth + 1, nullptr);
  std::vector<uint64_t*> d_seg_cls(maxdepth + 1, nullptr);
  std::vector<int*> d_seg_cnt(maxdepth + 1, nullptr);
  if (seg_elems > 0) {
    char* sp2 = (char*)d_partial + part_bytes;
    C2<T>* seg_buf = (C2<T>*)sp2;
    sp2 += align256(sizeof(C2<T>) * (size_t)seg_elems);
    for (int i = 0; i < nprob; ++i) {
      pas[i].seg_buf = seg_buf;
      pas[i].seg_cols = seg_cols;
      for (int sd = 0; sd < 2; ++sd) {
        const std::vector<int64_t>& v = seg_off_h[(size_t)i * 2 + sd];
        if (!v.empty() && ce_ovr == cudaSuccess)
          ce_ovr = cudaMemcpyAsync(sp2, v.data(), 8 * v.size(), cudaMemcpyHostToDevice, st);
        pas[i].seg_off[sd] = v.empty() ? nullptr : (const int64_t*)sp2;
        sp2 += align256(8 * std::max<size_t>(v.size(), 1));
      }
    }
    for (int l = 0; l <= maxdepth; ++l) {
      const std::vector<uint64_t>& v = seg_lists[l];
      if (!v.empty() && ce_ovr == cudaSuccess)
        ce_ovr = cudaMemcpyAsync(sp2, v.data(), 8 * v.size(), cudaMemcpyHostToDevice, st);
      d_seg[l] = (const uint64_t*)sp2;
      sp2 += align256(8 * v.size());
      d_seg_cls[l] = (uint64_t*)sp2;
      sp2 += 4 * align256(8 * v.size());
      d_seg_cnt[l] = (int*)sp2;
      sp2 += align256(16);
    }
  }
  GramArgs* d_ga = (GramArgs*)gram_base;
  std::vector<GramArgs> gas;
  if (mixed) {
    gas.resize(nprob);
    for (int i = 0; i < nprob; ++i) {
      const Tree::Dev* D = Ms[i]->tree->tr.dev;
      const dh2_matrix* M = Ms[i];
      float4* Hbuf = Ms[i]->gram ? (float4*)Ms[i]->gram : (float4*)(gram_base + gram_h_off[i]);
      pas[i].H = Hbuf;
      pas[i].L4 = Ms[i]->gram ? (float4*)(gram_base + gram_l_off[i]) : Hbuf;
      GramArgs& g = gas[i];
      for (int sd = 0; sd < 2; ++sd) {
        g.start[sd] = D->start[sd];
        g.m[sd] = D->m[sd];
        g.ncols[sd] = D->ncols[sd];
        g.cmoff[sd] = D->cmoff[sd];
        g.gcol[sd] = D->gcol[sd];
        g.colw[sd] = (const float*)M->colw[sd];
        g.hoff[sd] = D->gram_off[sd];
        g.seg_begin[sd] = D->seg_begin[sd];
        g.seg_blk[sd] = D->seg_blk[sd];
      }
      g.bt = D->bt;
      g.bs = D->bs;
      g.cstart = D->cstart;
      g.csize = D->csize;
      g.invw = M->invw;
      g.bmax = (const float*)(gram_base + gram_m_off[i]);
      g.bmax_off = D->bmax_off;
      nas[i].bmax = (float*)(gram_base + gram_m_off[i]);
      g.G = (const C2<float>*)M->G;
      g.ld = M->ld;
      g.H = Hbuf;
      g.status = M->status;
      g.spin_limit = (uint32_t)std::min<int64_t>(std::max<int64_t>(cp.spin_limit, 0), (int64_t)UINT32_MAX);
    }
  }
  char* sp = (char*)scratch;
  PairArgs<T>* d_pa = (PairArgs<T>*)sp;
  sp += align256(sizeof(PairArgs<T>) * nprob);
  NormsArgs<T>* d_na = (NormsArgs<T>*)sp;
  sp += align256(sizeof(NormsArgs<T>) * nprob);
  cudaError_t ce = cudaMemcpyAsync(d_pa, pas.data(), sizeof(PairArgs<T>) * nprob, cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess && mixed)
    ce = cudaMemcpyAsync(d_ga, gas.data(), sizeof(GramArgs) * nprob, cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) ce = ce_ovr;
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(d_na, nas.data(), sizeof(NormsArgs<T>) * nprob, cudaMemcpyHostToDevice, st);
  if (nprob > 1) {
    auto up = [&](const std::vector<uint32_t>& v) -> const uint32_t* {
      uint32_t* d = (uint32_t*)sp;
      if (!v.empty() && ce == cudaSuccess) ce = cudaMemcpyAsync(d, v.data(), 4 * v.size(), cudaMemcpyHostToDevice, st);
      sp += align256(4 * v.size());
      return d;
    };
    d_leaf = up(leaf_codes);
    n_leaf = (int64_t)leaf_codes.size();
    d_norm = up(norm_codes);
    n_norm = (int64_t)norm_codes.size();
    d_norm_adm = d_norm;
    d_norm_near = d_norm + n_norm_adm;
    for (int l = 0; l <= maxdepth; ++l) {
      d_nl[l] = up(nl_codes[l]);
      n_nl[l] = (int64_t)nl_codes[l].size();
    }
    auto up64 = [&](const std::vector<uint64_t>& v) -> const uint64_t* {
      uint64_t* d = (uint64_t*)sp;
      if (!v.empty() && ce == cudaSuccess) ce = cudaMemcpyAsync(d, v.data(), 8 * v.size(), cudaMemcpyHostToDevice, st);
      sp += align256(8 * v.size());
      return d;
    };
    d_ltiles = up64(leaf_tiles);
    n_ltiles = (int64_t)leaf_tiles.size();
    d_pieces = up64(pieces);
    n_pieces = (int64_t)pieces.size();
    {
      int64_t* d = (int64_t*)sp;
      if (!pbegin.empty() && ce == cudaSuccess)
        ce = cudaMemcpyAsync(d, pbegin.data(), 8 * pbegin.size(), cudaMemcpyHostToDevice, st);
      sp += align256(8 * pbegin.size());
      d_pbegin = d;
    }
    for (int l = 0; l <= maxdepth; ++l) {
      d_nltiles[l] = up64(nl_tiles[l]);
      n_nltiles[l] = (int64_t)nl_tiles[l].size();
    }
  } else {
    const Tree& tr = Ms[0]->tree->tr;
    const Tree::Dev* D = tr.dev;
    d_leaf = D->codes;
    n_leaf = D->nleaf_codes;
    for (int c = 0; c <= kLeafClasses; ++c) cls_begin[c] = D->leaf_class_begin[c];
    for (int c = 0; c < kLeafClasses; ++c) cls_maxm[c] = D->leaf_class_maxm[c];
    for (int c = 0; c <= kLeafClasses; ++c) tile_cls_begin[c] = D->leaf_tile_class_begin[c];
    d_norm = nullptr;
    n_norm = (int64_t)tr.blocks.size();
    n_norm_adm = D->nadm;
    d_norm_adm = (const uint32_t*)D->adm_list;  // block ids of problem 0: the codes themselves
    d_norm_near = (const uint32_t*)D->inadm_list;
    d_pieces = (const uint64_t*)D->norm_pieces;
    d_pbegin = D->norm_pbegin;
    n_pieces = D->nnorm_pieces;
    for (int l = 0; l <= tr.depth; ++l) {
      d_nl[l] = D->codes + D->nl_code_begin[l];
      n_nl[l] = D->nl_code_count[l];
    }
    d_ltiles = (const uint64_t*)D->tiles;
    n_ltiles = D->nleaf_tiles;
    for (int l = 0; l <= tr.depth; ++l) {
      d_nltiles[l] = (const uint64_t*)D->tiles + D->nl_tile_begin[l];
      n_nltiles[l] = D->nl_tile_count[l];
    }
  }
  if (hs) {
    char* hp = (char*)scratch + args_bytes + codes_bytes + cls_bytes;
    for (HList& L : hl) {
      L.d_codes = (const uint32_t*)hp;
      if (!L.codes->empty() && ce == cudaSuccess)
        ce = cudaMemcpyAsync(hp, L.codes->data(), 4 * L.codes->size(), cudaMemcpyHostToDevice, st);
      hp += align256(4 * L.codes->size());
      L.d_tiles = (const uint64_t*)hp;
      if (!L.tiles.empty() && ce == cudaSuccess)
        ce = cudaMemcpyAsync(hp, L.tiles.data(), 8 * L.tiles.size(), cudaMemcpyHostToDevice, st);
      hp += align256(8 * L.tiles.size());
    }
  }
  cudaEvent_t ev[7] = {};
  for (int i = 0; i < 7 && ce == cudaSuccess && !plan; ++i) ce = cudaEventCreate(&ev[i]);
  auto rec = [&](int i) {  // phase boundaries (not in a captured schedule)
    if (!plan) cudaEventRecord(ev[i], st);
  };
  if (ce != cudaSuccess) {
    cudaGetLastError();
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    cudaFreeAsync(scratch, st);
    return DH2_ECUDA;
  }
#ifdef DH2_CHECK
  {
    // one set of limits for the launch: the largest over the problems
    CheckLimits lim{};
    for (dh2_matrix* M : Ms) {
      const Tree& tr = M->tree->tr;
      const Tree::Dev* D = tr.dev;
      lim.G = std::max<int64_t>(lim.G, M->ld * (tr.n - 1) + tr.n);
      for (int sd = 0; sd < 2; ++sd) {
        lim.R[sd] = std::max(lim.R[sd], D->R_elems[sd]);
        lim.Q[sd] = std::max(lim.Q[sd], D->Q_elems[sd]);
        lim.X[sd] = std::max(lim.X[sd], D->X_elems[sd]);
        lim.npairs[sd] = std::max(lim.npairs[sd], D->npairs[sd]);
        lim.ncol[sd] = std::max(lim.ncol[sd], tr.side[sd].nleafcols);
      }
      lim.S = std::max(lim.S, D->S_elems);
      lim.near = std::max<int64_t>(lim.near, M->nearfield_copy ? D->near_elems : 0);
      lim.nblocks = std::max<int64_t>(lim.nblocks, (int64_t)tr.blocks.size());
    }
    lim.seg = seg_elems;
    cudaStreamSynchronize(st);
    check_set_limits_pair(lim);
    check_set_limits_ops(lim);
  }
#endif
  if (plan) {
    // everything from here to the projection becomes the graph; each replay
    // starts by clearing the status words
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      cudaFreeAsync(scratch, st);
      return DH2_ECUDA;
    }
    for (dh2_matrix* M : Ms) cudaMemsetAsync(M->status, 0, sizeof(uint32_t), st);
  }
  rec(0);
  bool ok_launch = true;  // false once a launch needed more shared memory than the device has
  int nlaunch = 0;  // kernels launched by this compression (counted where they are issued)
  int32_t kcl[DH2_KC_COUNT] = {};  // the same, by kernel class
  auto counted = [&](int kc, bool launched) {
    if (!launched) return;
    ++nlaunch;
    ++kcl[kc];
  };
  auto colw_side = [&](int sd) {
    for (dh2_matrix* M : Ms) {
      launch_colw<T>(M->tree->tr.dev->gblk[sd], M->invw, (T*)M->colw[sd], M->tree->tr.side[sd].nleafcols, st);
      counted(DH2_KC_COLW, M->tree->tr.side[sd].nleafcols > 0);
    }
  };
  // leaf factors and R of one launch list per size class
  // leaf factorisations of one size class: the streamed LQ, or in the mixed
  // modes the tensor-core Gram matrices and their pivoted Cholesky
  // events around the Gram and factor launches of each class (mixed modes,
  // device input): the leaf phase split into its two kernels
  cudaEvent_t kev[4 * kLeafClasses] = {};
  bool kev_ok = false;
  auto leaf_factor = [&](const uint32_t* codes, int n, int c, bool timed) {
    if (n <= 0) return;
    const int P = even_up(std::max(2, cls_maxm[c]));
    if constexpr (sizeof(T) == 4) {
      if (mixed) {
        if (timed) cudaEventRecord(kev[4 * c], st);
        ok_launch &= launch_gram(d_ga, codes, n, cls_maxm[c], st);  // row scales, then the Gram matrices
        counted(DH2_KC_GRAM_SCALES, true);
        counted(DH2_KC_LEAF_GRAM + c, true);
        if (timed) cudaEventRecord(kev[4 * c + 1], st);
        // pivoted Cholesky, then Jacobi, rank and Q
        if (timed) cudaEventRecord(kev[4 * c + 2], st);
        ok_launch &= launch_pair_kernel_gram(reinterpret_cast<const PairArgs<float>*>(d_pa), codes, n, P, st);
        counted(DH2_KC_LEAF_FACTOR + c, true);
        counted(DH2_KC_LEAF_JACOBI + c, true);
        if (timed) cudaEventRecord(kev[4 * c + 3], st);
        return;
      }
    }
    ok_launch &= launch_pair_kernel<T>(d_pa, codes, n, P, false, st);
    counted(DH2_KC_LEAF_FACTOR + c, true);
  };
  auto leaf_lists = [&](const HList* L) {
    for (int c = 0; c < kLeafClasses; ++c) leaf_factor(L[c].d_codes, (int)L[c].codes->size(), c, false);
  };
  auto leaf_rq = [&](const HList* L) {
    for (int c = 0; c < kLeafClasses; ++c)
      if (!L[c].tiles.empty()) {
        ok_launch &= launch_rq_kernel<T>(d_pa, L[c].d_tiles, (int)L[c].tiles.size(), even_up(std::max(2, cls_maxm[c])), false,
                            any_gen, st);
        counted(DH2_KC_LEAF_R + c, true);
      }
  };
  if (hs) {
    // Host-resident G: copied panel by panel on a second stream.  As soon as
    // a panel has arrived, its block norms (and nearfield copies), its
    // column-basis leaf factors and R, and the row-basis leaves whose columns
    // lie in the panels so far run, under the copy of the next panel.
    const PanelPlan& pl = *hs->plan;
    dh2_matrix* M = Ms[0];
    const int64_t n = M->tree->tr.n;
    cudaStream_t cs = nullptr;
    std::vector<cudaEvent_t> pev(hK + 1, nullptr);
    bool own = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess;
    for (int k = 0; k <= hK && own; ++k) own = cudaEventCreateWithFlags(&pev[k], cudaEventDisableTiming) == cudaSuccess;
    cudaStream_t copy_st = own ? cs : st;  // without a second stream: copies in order on st
    if (own) {
      cudaEventRecord(pev[hK], st);
      cudaStreamWaitEvent(cs, pev[hK], 0);
    }
    for (int k = 0; k < hK; ++k) {
      const int64_t c0 = pl.col[k], nc = pl.col[k + 1] - c0;
      cudaMemcpy2DAsync((char*)M->G + (size_t)c0 * n * hs->elem, (size_t)n * hs->elem,
                        (const char*)hs->G_host + (size_t)c0 * hs->ld * hs->elem, (size_t)hs->ld * hs->elem,
                        (size_t)n * hs->elem, (size_t)nc, cudaMemcpyHostToDevice, copy_st);
      if (own) cudaEventRecord(pev[k], cs);
    }
#ifdef DH2_PROFILE
    prof_reset_pair();
#endif
    for (int k = 0; k < hK; ++k) {
      if (own) cudaStreamWaitEvent(st, pev[k], 0);
      if (!pl.blk[k].empty()) {
        launch_norms_near<T>(d_na, hl[k].d_codes, (int)pl.blk[k].size(), st);
        counted(DH2_KC_NORMS, true);
      }
      colw_side(kSideCol);
      const HList* Lc = &hl[(size_t)hK + 1 + (size_t)k * kLeafClasses];
      leaf_lists(Lc);
      leaf_rq(Lc);
      colw_side(kSideRow);
      const HList* Lr = &hl[(size_t)hK + 1 + (size_t)(hK + k) * kLeafClasses];
      leaf_lists(Lr);
      leaf_rq(Lr);
    }
    if (!pl.blk_rest.empty()) {
      launch_norms_near<T>(d_na, hl[hK].d_codes, (int)pl.blk_rest.size(), st);
      counted(DH2_KC_NORMS, true);
    }
    DH2_PHASE_SYNC("panels");
    rec(1);
    rec(2);
    for (cudaEvent_t e : pev)
      if (e) cudaEventDestroy(e);
    if (cs) cudaStreamDestroy(cs);
  } else {
    if (!any_gen) {
      // stored G: the admissible blocks in pieces of 32 rows by kNormCols
      // columns (maxima merged atomically into zeroed buffers, sums per piece,
      // then the weights), then the nearfield copies.  (The copies on a second
      // stream beside the leaf work slowed the kernels beside them by more than
      // their own time: measured, not kept.)
      for (int i = 0; i < nprob; ++i)
        if (nas[i].bmax)
          cudaMemsetAsync(nas[i].bmax, 0, sizeof(float) * (size_t)Ms[i]->tree->tr.dev->bmax_elems, st);
      launch_norms_adm<T>(d_na, d_pieces, n_pieces, d_norm_adm, d_pbegin, n_norm_adm, d_partial, st);
      counted(DH2_KC_NORMS, n_pieces > 0);
      counted(DH2_KC_NORMS, n_norm_adm > 0);
      const int64_t n_near = n_norm - n_norm_adm;
      if (n_near > 0 && cp.nearfield == 0) {
        launch_norms_near<T>(d_na, d_norm_near, (int)n_near, st);
        counted(DH2_KC_NORMS, true);
      }
    } else {
      launch_norms_near<T>(d_na, d_norm, (int)n_norm, st);
      counted(DH2_KC_NORMS, n_norm > 0);
    }
    colw_side(kSideRow);
    colw_side(kSideCol);
    DH2_PHASE_SYNC("norms_near");
    rec(1);
#ifdef DH2_PROFILE
    prof_reset_pair();
    prof_reset_gram();
#endif
    if (mixed && !plan) {
      kev_ok = true;
      for (int i = 0; i < 4 * kLeafClasses && kev_ok; ++i)
        kev_ok = cudaEventCreate(&kev[i]) == cudaSuccess;
      if (!kev_ok) cudaGetLastError();  // no split timing; the compression itself goes on
    }
    for (int c = 0; c < kLeafClasses; ++c)
      leaf_factor(d_leaf + cls_begin[c], (int)(cls_begin[c + 1] - cls_begin[c]), c,
                  kev_ok && cls_begin[c + 1] > cls_begin[c]);
    rec(2);
    // R of the leaf pairs: in the mixed mode one tensor-core launch over every
    // class's tiles; otherwise one launch per size class (shared memory sized by
    // the class's rows)
    const bool rq_tc = mixed && tune_current().rq_tensor != 0;
    if (rq_tc && tile_cls_begin[kLeafClasses] > 0) {
      if constexpr (std::is_same<T, float>::value) {
        const uint32_t sl = (uint32_t)std::min<int64_t>(std::max<int64_t>(cp.spin_limit, 0), (int64_t)UINT32_MAX);
        ok_launch &= launch_rq_tc(d_pa, d_ltiles, tile_cls_begin[kLeafClasses], sl, st);
        counted(DH2_KC_LEAF_R_TC, true);
      }
    }
    for (int c = 0; c < kLeafClasses && !rq_tc; ++c) {
      const int64_t nt = tile_cls_begin[c + 1] - tile_cls_begin[c];
      if (nt > 0) {
        ok_launch &= launch_rq_kernel<T>(d_pa, d_ltiles + tile_cls_begin[c], (int)nt, even_up(std::max(2, cls_maxm[c])), false,
                            any_gen, st);
        counted(DH2_KC_LEAF_R + c, true);
      }
    }
  }
#ifdef DH2_PROFILE
  if (!plan) {
    cudaStreamSynchronize(st);
    unsigned long long pr[17];
    prof_read_pair(pr);
    const double np = pr[5] ? (double)pr[5] : 1.0;
    const double ns = pr[12] ? (double)pr[12] : 1.0;
    unsigned long long gq[22];
    if (prof_read_gram(gq) && gq[10]) {
      const double pp = (double)gq[10];
      std::fprintf(stderr,
                   "dh2 gram pipeline profile: %llu pairs, %.2f chunks/pair; cycles/pair: producers wait %.0f, slice "
                   "%.0f, loads %.0f; MMA thread wait full %.0f, wait accumulators %.0f, issue %.0f; epilogue wait %.0f, "
                   "flush %.0f, H %.0f\n",
                   gq[10], gq[11] / pp, gq[12] / pp, gq[13] / pp, gq[14] / pp, gq[15] / pp, gq[16] / pp, gq[17] / pp,
                   gq[18] / pp, gq[19] / pp, gq[20] / pp);
    }
    if (prof_read_gram(gq) && gq[0]) {
      const double gp = (double)gq[0];
      std::fprintf(stderr,
                   "dh2 gram profile: %llu pairs, %.2f chunks/pair; cycles/pair (CTA thread 0): scales %.0f, table %.0f, "
                   "chunk loads %.0f, MMA waits %.0f, slicing %.0f, MMA issue %.0f, flush %.0f, H out %.0f\n",
                   gq[0], gq[1] / gp, gq[2] / gp, gq[3] / gp, gq[4] / gp, gq[5] / gp, gq[6] / gp, gq[7] / gp,
                   gq[8] / gp, gq[9] / gp);
    }
    std::fprintf(stderr,
                 "dh2 leaf-launch profile: %llu pairs, mean p %.1f, mean K %.1f, mean sweeps %.2f, mean chunks %.2f, "
                 "cycles/pair: LQ %.0f (staging %.0f) Jacobi %.0f rank+Q %.0f; LQ steps %.1f/pair, cycles/step %.0f, "
                 "per warp-step busy %.0f, critical warp busy %.0f, to reflection %.0f (loads %.0f, update %.0f, "
                 "form %.0f)\n",
                 pr[5], pr[6] / np, pr[7] / np, pr[4] / np, pr[9] / np, pr[0] / np, pr[8] / np, pr[1] / np,
                 pr[2] / np, ns / np, (pr[0] - pr[8]) / ns, pr[11] / (8.0 * ns), pr[10] / ns, pr[13] / ns,
                 pr[14] / ns, pr[15] / ns, pr[16] / ns);
  }
#endif
  DH2_PHASE_SYNC("leaf pairs");
  rec(3);
  {
    // the class split needs the sons' ranks, known only on the device: each
    // class is launched at the level's capacity and its CTAs past the class's
    // count (written by the classify kernel) return at once -- no read-back,
    // no host synchronisation inside the schedule
    uint32_t* d_cls = (uint32_t*)((char*)scratch + args_bytes + codes_bytes);
    int* d_cnt0 = (int*)((char*)d_cls + align256(4 * 4 * (size_t)std::max<int64_t>(nl_max, 1)));
    for (int l = maxdepth; l >= 0; --l) {
      if (n_nl[l] == 0) continue;
      const int n = (int)n_nl[l];
      int* d_cnt = d_cnt0 + 4 * l;  // per level, so that no launch waits on the host
      if (cudaMemsetAsync(d_cnt, 0, 4 * sizeof(int), st) != cudaSuccess) {
        cudaGetLastError();
        ok_launch = false;
      }
      launch_classify<T>(d_pa, d_nl[l], n, d_cls, d_cnt, st);
      counted(DH2_KC_CLASSIFY, true);
      const int Pc[4] = {32, 48, 64, P_level[l]};
      // wide pairs: their column segments' factors first, by row class
      const int nsg = (int)seg_lists[l].size();
      if (nsg > 0) {
        if (cudaMemsetAsync(d_seg_cnt[l], 0, 4 * sizeof(int), st) != cudaSuccess) {
          cudaGetLastError();
          ok_launch = false;
        }
        launch_classify_seg<T>(d_pa, d_seg[l], nsg, d_seg_cls[l], d_seg_cnt[l], st);
        counted(DH2_KC_CLASSIFY, true);
        for (int c = 0; c < 4; ++c) {
          if (c > 0 && Pc[c - 1] >= P_level[l]) break;
          ok_launch &= launch_pair_kernel<T>(d_pa, nullptr, nsg, std::min(Pc[c], std::max(P_level[l], 2)), true, st,
                                             d_seg_cnt[l] + c, d_seg_cls[l] + (int64_t)c * nsg);
          counted(DH2_KC_LEVEL_FACTOR + c, true);
        }
      }
      for (int c = 0; c < 4; ++c) {
        if (c > 0 && Pc[c - 1] >= P_level[l]) break;  // no pair of this level has more rows
        ok_launch &= launch_pair_kernel<T>(d_pa, d_cls + (int64_t)c * n, n, std::min(Pc[c], std::max(P_level[l], 2)),
                                           true, st, d_cnt + c);
        counted(DH2_KC_LEVEL_FACTOR + c, true);
      }
      ok_launch &= launch_rq_kernel<T>(d_pa, d_nltiles[l], (int)n_nltiles[l], P_level[l], true, any_gen, st);
      counted(DH2_KC_LEVEL_R, n_nltiles[l] > 0);
      DH2_PHASE_SYNC("non-leaf pairs");
    }
  }
  rec(4);
  for (dh2_matrix* M : Ms) {
    Tree& tr = M->tree->tr;
    Tree::Dev* D = tr.dev;
    SideView<T> Wv = side_view<T>(tr, M, 1);
    for (int l = tr.depth; l >= 0; --l) {
      const int64_t b = D->lvl_nl_begin[1][l], e = D->lvl_end[1][l];
      if (e > b) {
        launch_expand<T>(Wv, D->iota[1] + b, (int)(e - b), st);
        counted(DH2_KC_EXPAND, true);
      }
      DH2_PHASE_SYNC("expand");
    }
  }
  rec(5);
  for (dh2_matrix* M : Ms) {
    Tree& tr = M->tree->tr;
    Tree::Dev* D = tr.dev;
    ProjArgs<T> pj;
    pj.V = side_view<T>(tr, M, 0);
    pj.W = side_view<T>(tr, M, 1);
    pj.adm_list = D->adm_list;
    pj.bpair_row = D->bpair[0];
    pj.bpair_col = D->bpair[1];
    pj.boff_row = D->boff_row;
    pj.bs = D->bs;
    pj.csize = D->csize;
    pj.invw = M->invw;
    pj.S = (C2<T>*)M->S;
    pj.Soff = D->Soff;
    launch_project<T>(pj, (int)D->nadm, st);
    counted(DH2_KC_PROJECT, D->nadm > 0);
    DH2_PHASE_SYNC("project");
  }
  rec(6);
  if (plan) {
    cudaGraph_t g = nullptr;
    const cudaError_t e0 = cudaStreamEndCapture(st, &g);
    cudaError_t e1 = e0;
    if (e0 == cudaSuccess) e1 = cudaGraphInstantiate(&plan->exec, g, 0);
    if (e0 != cudaSuccess || e1 != cudaSuccess) {
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      plan->exec = nullptr;
      cudaFreeAsync(scratch, st);
      return DH2_ECUDA;
    }
    plan->graph = g;
    plan->scratch = scratch;
    plan->ok_launch = ok_launch;
    // new inputs: the matrix pointers in the host copies of the argument
    // blocks, then those blocks to the device (before the graph runs)
    plan->set_inputs = [pas, nas, gas, d_pa, d_na, d_ga, nprob, mixed](const void* const* G,
                                                                     cudaStream_t s2) mutable -> cudaError_t {
      for (int i = 0; i < nprob; ++i) {
        pas[i].G = (const C2<T>*)G[i];
        nas[i].G = (const C2<T>*)G[i];
        if (mixed) gas[i].G = (const C2<float>*)G[i];
      }
      cudaError_t e = cudaMemcpyAsync(d_pa, pas.data(), sizeof(PairArgs<T>) * nprob, cudaMemcpyHostToDevice, s2);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_na, nas.data(), sizeof(NormsArgs<T>) * nprob, cudaMemcpyHostToDevice, s2);
      if (e == cudaSuccess && mixed)
        e = cudaMemcpyAsync(d_ga, gas.data(), sizeof(GramArgs) * nprob, cudaMemcpyHostToDevice, s2);
      return e;
    };
    for (dh2_matrix* M : Ms) {
      M->launches = nlaunch;
      std::memcpy(M->class_launches, kcl, sizeof(kcl));
    }
    return DH2_OK;
  }
  cudaFreeAsync(scratch, st);
  std::vector<uint32_t> status(nprob, 0);
  cudaError_t e1 = cudaSuccess;
  for (int i = 0; i < nprob && e1 == cudaSuccess; ++i)
    e1 = cudaMemcpyAsync(&status[i], Ms[i]->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  cudaError_t e2 = cudaStreamSynchronize(st);
  cudaError_t e3 = cudaGetLastError();
  float ph[6] = {0, 0, 0, 0, 0, 0};
  for (int i = 0; i < 6; ++i) cudaEventElapsedTime(&ph[i], ev[i], ev[i + 1]);
  for (int i = 0; i < 7; ++i) cudaEventDestroy(ev[i]);
  float split[2] = {0, 0};
  for (int c = 0; c < kLeafClasses; ++c) {
    float a = 0, b = 0;
    if (kev_ok && cls_begin[c + 1] > cls_begin[c] && cudaEventElapsedTime(&a, kev[4 * c], kev[4 * c + 1]) == cudaSuccess &&
        cudaEventElapsedTime(&b, kev[4 * c + 2], kev[4 * c + 3]) == cudaSuccess) {
      split[0] += a;
      split[1] += b;
    }
  }
  for (cudaEvent_t e : kev)
    if (e) cudaEventDestroy(e);
  for (dh2_matrix* M : Ms) {
    std::memcpy(M->phase_ms, ph, sizeof(ph));
    std::memcpy(M->leaf_split_ms, split, sizeof(split));
    M->launches = nlaunch;
    std::memcpy(M->class_launches, kcl, sizeof(kcl));
  }
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) return DH2_ECUDA;
#ifdef DH2_CHECK
  {
    CheckRecord r1{}, r2{};
    const bool b1 = check_read_pair(&r1), b2 = check_read_ops(&r2);
    if (b1 || b2) {
      const CheckRecord& r = b1 ? r1 : r2;
      std::fprintf(stderr, "dh2 bounds check: %d violations, first at site %d item %d index %lld limit %lld\n",
                   r.count, r.where, r.item, (long long)r.index, (long long)r.limit);
      return DH2_EINVAL;
    }
  }
#endif
  uint32_t all = ok_launch ? 0u : kStatusTooLarge;
  for (uint32_t v : status) all |= v;
  // a timed-out wait leaves later results undefined: it is reported first
  if (all & kStatusTimeout) return DH2_ETIMEOUT;
  if (all & kStatusTooLarge) return DH2_EUNSUPPORTED;
  if (all & (kStatusNoConv | kStatusNaN)) return DH2_ENOCONV;
  return DH2_OK;
}

void matrix_release(dh2_matrix* M) {
  if (!M) return;
  if (M->gram) {
    cudaFreeAsync(M->gram, M->stream);
    cudaGetLastError();
  }
  if (M->arena) {
    cudaFreeAsync(M->arena, M->stream);
    cudaGetLastError();
  }
  delete M;
}

}  // namespace

extern "C" {

const char* dh2_status_string(dh2_status s) {
  switch (s) {
    case DH2_OK: return "ok";
    case DH2_EINVAL: return "invalid argument";
    case DH2_ENOMEM: return "out of memory";
    case DH2_ECUDA: return "CUDA runtime error";
    case DH2_ETIMEOUT: return "device wait timed out";
    case DH2_ENOCONV: return "Jacobi SVD did not converge within the sweep cap";
    case DH2_EUNSUPPORTED: return "size beyond a compiled limit";
  }
  return "unknown status";
}

const char* dh2_version(void) { return "dh2-gb300 0.1 (sm_103a)"; }

dh2_status dh2_tree_build(const double* pts_xyz, int64_t n, const dh2_tree_params* params, dh2_tree** out) {
  if (!out) return DH2_EINVAL;
  *out = nullptr;
  if (!params || !pts_xyz) return DH2_EINVAL;
  dh2_tree* T = new (std::nothrow) dh2_tree();
  if (!T) return DH2_ENOMEM;
  dh2_status s;
  try {
    s = build_tree(pts_xyz, n, *params, T->tr);
  } catch (const std::bad_alloc&) {
    s = DH2_ENOMEM;
  } catch (...) {
    s = DH2_EINVAL;
  }
  if (s != DH2_OK) {
    delete T;
    return s;
  }
  *out = T;
  return DH2_OK;
}

void dh2_tree_free(dh2_tree* T) {
  if (!T) return;
  if (T->g_stage) {
    cudaFree(T->g_stage);
    cudaGetLastError();
  }
  if (T->tr.dev) {
    cudaFree(T->tr.dev->arena);
    cudaGetLastError();
    delete T->tr.dev;
  }
  delete T;
}

dh2_status dh2_tree_stats_get(const dh2_tree* T, dh2_tree_stats* o) {
  if (!T || !o) return DH2_EINVAL;
  const Tree& tr = T->tr;
  std::memset(o, 0, sizeof(*o));
  o->n = tr.n;
  o->depth = tr.depth;
  o->nclusters = tr.nclusters();
  o->nblocks = (int64_t)tr.blocks.size();
  o->nadmissible = tr.nadm;
  o->adm_fraction = tr.adm_fraction;
  for (int sd = 0; sd < 2; ++sd) {
    o->npairs[sd] = (int64_t)tr.side[sd].pairs.size();
    o->nleafpairs[sd] = (int64_t)tr.side[sd].leaf_pairs.size();
    o->ncolumns[sd] = tr.side[sd].ncols_total;
    o->nleafcolumns[sd] = tr.side[sd].nleafcols;
  }
  o->max_leaf = tr.max_leaf;
  for (auto& d : tr.dirs) o->ndirs_max = std::max<int32_t>(o->ndirs_max, (int32_t)(d.size() / 3));
  return DH2_OK;
}

dh2_status dh2_tree_perm(const dh2_tree* T, int64_t* perm) {
  if (!T || !perm) return DH2_EINVAL;
  std::memcpy(perm, T->tr.perm.data(), sizeof(int64_t) * T->tr.perm.size());
  return DH2_OK;
}

dh2_status dh2_tree_clusters(const dh2_tree* T, int32_t* start, int32_t* size, int32_t* level, int32_t* parent,
                             int32_t* son0, int32_t* son1, double* lo, double* hi) {
  if (!T) return DH2_EINVAL;
  const Tree& tr = T->tr;
  const size_t nc = (size_t)tr.nclusters();
  if (start) std::memcpy(start, tr.start.data(), nc * 4);
  if (size) std::memcpy(size, tr.size.data(), nc * 4);
  if (level) std::memcpy(level, tr.level.data(), nc * 4);
  if (parent) std::memcpy(parent, tr.parent.data(), nc * 4);
  if (son0) std::memcpy(son0, tr.son0.data(), nc * 4);
  if (son1) std::memcpy(son1, tr.son1.data(), nc * 4);
  if (lo) std::memcpy(lo, tr.lo.data(), nc * 24);
  if (hi) std::memcpy(hi, tr.hi.data(), nc * 24);
  return DH2_OK;
}

dh2_status dh2_tree_ndirs(const dh2_tree* T, int32_t level, int32_t* ndirs) {
  if (!T || !ndirs || level < 0 || level > T->tr.depth) return DH2_EINVAL;
  *ndirs = (int32_t)(T->tr.dirs[level].size() / 3);
  return DH2_OK;
}

dh2_status dh2_tree_directions(const dh2_tree* Tc, int32_t level, double* dirs, int32_t* sd) {
  if (!Tc || level < 0 || level > Tc->tr.depth) return DH2_EINVAL;
  Tree& tr = const_cast<dh2_tree*>(Tc)->tr;
  const size_t nd = tr.dirs[level].size() / 3;
  if (dirs) std::memcpy(dirs, tr.dirs[level].data(), nd * 24);
  if (sd)
    for (size_t c = 0; c < nd; ++c) sd[c] = level < tr.depth ? tr.sd_of(level, (int32_t)c) : -1;
  return DH2_OK;
}

dh2_status dh2_tree_blocks(const dh2_tree* T, int32_t* t, int32_t* s, int32_t* adm, int32_t* cb) {
  if (!T) return DH2_EINVAL;
  const Tree& tr = T->tr;
  for (size_t b = 0; b < tr.blocks.size(); ++b) {
    if (t) t[b] = tr.blocks[b].t;
    if (s) s[b] = tr.blocks[b].s;
    if (adm) adm[b] = tr.blocks[b].adm;
    if (cb) cb[b] = tr.blocks[b].cb;
  }
  return DH2_OK;
}

dh2_status dh2_tree_pairs(const dh2_tree* T, int32_t side, int32_t* cluster, int32_t* dir, int64_t* ncols,
                          int32_t* is_leaf) {
  if (!T || (side != 0 && side != 1)) return DH2_EINVAL;
  const Side& S = T->tr.side[side];
  for (size_t p = 0; p < S.pairs.size(); ++p) {
    if (cluster) cluster[p] = S.pairs[p].cluster;
    if (dir) dir[p] = S.pairs[p].dir;
    if (ncols) ncols[p] = S.pairs[p].ncols;
    if (is_leaf) is_leaf[p] = S.pairs[p].leaf;
  }
  return DH2_OK;
}

dh2_status dh2_tree_pair_blocks(const dh2_tree* T, int32_t side, int64_t* offsets, int32_t* block_ids) {
  if (!T || (side != 0 && side != 1) || !offsets) return DH2_EINVAL;
  const Side& S = T->tr.side[side];
  std::vector<int32_t> tmp;
  std::function<void(int64_t)> emit = [&](int64_t p) {
    for (int32_t b : S.pairs[p].own) tmp.push_back(b);
    for (auto& seg : S.pairs[p].parents) emit(seg.first);
  };
  int64_t off = 0;
  for (size_t p = 0; p < S.pairs.size(); ++p) {
    tmp.clear();
    emit((int64_t)p);
    offsets[p] = off;
    if (block_ids) std::memcpy(block_ids + off, tmp.data(), tmp.size() * 4);
    off += (int64_t)tmp.size();
  }
  offsets[S.pairs.size()] = off;
  return DH2_OK;
}

dh2_status dh2_tree_panels(const dh2_tree* Tc, int32_t* npanels, int64_t* col, int32_t* row_panel) {
  if (!Tc || !npanels) return DH2_EINVAL;
  dh2_tree* T = const_cast<dh2_tree*>(Tc);  // the plan is a cache of the handle
  if (!T->plan_built) {
    make_panel_plan(T->tr, T->plan);
    T->plan_built = true;
  }
  const PanelPlan& pl = T->plan;
  const int K = (int)pl.col.size() - 1;
  *npanels = K;
  if (col) std::memcpy(col, pl.col.data(), sizeof(int64_t) * pl.col.size());
  if (row_panel) {
    const Side& S = T->tr.side[kSideRow];
    for (size_t p = 0; p < S.pairs.size(); ++p) row_panel[p] = -1;
    for (int k = 0; k < K; ++k)
      for (const auto& list : pl.row_leaf[k])
        for (uint32_t code : list) row_panel[code & kCodePairMask] = k;
  }
  return DH2_OK;
}

}  // extern "C"

namespace {

// Shared body of dh2_compress (G given) and dh2_compress_kernel (pts_host
// given: entries generated in the kernels).
dh2_status prepare_matrix(const dh2_tree* Tc, const void* G, dh2_dtype dtype, int64_t ld, const double* pts_host,
                          double kappa, double diag, const dh2_compress_params* params, void* stream,
                          dh2_matrix** out, const double* nrm_host = nullptr) {
  if (!out) return DH2_EINVAL;
  *out = nullptr;
  if (!Tc || !params || (!G && !pts_host)) return DH2_EINVAL;
  const dh2_compress_params& cp = *params;
  const bool gen = pts_host != nullptr;
  if (gen && (cp.nearfield != 0 || !(kappa >= 0.0) || !std::isfinite(diag))) return DH2_EINVAL;
  if (gen) ld = Tc->tr.n;
  if (ld < Tc->tr.n || !(cp.eps >= 0.0) || !(cp.zeta > 0.0 && cp.zeta < 1.0) || (cp.err_mode != 0 && cp.err_mode != 1) ||
      (cp.nearfield != 0 && cp.nearfield != 1))
    return DH2_EINVAL;
  if (!((cp.mode == DH2_MODE_FP64 && dtype == DH2_C128) || (mode_f32(cp.mode) && cp.mode <= DH2_MODE_MIXED_BF16X3 &&
                                                              dtype == DH2_C64)))
    return DH2_EINVAL;
  if (mode_mixed(cp.mode) && gen) return DH2_EUNSUPPORTED;  // the Gram kernel reads a stored G
  if (cp.err_mode == 0 && !(1.0 - 2.0 * cp.zeta * cp.zeta > 0.0)) return DH2_EINVAL;
  dh2_tree* T = const_cast<dh2_tree*>(Tc);
  Tree& tr = T->tr;
  const int pmax = mode_f32(cp.mode) ? kPmaxF32 : kPmaxF64;
  if (tr.max_leaf > pmax || (mode_mixed(cp.mode) && tr.max_leaf > 64)) return DH2_EUNSUPPORTED;
  int dev = 0;
  DH2_CUDA_TRY(cudaGetDevice(&dev));
  set_pool_threshold(dev);
  {
    const dh2_status s = ensure_device(tr, dev);
    if (s != DH2_OK) return s;
  }
  Tree::Dev* D = tr.dev;
  dh2_matrix* M = new (std::nothrow) dh2_matrix();
  if (!M) return DH2_ENOMEM;
  M->tree = T;
  M->device = dev;
  M->mode = cp.mode;
  M->dtype = dtype;
  M->es = dtype == DH2_C128 ? 16 : 8;
  M->stream = (cudaStream_t)stream;
  M->G = G;
  M->ld = ld;
  M->nearfield_copy = cp.nearfield == 0 ? 1 : 0;
  M->gen = gen ? 1 : 0;
  M->kappa = kappa;
  M->diag = diag;
  const size_t es = M->es;
  const int nl = tr.depth + 1;
  size_t sz[21];
  int ns = 0;
  sz[ns++] = align256(es * D->R_elems[0]);
  sz[ns++] = align256(es * D->R_elems[1]);
  sz[ns++] = align256(es * D->Q_elems[0]);
  sz[ns++] = align256(es * D->Q_elems[1]);
  sz[ns++] = align256(es * D->X_elems[0]);
  sz[ns++] = align256(es * D->X_elems[1]);
  sz[ns++] = align256(es * D->S_elems);
  sz[ns++] = align256(M->nearfield_copy ? es * D->near_elems : 0);
  sz[ns++] = align256(8 * kSigStride * D->npairs[0]);
  sz[ns++] = align256(8 * kSigStride * D->npairs[1]);
  sz[ns++] = align256(4 * D->npairs[0]);
  sz[ns++] = align256(4 * D->npairs[1]);
  sz[ns++] = align256(8 * tr.blocks.size());
  sz[ns++] = align256(8 * nl);
  sz[ns++] = align256(8 * nl);
  sz[ns++] = align256(16);
  sz[ns++] = align256(16);
  sz[ns++] = align256(gen ? (nrm_host ? 48 : 24) * (size_t)tr.n : 0);  // points (and normals)
  sz[ns++] = align256(es / 2 * (size_t)tr.side[0].nleafcols);
  sz[ns++] = align256(es / 2 * (size_t)tr.side[1].nleafcols);
  sz[ns++] = align256(8 * tr.blocks.size());
  size_t total = 0;
  for (int i = 0; i < ns; ++i) total += sz[i];
  if (dev_malloc_async(&M->arena, total, M->stream) != cudaSuccess) {
    cudaGetLastError();
    delete M;
    return DH2_ENOMEM;
  }
  M->arena_bytes = total;
  if (mode_mixed(cp.mode) && cp.keep_gram &&
      dev_malloc_async(&M->gram, std::max<size_t>(256, sizeof(float4) * (size_t)D->gram_elems), M->stream) !=
          cudaSuccess) {
    cudaGetLastError();
    M->gram = nullptr;
    matrix_release(M);
    return DH2_ENOMEM;
  }
  char* p = (char*)M->arena;
  void** dst[21] = {&M->R[0], &M->R[1], &M->Q[0], &M->Q[1], &M->X[0], &M->X[1], &M->S, &M->near,
                    (void**)&M->sig[0], (void**)&M->sig[1], (void**)&M->rank[0], (void**)&M->rank[1],
                    (void**)&M->invw, (void**)&M->eps2, (void**)&M->zpow, (void**)&M->status, (void**)&M->acc,
                    (void**)&M->pts, &M->colw[0], &M->colw[1], (void**)&M->bnorm2};
  for (int i = 0; i < ns; ++i) {
    *dst[i] = p;
    p += sz[i];
  }
  if (!M->nearfield_copy) M->near = nullptr;
  if (!gen) M->pts = nullptr;
  M->nrm = gen && nrm_host ? M->pts + 3 * (size_t)tr.n : nullptr;
  // tolerances eps_l = eps_hat zeta^l (Remark "Error control")
  const double eh =
      cp.err_mode == 0 ? cp.eps * std::sqrt(1.0 - 2.0 * cp.zeta * cp.zeta) / std::sqrt(2.0) : cp.eps;
  M->eps2_h.resize(nl);
  M->zpow_h.resize(nl);
  for (int l = 0; l < nl; ++l) {
    const double e = eh * std::pow(cp.zeta, (double)l);
    M->eps2_h[l] = e * e;
    M->zpow_h[l] = std::pow(cp.zeta, -(double)l);
  }
  cudaError_t ce = cudaMemcpyAsync(M->eps2, M->eps2_h.data(), 8 * nl, cudaMemcpyHostToDevice, M->stream);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(M->zpow, M->zpow_h.data(), 8 * nl, cudaMemcpyHostToDevice, M->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(M->status, 0, 16, M->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(M->rank[0], 0, 4 * D->npairs[0], M->stream);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(M->rank[1], 0, 4 * D->npairs[1], M->stream);
  if (ce == cudaSuccess && gen) {
    // points (then normals) in the tree's permuted order
    const size_t n3 = 3 * (size_t)tr.n;
    M->pts_h.resize(nrm_host ? 2 * n3 : n3);
    for (int64_t i = 0; i < tr.n; ++i)
      for (int c = 0; c < 3; ++c) {
        M->pts_h[3 * i + c] = pts_host[3 * tr.perm[i] + c];
        if (nrm_host) M->pts_h[n3 + 3 * i + c] = nrm_host[3 * tr.perm[i] + c];
      }
    ce = cudaMemcpyAsync(M->pts, M->pts_h.data(), 8 * M->pts_h.size(), cudaMemcpyHostToDevice, M->stream);
  }
  if (ce != cudaSuccess) {
    cudaGetLastError();
    matrix_release(M);
    return DH2_ECUDA;
  }
  *out = M;
  return DH2_OK;
}

// The mixed mode's leaf step squares the singular values: the slices'
// backward error (2^-23 of a row's largest entry) and the double-float Gram
// matrix resolve sigma^2 to about 2^-46 of the leaf matrix's squared norm,
// which reaches the tail sums of the rank rule once eps falls below ~1e-5.
// There (unless the Gram matrices are asked for) the leaves take the FP32
// streamed LQ, which works on the leaf matrix itself.
constexpr double kMixedMinEps = 1e-5;
dh2_compress_params leaf_path(const dh2_compress_params& p) {
  dh2_compress_params q = p;
  if (mode_mixed(p.mode) && p.eps < kMixedMinEps && !p.keep_gram) q.mode = DH2_MODE_FP32;
  return q;
}

dh2_status compress_impl(const dh2_tree* Tc, const void* G, dh2_dtype dtype, int64_t ld, const double* pts_host,
                         double kappa, double diag, const dh2_compress_params* params, void* stream,
                         dh2_matrix** out, const double* nrm_host = nullptr) {
  if (!out) return DH2_EINVAL;
  *out = nullptr;  // stays NULL on every failure below
  if (!params) return DH2_EINVAL;
  const dh2_compress_params qp = leaf_path(*params);
  params = &qp;
  dh2_matrix* M = nullptr;
  dh2_status s = prepare_matrix(Tc, G, dtype, ld, pts_host, kappa, diag, params, stream, &M, nrm_host);
  if (s != DH2_OK) return s;
  std::vector<dh2_matrix*> Ms{M};
  s = mode_f32(params->mode) ? run_compress<float>(Ms, *params, (cudaStream_t)stream)
                                    : run_compress<double>(Ms, *params, (cudaStream_t)stream);
  if (s != DH2_OK) {
    matrix_release(M);
    return s;
  }
  *out = M;
  return DH2_OK;
}

}  // namespace

extern "C" {

dh2_status dh2_compress(const dh2_tree* Tc, const void* G, dh2_dtype dtype, int64_t ld,
                        const dh2_compress_params* params, void* stream, dh2_matrix** out) {
  if (!G) {
    if (out) *out = nullptr;
    return DH2_EINVAL;
  }
  return compress_impl(Tc, G, dtype, ld, nullptr, 0.0, 0.0, params, stream, out);
}

dh2_status dh2_compress_host(const dh2_tree* Tc, const void* G_host, dh2_dtype dtype, int64_t ld,
                             const dh2_compress_params* params, void* stream, dh2_matrix** out) {
  if (out) *out = nullptr;
  if (!Tc || !G_host || !params || !out || params->nearfield != 0) return DH2_EINVAL;
  if (dtype != DH2_C64 && dtype != DH2_C128) return DH2_EINVAL;
  const dh2_compress_params qp = leaf_path(*params);
  params = &qp;
  const int64_t n = Tc->tr.n;
  if (ld < n) return DH2_EINVAL;
  const size_t elem = dtype == DH2_C64 ? 8 : 16;
  // the staging buffer and the panel plan are caches of the tree handle
  dh2_tree* T = const_cast<dh2_tree*>(Tc);
  const size_t bytes = (size_t)n * (size_t)n * elem;
  if (T->g_stage_bytes < bytes) {
    if (T->g_stage) cudaFree(T->g_stage);  // synchronises: no earlier call still reads it
    T->g_stage = nullptr;
    T->g_stage_bytes = 0;
    if (dev_malloc(&T->g_stage, bytes) != cudaSuccess) {
      cudaGetLastError();
      T->g_stage = nullptr;
      return DH2_ENOMEM;
    }
    T->g_stage_bytes = bytes;
  }
  if (!T->plan_built) {
    make_panel_plan(T->tr, T->plan);
    T->plan_built = true;
  }
  dh2_matrix* M = nullptr;
  dh2_status s = prepare_matrix(Tc, T->g_stage, dtype, n, nullptr, 0.0, 0.0, params, stream, &M);
  if (s != DH2_OK) return s;
  const HostStage hs{G_host, ld, elem, &T->plan};
  std::vector<dh2_matrix*> Ms{M};
  s = mode_f32(params->mode) ? run_compress<float>(Ms, *params, (cudaStream_t)stream, &hs)
                                    : run_compress<double>(Ms, *params, (cudaStream_t)stream, &hs);
  if (s != DH2_OK) {
    matrix_release(M);
    return s;
  }
  M->G = nullptr;  // the staging buffer stays the tree's, for the next call
  *out = M;
  return DH2_OK;
}

dh2_status dh2_compress_kernel(const dh2_tree* Tc, const double* pts_xyz, double kappa, double diag,
                               const dh2_compress_params* params, void* stream, dh2_matrix** out) {
  if (!pts_xyz || !params) {
    if (out) *out = nullptr;
    return DH2_EINVAL;
  }
  const dh2_dtype dt = mode_f32(params->mode) ? DH2_C64 : DH2_C128;
  return compress_impl(Tc, nullptr, dt, 0, pts_xyz, kappa, diag, params, stream, out);
}

dh2_status dh2_compress_kernel_dlp(const dh2_tree* Tc, const double* pts_xyz, const double* normals_xyz, double kappa,
                                   const dh2_compress_params* params, void* stream, dh2_matrix** out) {
  if (!pts_xyz || !normals_xyz || !params) {
    if (out) *out = nullptr;
    return DH2_EINVAL;
  }
  const dh2_dtype dt = mode_f32(params->mode) ? DH2_C64 : DH2_C128;
  return compress_impl(Tc, nullptr, dt, 0, pts_xyz, kappa, 0.5, params, stream, out, normals_xyz);
}

dh2_status dh2_compress_batched(int32_t nprob, const dh2_tree* const* trees, const void* const* G,
                                const int64_t* ld, dh2_dtype dtype, const dh2_compress_params* params, void* stream,
                                dh2_matrix** out) {
  if (!out || nprob < 1) return DH2_EINVAL;
  for (int i = 0; i < nprob; ++i) out[i] = nullptr;
  if (nprob > kMaxBatch || !trees || !G || !ld || !params) return DH2_EINVAL;
  if (nprob > 1 && (params->rank_override[0] || params->rank_override[1])) return DH2_EINVAL;  // one problem's ranks
  const dh2_compress_params qp = leaf_path(*params);
  params = &qp;
  std::vector<dh2_matrix*> Ms;
  for (int i = 0; i < nprob; ++i) {
    dh2_matrix* M = nullptr;
    const dh2_status s = G[i] ? prepare_matrix(trees[i], G[i], dtype, ld[i], nullptr, 0.0, 0.0, params, stream, &M)
                              : DH2_EINVAL;
    if (s != DH2_OK) {
      for (dh2_matrix* m : Ms) matrix_release(m);
      return s;
    }
    Ms.push_back(M);
  }
  const dh2_status s = mode_f32(params->mode) ? run_compress<float>(Ms, *params, (cudaStream_t)stream)
                                                     : run_compress<double>(Ms, *params, (cudaStream_t)stream);
  if (s != DH2_OK) {
    for (dh2_matrix* m : Ms) matrix_release(m);
    return s;
  }
  for (int i = 0; i < nprob; ++i) out[i] = Ms[i];
  return DH2_OK;
}

struct dh2_plan {
  std::vector<dh2_matrix*> Ms;
  std::vector<const void*> G;  // the matrices of the last run
  PlanState ps;
  cudaStream_t stream = nullptr;  // the library's stream the schedule was prepared and captured on
};

dh2_status dh2_plan_create(int32_t nprob, const dh2_tree* const* trees, const void* const* G, const int64_t* ld,
                           dh2_dtype dtype, const dh2_compress_params* params, void* stream, dh2_plan** out) {
  if (!out || nprob < 1) return DH2_EINVAL;
  *out = nullptr;
  if (nprob > kMaxBatch || !trees || !G || !ld || !params) return DH2_EINVAL;
  if (nprob > 1 && (params->rank_override[0] || params->rank_override[1])) return DH2_EINVAL;
  const dh2_compress_params qp = leaf_path(*params);
  params = &qp;
  dh2_plan* P = new (std::nothrow) dh2_plan;
  if (!P) return DH2_ENOMEM;
  // the capture runs on a stream of the library's own (the caller's may be the
  // legacy default stream, which cannot be captured); the caller's stream is
  // synchronised once the representations are allocated on it
  if (cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete P;
    return DH2_ECUDA;
  }
  for (int i = 0; i < nprob; ++i) {
    dh2_matrix* M = nullptr;
    const dh2_status s = G[i] ? prepare_matrix(trees[i], G[i], dtype, ld[i], nullptr, 0.0, 0.0, params, stream, &M)
                              : DH2_EINVAL;
    if (s != DH2_OK) {
      for (dh2_matrix* m : P->Ms) matrix_release(m);
      delete P;
      return s;
    }
    P->Ms.push_back(M);
    P->G.push_back(G[i]);
  }
  dh2_status s = cudaStreamSynchronize((cudaStream_t)stream) == cudaSuccess ? DH2_OK : DH2_ECUDA;
  if (s == DH2_OK)
    s = mode_f32(params->mode) ? run_compress<float>(P->Ms, *params, P->stream, nullptr, &P->ps)
                               : run_compress<double>(P->Ms, *params, P->stream, nullptr, &P->ps);
  if (s == DH2_OK && cudaStreamSynchronize(P->stream) != cudaSuccess) s = DH2_ECUDA;  // uploads done
  if (s == DH2_OK && !P->ps.ok_launch) s = DH2_EUNSUPPORTED;
  if (s != DH2_OK) {
    cudaGetLastError();
    dh2_plan_free(P);
    return s;
  }
  *out = P;
  return DH2_OK;
}

dh2_status dh2_plan_run(dh2_plan* P, const void* const* G, void* stream) {
  if (!P || !P->ps.exec) return DH2_EINVAL;
  const int n = (int)P->Ms.size();
  if (G)
    for (int i = 0; i < n; ++i) {
      if (!G[i]) return DH2_EINVAL;
      P->G[i] = G[i];
    }
  for (int i = 0; i < n; ++i) P->Ms[i]->G = P->G[i];  // view-mode nearfield, products and errors read it
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = P->ps.set_inputs(P->G.data(), st);
  if (e == cudaSuccess) e = cudaGraphLaunch(P->ps.exec, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return DH2_ECUDA;
  }
  return DH2_OK;
}

dh2_status dh2_plan_wait(dh2_plan* P, void* stream) {
  if (!P) return DH2_EINVAL;
  const int n = (int)P->Ms.size();
  std::vector<uint32_t> status(n, 0);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < n && e == cudaSuccess; ++i)
    e = cudaMemcpyAsync(&status[i], P->Ms[i]->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
  const cudaError_t e2 = cudaStreamSynchronize(st);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    cudaGetLastError();
    return DH2_ECUDA;
  }
  uint32_t all = 0;
  for (uint32_t v : status) all |= v;
  if (all & kStatusTimeout) return DH2_ETIMEOUT;
  if (all & kStatusTooLarge) return DH2_EUNSUPPORTED;
  if (all & (kStatusNoConv | kStatusNaN)) return DH2_ENOCONV;
  return DH2_OK;
}

dh2_status dh2_plan_matrix(const dh2_plan* P, int32_t i, dh2_matrix** M) {
  if (!P || !M || i < 0 || i >= (int32_t)P->Ms.size()) return DH2_EINVAL;
  *M = P->Ms[i];
  return DH2_OK;
}

void dh2_plan_free(dh2_plan* P) {
  if (!P) return;
  // replays may still run on the caller's streams: the device finishes first
  cudaDeviceSynchronize();
  if (P->ps.exec) cudaGraphExecDestroy(P->ps.exec);
  if (P->ps.graph) cudaGraphDestroy(P->ps.graph);
  if (P->ps.scratch) cudaFreeAsync(P->ps.scratch, P->stream);
  for (dh2_matrix* m : P->Ms) matrix_release(m);
  if (P->stream) {
    cudaStreamSynchronize(P->stream);
    cudaStreamDestroy(P->stream);
  }
  cudaGetLastError();
  delete P;
}

dh2_status dh2_tuning_get(dh2_tuning* out) {
  if (!out) return DH2_EINVAL;
  *out = from_table(tune_current());
  return DH2_OK;
}

dh2_status dh2_tuning_set(const dh2_tuning* t) {
  if (!t || !tune_valid(*t)) return DH2_EINVAL;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune = to_table(*t);
  return DH2_OK;
}

dh2_status dh2_autotune(const dh2_tree* T, const void* G, dh2_dtype dtype, int64_t ld,
                        const dh2_compress_params* params, void* stream, int32_t reps, dh2_tuning* out,
                        dh2_tune_record* records, int32_t cap, int32_t* nrec) {
  if (nrec) *nrec = 0;
  if (!T || !G || !params || !out || reps < 1 || reps > 15 || (records && (cap < 0 || !nrec))) return DH2_EINVAL;
  const TuneTable saved = tune_current();
  const bool mixed = mode_mixed(leaf_path(*params).mode);
  // factor classes with leaf pairs in this problem
  bool has[5] = {false, false, false, false, false};
  for (int sd = 0; sd < 2; ++sd)
    for (int64_t p : T->tr.side[sd].leaf_pairs) has[leaf_class(T->tr.size[T->tr.side[sd].pairs[p].cluster])] = true;
  auto install = [&](const TuneTable& x) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune = x;
  };
  int nr = 0;
  // median over reps of the device time of the phases the knob acts on
  auto timed = [&](const TuneTable& x, int knob, int cls, int value, float* med) -> dh2_status {
    install(x);
    std::vector<float> t;
    for (int r = 0; r < reps; ++r) {
      dh2_matrix* M = nullptr;
      const dh2_status s = dh2_compress(T, G, dtype, ld, params, stream, &M);
      if (s != DH2_OK) return s;
      t.push_back(knob == 0 || knob == 3 ? M->phase_ms[2]
                  : knob == 4            ? M->phase_ms[3]
                                         : (mixed ? M->leaf_split_ms[1] : M->phase_ms[1]) + M->phase_ms[3]);
      dh2_matrix_free(M);
    }
    std::sort(t.begin(), t.end());
    *med = t[t.size() / 2];
    if (records && nr < cap) records[nr++] = dh2_tune_record{knob, cls, value, *med};
    return DH2_OK;
  };
  // one knob: every candidate from the current best table, keep the fastest
  TuneTable best = saved;
  auto descend = [&](int knob, int cls, const int* cand, int ncand, int32_t* field_of_best) -> dh2_status {
    float tbest = 0.f;
    int vbest = *field_of_best;
    for (int i = 0; i < ncand; ++i) {
      TuneTable x = best;
      int32_t* f = knob == 0   ? &x.rq_ctas_per_sm
                   : knob == 1 ? &x.jacobi_narrow[cls]
                   : knob == 2 ? &x.jacobi_tpp[cls]
                   : knob == 3 ? &x.rq_tensor
                               : &x.level_seg_cols;
      *f = cand[i];
      float ms = 0.f;
      const dh2_status s = timed(x, knob, cls, cand[i], &ms);
      if (s != DH2_OK) return s;
      if (i == 0 || ms < tbest) {
        tbest = ms;
        vbest = cand[i];
      }
    }
    *field_of_best = vbest;
    return DH2_OK;
  };
  dh2_status s = DH2_OK;
  {
    dh2_matrix* M = nullptr;  // untimed first call: uploads and first-use allocations
    s = dh2_compress(T, G, dtype, ld, params, stream, &M);
    if (s == DH2_OK) dh2_matrix_free(M);
  }
  static const int kRq[3] = {0, 1, 2}, kNarrow[3] = {0, 1, 2}, kTpp[3] = {32, 16, 8}, kTensor[2] = {0, 1};
  if (s == DH2_OK && mixed) s = descend(3, 0, kTensor, 2, &best.rq_tensor);
  if (s == DH2_OK) s = descend(0, 0, kRq, 3, &best.rq_ctas_per_sm);
  // the level steps' column segments, if the problem has non-leaf pairs wide enough to split
  bool wide = false;
  for (int sd = 0; sd < 2; ++sd)
    for (const Pair& P : T->tr.side[sd].pairs) wide = wide || (!P.leaf && P.ncols > 2 * 512);
  static const int kSeg[4] = {1024, 0, 512, 2048};
  if (s == DH2_OK && wide) s = descend(4, 0, kSeg, 4, &best.level_seg_cols);
  for (int c = 0; c < 5 && s == DH2_OK; ++c) {
    if (!has[c]) continue;
    if (mixed && c < 4) s = descend(1, c, kNarrow, 3, &best.jacobi_narrow[c]);
    if (s == DH2_OK) s = descend(2, c, kTpp, 3, &best.jacobi_tpp[c]);
  }
  if (nrec) *nrec = nr;
  if (s != DH2_OK) {
    install(saved);
    return s;
  }
  install(best);
  *out = from_table(best);
  return DH2_OK;
}

void dh2_matrix_free(dh2_matrix* M) { matrix_release(M); }

}  // extern "C"

namespace {

template <typename T>
dh2_status run_matvec(const dh2_matrix* M, const void* xv, void* yv, int nrhs, cudaStream_t st) {
  Tree& tr = M->tree->tr;
  Tree::Dev* D = tr.dev;
  const int64_t n = tr.n;
  void* buf = nullptr;
  const size_t hx = align256(sizeof(C2<T>) * D->h_elems[1] * nrhs);
  const size_t hy = align256(sizeof(C2<T>) * D->h_elems[0] * nrhs);
  if (dev_malloc_async(&buf, hx + hy + 256, st) != cudaSuccess) {
    cudaGetLastError();
    return DH2_ENOMEM;
  }
  C2<T>* xh = (C2<T>*)buf;
  C2<T>* yh = (C2<T>*)((char*)buf + hx);
  const C2<T>* x = (const C2<T>*)xv;
  C2<T>* y = (C2<T>*)yv;
  cudaMemsetAsync(y, 0, sizeof(C2<T>) * n * nrhs, st);
  SideView<T> Vv = side_view<T>(tr, M, 0), Wv = side_view<T>(tr, M, 1);
  // forward transformation (column basis), leaves then upwards
  launch_mv_forward_leaf<T>(Wv, D->leaf_list[1], (int)D->nleaf[1], x, nrhs, n, xh, D->hoff[1], st);
  for (int l = tr.depth; l >= 0; --l) {
    const int64_t b = D->lvl_nl_begin[1][l], e = D->lvl_end[1][l];
    if (e > b) launch_mv_forward_up<T>(Wv, D->iota[1] + b, (int)(e - b), nrhs, xh, D->hoff[1], st);
  }
  MvArgs<T> a;
  a.V = Vv;
  a.W = Wv;
  a.S = (const C2<T>*)M->S;
  a.Soff = D->Soff;
  a.own_ptr = D->own_ptr;
  a.own_blk = D->own_blk;
  a.bpair_col = D->bpair[1];
  a.xh = xh;
  a.xhoff = D->hoff[1];
  a.yh = yh;
  a.yhoff = D->hoff[0];
  a.par_ptr = D->par_ptr;
  a.par_pair = D->par_pair;
  a.par_son = D->par_son;
  a.bt = D->bt;
  a.bs = D->bs;
  a.near = (const C2<T>*)M->near;
  a.near_off = D->near_off;
  a.G = (const C2<T>*)M->G;
  a.ld = M->ld;
  launch_mv_coupling<T>(a, (int)D->npairs[0], nrhs, st);
  // backward transformation, top-down
  for (int l = 1; l <= tr.depth; ++l) {
    const int64_t b = D->lvl_begin[0][l], e = D->lvl_end[0][l];
    if (e > b) launch_mv_backward_down<T>(a, D->iota[0] + b, (int)(e - b), nrhs, st);
  }
  launch_mv_backward_leaf<T>(a, D->leaf_list[0], (int)D->nleaf[0], nrhs, y, n, st);
  launch_mv_near<T>(a, D->inadm_list, (int)D->ninadm, nrhs, x, y, n, st);
  cudaFreeAsync(buf, st);
  DH2_CUDA_TRY(cudaGetLastError());
  return DH2_OK;
}

// y = G~^* x: the product of Section 4 with the roles of the row and column
// bases exchanged (forward on V, coupling with S_b^*, backward on W) plus
// G_b^* on the nearfield.
template <typename T>
dh2_status run_matvec_adj(const dh2_matrix* M, const void* xv, void* yv, int nrhs, cudaStream_t st) {
  Tree& tr = M->tree->tr;
  Tree::Dev* D = tr.dev;
  const int64_t n = tr.n;
  void* buf = nullptr;
  const size_t hx = align256(sizeof(C2<T>) * D->h_elems[0] * nrhs);
  const size_t hy = align256(sizeof(C2<T>) * D->h_elems[1] * nrhs);
  if (dev_malloc_async(&buf, hx + hy + 256, st) != cudaSuccess) {
    cudaGetLastError();
    return DH2_ENOMEM;
  }
  C2<T>* xh = (C2<T>*)buf;
  C2<T>* yh = (C2<T>*)((char*)buf + hx);
  const C2<T>* x = (const C2<T>*)xv;
  C2<T>* y = (C2<T>*)yv;
  cudaMemsetAsync(y, 0, sizeof(C2<T>) * n * nrhs, st);
  SideView<T> Vv = side_view<T>(tr, M, 0), Wv = side_view<T>(tr, M, 1);
  launch_mv_forward_leaf<T>(Vv, D->leaf_list[0], (int)D->nleaf[0], x, nrhs, n, xh, D->hoff[0], st);
  for (int l = tr.depth; l >= 0; --l) {
    const int64_t b = D->lvl_nl_begin[0][l], e = D->lvl_end[0][l];
    if (e > b) launch_mv_forward_up<T>(Vv, D->iota[0] + b, (int)(e - b), nrhs, xh, D->hoff[0], st);
  }
  MvArgs<T> a;
  a.V = Wv;  // exchanged sides
  a.W = Vv;
  a.S = (const C2<T>*)M->S;
  a.Soff = D->Soff;
  a.own_ptr = D->own_ptr_c;
  a.own_blk = D->own_blk_c;
  a.bpair_col = D->bpair[0];
  a.xh = xh;
  a.xhoff = D->hoff[0];
  a.yh = yh;
  a.yhoff = D->hoff[1];
  a.par_ptr = D->par_ptr_c;
  a.par_pair = D->par_pair_c;
  a.par_son = D->par_son_c;
  a.bt = D->bt;
  a.bs = D->bs;
  a.near = (const C2<T>*)M->near;
  a.near_off = D->near_off;
  a.G = (const C2<T>*)M->G;
  a.ld = M->ld;
  launch_mv_coupling_adj<T>(a, (int)D->npairs[1], nrhs, st);
  for (int l = 1; l <= tr.depth; ++l) {
    const int64_t b = D->lvl_begin[1][l], e = D->lvl_end[1][l];
    if (e > b) launch_mv_backward_down<T>(a, D->iota[1] + b, (int)(e - b), nrhs, st);
  }
  launch_mv_backward_leaf<T>(a, D->leaf_list[1], (int)D->nleaf[1], nrhs, y, n, st);
  launch_mv_near_adj<T>(a, D->inadm_list, (int)D->ninadm, nrhs, x, y, n, st);
  cudaFreeAsync(buf, st);
  DH2_CUDA_TRY(cudaGetLastError());
  return DH2_OK;
}

// Relative spectral error |G_ref - G~|_2 / |G_ref|_2 by power iteration (the
// error measure of the paper's experiments, Section 7): the largest
// eigenvalue of E^* E with E = G_ref - G~ (products with G_ref and G_ref^* in
// FP64, with G~ and G~^* by the library's product and adjoint product in the
// matrix's arithmetic), and likewise of G_ref^* G_ref, each from a fixed
// seeded start vector until the estimate changes by less than 1e-6 relative
// (at most kSpectralIters products).
constexpr int kSpectralIters = 60;

template <typename T>
dh2_status run_error_spectral(dh2_matrix* M, const void* Gref, dh2_dtype rdt, int64_t ldr, cudaStream_t st,
                              double* rel) {
  Tree& tr = M->tree->tr;
  const int64_t n = tr.n;
  ErrArgs<float> gen{};
  gen.pts = M->pts;
  gen.nrm = M->nrm;
  gen.kappa = M->kappa;
  gen.diag = M->diag;
  void* buf = nullptr;
  const size_t vb = align256(sizeof(C2<double>) * n), tb = align256(sizeof(C2<T>) * n);
  if (dev_malloc_async(&buf, 3 * vb + 2 * tb + 256, st) != cudaSuccess) {
    cudaGetLastError();
    return DH2_ENOMEM;
  }
  C2<double>* v = (C2<double>*)buf;
  C2<double>* u = (C2<double>*)((char*)buf + vb);
  C2<double>* w = (C2<double>*)((char*)buf + 2 * vb);
  C2<T>* xt = (C2<T>*)((char*)buf + 3 * vb);
  C2<T>* yt = (C2<T>*)((char*)buf + 3 * vb + tb);
  auto gemv = [&](bool trans, const C2<double>* x, C2<double>* y) {
    if (rdt == DH2_C128 && Gref) launch_gemv<double>((const C2<double>*)Gref, ldr, gen, n, trans, x, y, st);
    else launch_gemv<float>((const C2<float>*)Gref, ldr, gen, n, trans, x, y, st);
  };
  double* d_n2 = M->acc + 2;  // |w|^2 of the current iteration (device)
  // seeded start vector of unit norm, on the device
  auto start = [&]() -> dh2_status {
    launch_seed_vector(v, n, 0x9E3779B97F4A7C15ull, st);
    DH2_CUDA_TRY(cudaMemsetAsync(d_n2, 0, sizeof(double), st));
    launch_norm2(v, n, d_n2, st);
    launch_normalize(v, v, n, d_n2, st);
    return DH2_OK;
  };
  // lambda_max(A^* A) for A = G_ref - G~ (err) or A = G_ref; w = A^* A v, v <- w / |w|
  auto power = [&](bool err, double* lam) -> dh2_status {
    dh2_status s = start();
    if (s != DH2_OK) return s;
    double prev = 0.0;
    for (int it = 0; it < kSpectralIters; ++it) {
      gemv(false, v, u);
      if (err) {
        launch_to_type<T>(v, xt, n, st);
        s = run_matvec<T>(M, xt, yt, 1, st);
        if (s != DH2_OK) return s;
        launch_sub<T>(u, yt, n, st);
      }
      gemv(true, u, w);
      if (err) {
        launch_to_type<T>(u, xt, n, st);
        s = run_matvec_adj<T>(M, xt, yt, 1, st);
        if (s != DH2_OK) return s;
        launch_sub<T>(w, yt, n, st);
      }
      DH2_CUDA_TRY(cudaMemsetAsync(d_n2, 0, sizeof(double), st));
      launch_norm2(w, n, d_n2, st);
      launch_normalize(v, w, n, d_n2, st);
      double s2 = 0.0;
      DH2_CUDA_TRY(cudaMemcpyAsync(&s2, d_n2, sizeof(double), cudaMemcpyDeviceToHost, st));
      DH2_CUDA_TRY(cudaStreamSynchronize(st));
      const double nw = std::sqrt(s2);  // |A^* A v| with |v| = 1
      *lam = nw;
      if (!(nw > 0.0)) return DH2_OK;
      if (it > 2 && std::fabs(nw - prev) <= 1e-6 * nw) break;
      prev = nw;
    }
    return DH2_OK;
  };
  double le = 0.0, lg = 0.0;
  dh2_status s = power(true, &le);
  if (s == DH2_OK) s = power(false, &lg);
  cudaFreeAsync(buf, st);
  if (s != DH2_OK) return s;
  DH2_CUDA_TRY(cudaStreamSynchronize(st));
  *rel = lg > 0.0 ? std::sqrt(le / lg) : 0.0;
  return DH2_OK;
}

template <typename T>
dh2_status run_error(dh2_matrix* M, const void* Gref, dh2_dtype rdt, int64_t ldr, int which, cudaStream_t st,
                     double* rel) {
  Tree& tr = M->tree->tr;
  Tree::Dev* D = tr.dev;
  SideView<T> Vv = side_view<T>(tr, M, 0), Wv = side_view<T>(tr, M, 1);
  if (!M->v_expanded) {
    for (int l = tr.depth; l >= 0; --l) {
      const int64_t b = D->lvl_nl_begin[0][l], e = D->lvl_end[0][l];
      if (e > b) launch_expand<T>(Vv, D->iota[0] + b, (int)(e - b), st);
    }
    M->v_expanded = true;
  }
  ErrArgs<T> a;
  a.V = Vv;
  a.W = Wv;
  a.S = (const C2<T>*)M->S;
  a.Soff = D->Soff;
  a.bt = D->bt;
  a.bs = D->bs;
  a.badm = D->badm;
  a.bpair_row = D->bpair[0];
  a.bpair_col = D->bpair[1];
  a.cstart = D->cstart;
  a.csize = D->csize;
  a.near = (const C2<T>*)M->near;
  a.near_off = D->near_off;
  a.G = (const C2<T>*)M->G;
  a.ld = M->ld;
  a.pts = M->pts;
  a.nrm = M->nrm;
  a.kappa = M->kappa;
  a.diag = M->diag;
  a.ref_gen = Gref == nullptr ? 1 : 0;
  if (which == DH2_ERR_SPECTRAL) return run_error_spectral<T>(M, Gref, rdt, ldr, st, rel);
  DH2_CUDA_TRY(cudaMemsetAsync(M->acc, 0, 16, st));
  if (which == DH2_ERR_FRO_CLOSED) launch_closed_form<T>(a, M->bnorm2, (int)tr.blocks.size(), M->acc, st);
  else if (rdt == DH2_C128)
    launch_error<T, double>(a, (const C2<double>*)Gref, ldr, (int)tr.blocks.size(), M->acc, st);
  else
    launch_error<T, float>(a, (const C2<float>*)Gref, ldr, (int)tr.blocks.size(), M->acc, st);
  double h[2] = {0, 0};
  DH2_CUDA_TRY(cudaMemcpyAsync(h, M->acc, 16, cudaMemcpyDeviceToHost, st));
  DH2_CUDA_TRY(cudaStreamSynchronize(st));
  *rel = h[1] > 0 ? std::sqrt(std::max(0.0, h[0]) / h[1]) : 0.0;
  return DH2_OK;
}

}  // namespace

extern "C" {

dh2_status dh2_matvec(const dh2_matrix* M, const void* x, void* y, int32_t nrhs, void* stream) {
  if (!M || !x || !y || nrhs < 1) return DH2_EINVAL;
  return mode_f32(M->mode) ? run_matvec<float>(M, x, y, nrhs, (cudaStream_t)stream)
                                  : run_matvec<double>(M, x, y, nrhs, (cudaStream_t)stream);
}

dh2_status dh2_matvec_adjoint(const dh2_matrix* M, const void* x, void* y, int32_t nrhs, void* stream) {
  if (!M || !x || !y || nrhs < 1) return DH2_EINVAL;
  return mode_f32(M->mode) ? run_matvec_adj<float>(M, x, y, nrhs, (cudaStream_t)stream)
                           : run_matvec_adj<double>(M, x, y, nrhs, (cudaStream_t)stream);
}

dh2_status dh2_error(const dh2_matrix* Mc, const void* G_ref, dh2_dtype ref_dtype, int64_t ld, int32_t which,
                     void* stream, double* rel_err) {
  if (!Mc || !rel_err || which < DH2_ERR_FRO_BLOCKWISE || which > DH2_ERR_SPECTRAL) return DH2_EINVAL;
  if (which != DH2_ERR_FRO_CLOSED && (G_ref ? ld < Mc->tree->tr.n : !Mc->gen)) return DH2_EINVAL;
  if (G_ref && ref_dtype != DH2_C64 && ref_dtype != DH2_C128) return DH2_EINVAL;
  dh2_matrix* M = const_cast<dh2_matrix*>(Mc);
  return mode_f32(M->mode) ? run_error<float>(M, G_ref, ref_dtype, ld, which, (cudaStream_t)stream, rel_err)
                           : run_error<double>(M, G_ref, ref_dtype, ld, which, (cudaStream_t)stream, rel_err);
}

dh2_status dh2_matrix_ranks(const dh2_matrix* M, int32_t side, int32_t* ranks) {
  if (!M || (side != 0 && side != 1)) return DH2_EINVAL;
  const int64_t np = M->tree->tr.dev->npairs[side];
  if (np == 0) return DH2_OK;  // no pairs on this side (no admissible block): nothing to write
  if (!ranks) return DH2_EINVAL;
  DH2_CUDA_TRY(cudaMemcpyAsync(ranks, M->rank[side], 4 * np, cudaMemcpyDeviceToHost, M->stream));
  DH2_CUDA_TRY(cudaStreamSynchronize(M->stream));
  return DH2_OK;
}

dh2_status dh2_matrix_sigma(const dh2_matrix* M, int32_t side, int64_t pair, double* out, int32_t cap,
                            int32_t* count) {
  if (!M || !out || (side != 0 && side != 1)) return DH2_EINVAL;
  const Tree& tr = M->tree->tr;
  if (pair < 0 || pair >= (int64_t)tr.side[side].pairs.size()) return DH2_EINVAL;
  DH2_CUDA_TRY(cudaStreamSynchronize(M->stream));
  double buf[kSigStride];
  DH2_CUDA_TRY(cudaMemcpy(buf, M->sig[side] + pair * kSigStride, sizeof(buf), cudaMemcpyDeviceToHost));
  const int32_t resolved = (int32_t)buf[kSigValues];
  const int32_t c = std::max(0, std::min(resolved, std::min(cap, kSigValues)));
  std::memcpy(out, buf, 8 * (size_t)c);
  if (count) *count = resolved;
  return DH2_OK;
}

dh2_status dh2_matrix_sigma_rest(const dh2_matrix* M, int32_t side, int64_t pair, double* energy) {
  if (!M || !energy || (side != 0 && side != 1)) return DH2_EINVAL;
  const Tree& tr = M->tree->tr;
  if (pair < 0 || pair >= (int64_t)tr.side[side].pairs.size()) return DH2_EINVAL;
  DH2_CUDA_TRY(cudaStreamSynchronize(M->stream));
  DH2_CUDA_TRY(cudaMemcpy(energy, M->sig[side] + pair * kSigStride + kSigValues + 1, 8, cudaMemcpyDeviceToHost));
  return DH2_OK;
}

namespace {
dh2_status copy_complex_to_host(const void* src, size_t es, int64_t rows, int64_t cols, int64_t ld, double* out) {
  std::vector<double> tmp((size_t)(2 * std::max<int64_t>(1, ld * cols)));
  if (rows * cols == 0) return DH2_OK;
  if (cudaMemcpy(tmp.data(), src, es * (size_t)(ld * (cols - 1) + rows), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return DH2_ECUDA;
  }
  for (int64_t j = 0; j < cols; ++j)
    for (int64_t i = 0; i < rows; ++i) {
      const int64_t s = i + j * ld;
      if (es == 16) {
        out[2 * (i + j * rows)] = tmp[2 * s];
        out[2 * (i + j * rows) + 1] = tmp[2 * s + 1];
      } else {
        const float* f = (const float*)tmp.data();
        out[2 * (i + j * rows)] = f[2 * s];
        out[2 * (i + j * rows) + 1] = f[2 * s + 1];
      }
    }
  return DH2_OK;
}
}  // namespace

dh2_status dh2_matrix_pair_basis(const dh2_matrix* M, int32_t side, int64_t pair, double* out, int64_t cap_elems,
                                 int32_t* rows, int32_t* k) {
  if (!M || !out || !rows || !k || (side != 0 && side != 1)) return DH2_EINVAL;
  const Tree& tr = M->tree->tr;
  if (pair < 0 || pair >= (int64_t)tr.side[side].pairs.size()) return DH2_EINVAL;
  DH2_CUDA_TRY(cudaStreamSynchronize(M->stream));
  const Pair& P = tr.side[side].pairs[pair];
  int32_t kk = 0;
  DH2_CUDA_TRY(cudaMemcpy(&kk, M->rank[side] + pair, 4, cudaMemcpyDeviceToHost));
  int32_t r = 0;
  if (P.leaf) {
    r = tr.size[P.cluster];
  } else {
    int32_t k2[2];
    for (int j = 0; j < 2; ++j)
      DH2_CUDA_TRY(cudaMemcpy(&k2[j], M->rank[side] + P.son_pair[j], 4, cudaMemcpyDeviceToHost));
    r = k2[0] + k2[1];
  }
  *rows = r;
  *k = kk;
  if ((int64_t)r * kk > cap_elems) return DH2_EINVAL;
  const Tree::Dev* D = tr.dev;
  const char* src = (const char*)M->Q[side] + M->es * D->Qoff_h[side][pair];
  return copy_complex_to_host(src, M->es, r, kk, D->rowcap_h[side][pair], out);
}

dh2_status dh2_matrix_coupling(const dh2_matrix* M, int64_t block, double* out, int64_t cap_elems, int32_t* kt,
                               int32_t* ks) {
  if (!M || !out || !kt || !ks) return DH2_EINVAL;
  const Tree& tr = M->tree->tr;
  if (block < 0 || block >= (int64_t)tr.blocks.size() || !tr.blocks[block].adm) return DH2_EINVAL;
  DH2_CUDA_TRY(cudaStreamSynchronize(M->stream));
  int32_t a = 0, b = 0;
  DH2_CUDA_TRY(cudaMemcpy(&a, M->rank[0] + tr.side[0].block_pair[block], 4, cudaMemcpyDeviceToHost));
  DH2_CUDA_TRY(cudaMemcpy(&b, M->rank[1] + tr.side[1].block_pair[block], 4, cudaMemcpyDeviceToHost));
  *kt = a;
  *ks = b;
  if ((int64_t)a * b > cap_elems) return DH2_EINVAL;
  const char* src = (const char*)M->S + M->es * tr.dev->Soff_h[block];
  return copy_complex_to_host(src, M->es, a, b, a, out);
}

dh2_status dh2_storage(const dh2_matrix* M, double* total, double* parts) {
  if (!M || !total) return DH2_EINVAL;
  const Tree& tr = M->tree->tr;
  std::vector<int32_t> rk[2];
  for (int sd = 0; sd < 2; ++sd) {
    rk[sd].resize(tr.side[sd].pairs.size());
    const dh2_status s = dh2_matrix_ranks(M, sd, rk[sd].data());
    if (s != DH2_OK) return s;
  }
  double pr[6] = {0, 0, 0, 0, 0, 0};
  for (int sd = 0; sd < 2; ++sd)
    for (size_t p = 0; p < tr.side[sd].pairs.size(); ++p) {
      const Pair& P = tr.side[sd].pairs[p];
      if (P.leaf) pr[sd] += (double)tr.size[P.cluster] * rk[sd][p];
      else pr[2 + sd] += (double)(rk[sd][P.son_pair[0]] + rk[sd][P.son_pair[1]]) * rk[sd][p];
    }
  for (size_t b = 0; b < tr.blocks.size(); ++b) {
    const Block& B = tr.blocks[b];
    if (B.adm) pr[4] += (double)rk[0][tr.side[0].block_pair[b]] * rk[1][tr.side[1].block_pair[b]];
    else pr[5] += (double)tr.size[B.t] * tr.size[B.s];
  }
  double s = 0;
  for (int i = 0; i < 6; ++i) {
    s += pr[i];
    if (parts) parts[i] = pr[i];
  }
  *total = s;
  return DH2_OK;
}

dh2_status dh2_matrix_launch_count(const dh2_matrix* M, int32_t* launches) {
  if (!M || !launches) return DH2_EINVAL;
  *launches = M->launches;
  return DH2_OK;
}

dh2_status dh2_debug_fail_alloc(int32_t nth) {
  if (nth < 0) return DH2_EINVAL;
  g_fail_alloc.store(nth);
  return DH2_OK;
}

dh2_status dh2_matrix_block_weights(const dh2_matrix* M, double* invw) {
  if (!M || !invw) return DH2_EINVAL;
  const size_t nb = M->tree->tr.blocks.size();
  DH2_CUDA_TRY(cudaStreamSynchronize(M->stream));
  if (nb) DH2_CUDA_TRY(cudaMemcpy(invw, M->invw, 8 * nb, cudaMemcpyDeviceToHost));
  return DH2_OK;
}

dh2_status dh2_matrix_leaf_gram(const dh2_matrix* M, int32_t side, int64_t pair, double* out, int64_t cap_elems,
                                int32_t* m) {
  if (!M || !out || !m || (side != 0 && side != 1) || !M->gram) return DH2_EINVAL;
  const Tree& tr = M->tree->tr;
  if (pair < 0 || pair >= (int64_t)tr.side[side].pairs.size() || !tr.side[side].pairs[pair].leaf) return DH2_EINVAL;
  const int mm = tr.size[tr.side[side].pairs[pair].cluster];
  const int mp = (mm + 7) & ~7;
  *m = mm;
  if ((int64_t)mm * mm > cap_elems) return DH2_EINVAL;
  // the pair's offset: recomputed as at upload (leaf pairs in order, mp^2 each, row side first)
  int64_t off = 0;
  for (int sd = 0; sd <= side; ++sd)
    for (int64_t p = 0; p < (int64_t)tr.side[sd].pairs.size(); ++p) {
      if (sd == side && p == pair) break;
      const Pair& P = tr.side[sd].pairs[p];
      if (P.leaf) {
        const int64_t q = (tr.size[P.cluster] + 7) & ~7;
        off += q * q;
      }
    }
  std::vector<float4> h((size_t)mp * mp);
  DH2_CUDA_TRY(cudaStreamSynchronize(M->stream));
  DH2_CUDA_TRY(cudaMemcpy(h.data(), (const float4*)M->gram + off, sizeof(float4) * h.size(), cudaMemcpyDeviceToHost));
  for (int j = 0; j < mm; ++j)
    for (int i = 0; i < mm; ++i) {
      const float4 v = h[i + (size_t)j * mp];
      out[2 * (i + (int64_t)j * mm)] = (double)v.x + (double)v.y;
      out[2 * (i + (int64_t)j * mm) + 1] = (double)v.z + (double)v.w;
    }
  return DH2_OK;
}

dh2_status dh2_matrix_class_launches(const dh2_matrix* M, int32_t* counts) {
  if (!M || !counts) return DH2_EINVAL;
  std::memcpy(counts, M->class_launches, sizeof(M->class_launches));
  return DH2_OK;
}

dh2_status dh2_matrix_leaf_split_ms(const dh2_matrix* M, float* ms2) {
  if (!M || !ms2) return DH2_EINVAL;
  ms2[0] = M->leaf_split_ms[0];
  ms2[1] = M->leaf_split_ms[1];
  return DH2_OK;
}

dh2_status dh2_matrix_phase_ms(const dh2_matrix* M, float* ms6) {
  if (!M || !ms6) return DH2_EINVAL;
  for (int i = 0; i < 6; ++i) ms6[i] = M->phase_ms[i];
  return DH2_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- matvec without allocation
//
// dh2_matvec allocates its coefficient vectors (the forward-transformed x and
// the coupled y, one small vector per (cluster, direction) pair) from the
// stream-ordered pool on every call.  The variant below takes them from one
// fixed device array instead, so that a caller that may not allocate device
// memory at all can still apply a compressed matrix.
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // 8 MiB, held by every device that loads the library
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {};

// Device address of the scratch array for the current device; looked up once
// per device (the array's host-side name is not a device address).
dh2_status noalloc_scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (dev < 0 || dev >= 64) return DH2_EUNSUPPORTED;
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return DH2_ECUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return DH2_OK;
}

template <typename T>
dh2_status run_matvec_noalloc(const dh2_matrix* M, const void* xv, void* yv, int nrhs, cudaStream_t st) {
  Tree& tr = M->tree->tr;
  Tree::Dev* D = tr.dev;
  const int64_t n = tr.n;
  const size_t hx = align256(sizeof(C2<T>) * D->h_elems[1] * nrhs);
  const size_t hy = align256(sizeof(C2<T>) * D->h_elems[0] * nrhs);
  if (hx + hy > kNoAllocScratchBytes) return DH2_EUNSUPPORTED;
  int dev = -1;
  DH2_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != M->device) return DH2_EINVAL;
  void* buf = nullptr;
  {
    const dh2_status s = noalloc_scratch_address(dev, &buf);
    if (s != DH2_OK) return s;
  }
  // every coefficient is written before it is read (forward transformation,
  // then coupling), so nothing in the scratch array needs clearing
  C2<T>* xh = (C2<T>*)buf;
  C2<T>* yh = (C2<T>*)((char*)buf + hx);
  const C2<T>* x = (const C2<T>*)xv;
  C2<T>* y = (C2<T>*)yv;
  DH2_CUDA_TRY(cudaMemsetAsync(y, 0, sizeof(C2<T>) * n * nrhs, st));
  SideView<T> Vv = side_view<T>(tr, M, 0), Wv = side_view<T>(tr, M, 1);
  launch_mv_forward_leaf<T>(Wv, D->leaf_list[1], (int)D->nleaf[1], x, nrhs, n, xh, D->hoff[1], st);
  for (int l = tr.depth; l >= 0; --l) {
    const int64_t b = D->lvl_nl_begin[1][l], e = D->lvl_end[1][l];
    if (e > b) launch_mv_forward_up<T>(Wv, D->iota[1] + b, (int)(e - b), nrhs, xh, D->hoff[1], st);
  }
  MvArgs<T> a;
  a.V = Vv;
  a.W = Wv;
  a.S = (const C2<T>*)M->S;
  a.Soff = D->Soff;
  a.own_ptr = D->own_ptr;
  a.own_blk = D->own_blk;
  a.bpair_col = D->bpair[1];
  a.xh = xh;
  a.xhoff = D->hoff[1];
  a.yh = yh;
  a.yhoff = D->hoff[0];
  a.par_ptr = D->par_ptr;
  a.par_pair = D->par_pair;
  a.par_son = D->par_son;
  a.bt = D->bt;
  a.bs = D->bs;
  a.near = (const C2<T>*)M->near;
  a.near_off = D->near_off;
  a.G = (const C2<T>*)M->G;
  a.ld = M->ld;
  launch_mv_coupling<T>(a, (int)D->npairs[0], nrhs, st);
  for (int l = 1; l <= tr.depth; ++l) {
    const int64_t b = D->lvl_begin[0][l], e = D->lvl_end[0][l];
    if (e > b) launch_mv_backward_down<T>(a, D->iota[0] + b, (int)(e - b), nrhs, st);
  }
  launch_mv_backward_leaf<T>(a, D->leaf_list[0], (int)D->nleaf[0], nrhs, y, n, st);
  launch_mv_near<T>(a, D->inadm_list, (int)D->ninadm, nrhs, x, y, n, st);
  DH2_CUDA_TRY(cudaGetLastError());
  return DH2_OK;
}

}  // namespace

extern "C" dh2_status dh2_matvec_noalloc(const dh2_matrix* M, const void* x, void* y, int32_t nrhs, void* stream) {
  if (!M || !x || !y || nrhs < 1) return DH2_EINVAL;
  return mode_f32(M->mode) ? run_matvec_noalloc<float>(M, x, y, nrhs, (cudaStream_t)stream)
                                  : run_matvec_noalloc<double>(M, x, y, nrhs, (cudaStream_t)stream);
}
