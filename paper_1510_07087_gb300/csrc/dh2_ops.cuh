// Argument structures of the kernels around the per-pair factorisation.
#pragma once

#include "dh2_kernels.cuh"

namespace dh2 {

// Device view of one side's pairs and outputs.
template <typename T>
struct SideView {
  const int32_t* cluster;  // per pair
  const int32_t* leaf;     // per pair
  const int32_t* son;      // 2 per pair
  const int32_t* rowcap;   // per pair, ld of stored Q / [E1;E2]
  const int32_t* kcap;     // per pair, ld of R
  const int64_t* Roff;
  const int64_t* Qoff;
  const int64_t* Xoff;     // expansion buffer offsets (non-leaf pairs)
  const int32_t* cstart;   // per cluster
  const int32_t* csize;    // per cluster
  const int32_t* rank;     // per pair
  int side;
  C2<T>* R;
  C2<T>* Q;
  C2<T>* X;
};

template <typename T>
struct NormsArgs {
  const C2<T>* G;
  int64_t ld;
  const int32_t* bt;
  const int32_t* bs;
  const int32_t* badm;
  const int32_t* cstart;
  const int32_t* csize;
  const int32_t* clevel;
  const double* zpow;      // zeta^-level
  double* invw;            // per block 1/omega_b
  C2<T>* near;
  const int64_t* near_off;
  int copy;
  const double* pts;  // matrix-free mode
  const double* nrm;  // matrix-free double layer: normals (NULL: single layer)
  double kappa;
  double diag;
  int gen;
  // mixed modes: per admissible block the largest |re|, |im| of each of its
  // rows, then of each of its columns (bmax + bmax_off[b]); NULL otherwise
  float* bmax;
  const int64_t* bmax_off;
  double* bnorm2;  // per block |G_b|_F^2 of the admissible blocks (closed-form error)
};

template <typename T>
struct ProjArgs {
  SideView<T> V, W;
  const int32_t* adm_list;
  const int32_t* bpair_row;
  const int32_t* bpair_col;
  const int32_t* boff_row;
  const int32_t* bs;
  const int32_t* csize;
  const double* invw;
  C2<T>* S;
  const int64_t* Soff;
};

template <typename T>
struct MvArgs {
  SideView<T> V, W;
  const C2<T>* S;
  const int64_t* Soff;
  const int64_t* own_ptr;   // row pairs: own blocks (CSR)
  const int32_t* own_blk;
  const int32_t* bpair_col;
  const C2<T>* xh;
  const int64_t* xhoff;     // column pairs
  C2<T>* yh;
  const int64_t* yhoff;     // row pairs
  const int64_t* par_ptr;   // row pairs: father pairs (CSR)
  const int32_t* par_pair;
  const int32_t* par_son;
  const int32_t* bt;
  const int32_t* bs;
  const C2<T>* near;
  const int64_t* near_off;
  const C2<T>* G;
  int64_t ld;
};

template <typename T>
struct ErrArgs {
  SideView<T> V, W;
  const C2<T>* S;
  const int64_t* Soff;
  const int32_t* bt;
  const int32_t* bs;
  const int32_t* badm;
  const int32_t* bpair_row;
  const int32_t* bpair_col;
  const int32_t* cstart;
  const int32_t* csize;
  const C2<T>* near;
  const int64_t* near_off;
  const C2<T>* G;
  int64_t ld;
  const double* pts;  // reference generated from points (FP64) when ref_gen
  const double* nrm;  // and normals for the double layer (NULL: single layer)
  double kappa;
  double diag;
  int ref_gen;
};

// Leaf column maps (global column, block id) from their segments (dst, first
// column, width, block)
void launch_colmap_expand(const int64_t* dst, const int32_t* col0, const int32_t* w, const int32_t* blk, int64_t nseg,
                          int32_t* gcol, int32_t* gblk, cudaStream_t st);
// colw[j] = 1/omega of the block of column j of a column map (n entries)
template <typename T>
void launch_colw(const int32_t* gblk, const double* invw, T* colw, int64_t n, cudaStream_t st);
// codes: (problem << 26) | block for a batch, or NULL for blocks 0..n-1 of args_dev[0]
template <typename T>
void launch_norms_near(const NormsArgs<T>* args_dev, const uint32_t* codes, int n, cudaStream_t st);
// admissible blocks of a stored G in pieces (code << 32 | 32-row slab << 16 |
// kNormCols-column group; block i's pieces are pbegin[i] .. pbegin[i+1] - 1):
// partial sums per piece (scratch `partial`, npieces doubles), in the mixed modes
// the row/column maxima (zeroed before) merged atomically, then bnorm2 and the
// weights of the nblocks codes
template <typename T>
void launch_norms_adm(const NormsArgs<T>* args_dev, const uint64_t* pieces, int64_t npieces, const uint32_t* codes,
                      const int64_t* pbegin, int64_t nblocks, double* partial, cudaStream_t st);
template <typename T> void launch_expand(const SideView<T>& S, const int32_t* pairs, int n, cudaStream_t st);
template <typename T> void launch_project(const ProjArgs<T>& a, int nadm, cudaStream_t st);
template <typename T>
void launch_mv_forward_leaf(const SideView<T>& W, const int32_t* pairs, int np, const C2<T>* x, int nrhs,
                            int64_t n, C2<T>* xh, const int64_t* hoff, cudaStream_t st);
template <typename T>
void launch_mv_forward_up(const SideView<T>& W, const int32_t* pairs, int np, int nrhs, C2<T>* xh,
                          const int64_t* hoff, cudaStream_t st);
template <typename T> void launch_mv_coupling(const MvArgs<T>& a, int npairs_row, int nrhs, cudaStream_t st);
template <typename T>
void launch_mv_backward_down(const MvArgs<T>& a, const int32_t* pairs, int np, int nrhs, cudaStream_t st);
template <typename T>
void launch_mv_backward_leaf(const MvArgs<T>& a, const int32_t* pairs, int np, int nrhs, C2<T>* y, int64_t n,
                             cudaStream_t st);
template <typename T>
void launch_mv_near(const MvArgs<T>& a, const int32_t* blocks, int nb, int nrhs, const C2<T>* x, C2<T>* y,
                    int64_t n, cudaStream_t st);
template <typename T, typename RT>
void launch_error(const ErrArgs<T>& a, const C2<RT>* Gref, int64_t ldr, int nblocks, double* acc,
                  cudaStream_t st);
// adjoint product: coupling with S_b^* into column pairs, nearfield with G_b^*
// (MvArgs with the sides exchanged: V = column basis, W = row basis, own and
// father lists of the column side, bpair_col = the blocks' row pairs)
template <typename T> void launch_mv_coupling_adj(const MvArgs<T>& a, int npairs_col, int nrhs, cudaStream_t st);
template <typename T>
void launch_mv_near_adj(const MvArgs<T>& a, const int32_t* blocks, int nb, int nrhs, const C2<T>* x, C2<T>* y,
                        int64_t n, cudaStream_t st);
// y = G_ref x or G_ref^* x in FP64 (G NULL: entries generated from gen's points)
template <typename RT>
void launch_gemv(const C2<RT>* G, int64_t ld, const ErrArgs<float>& gen, int64_t n, bool trans, const C2<double>* x,
                 C2<double>* y, cudaStream_t st);
// acc[0] += sum_adm |G_b|^2 - |S_b|^2, acc[1] += sum_all |G_b|^2
template <typename T>
void launch_closed_form(const ErrArgs<T>& a, const double* bnorm2, int nblocks, double* acc, cudaStream_t st);
// o = (T) v; u -= t  (vectors of n complex entries)
template <typename T> void launch_to_type(const C2<double>* v, C2<T>* o, int64_t n, cudaStream_t st);
// *acc += |v|^2; v = w / sqrt(*n2) (device scalar; v may be w); a seeded vector with entries in [-1/2, 1/2)^2
void launch_norm2(const C2<double>* v, int64_t n, double* acc, cudaStream_t st);
void launch_normalize(C2<double>* v, const C2<double>* w, int64_t n, const double* n2, cudaStream_t st);
void launch_seed_vector(C2<double>* v, int64_t n, uint64_t seed, cudaStream_t st);
template <typename T> void launch_sub(C2<double>* u, const C2<T>* t, int64_t n, cudaStream_t st);

}  // namespace dh2
