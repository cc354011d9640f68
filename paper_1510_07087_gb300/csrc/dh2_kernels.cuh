// Device-side types and kernel entry points of the compression library.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace dh2 {

template <typename T>
struct __align__(2 * sizeof(T)) C2 {
  T re, im;
};

// Arguments of the per-pair factorisation kernel (one CTA per (cluster,
// direction) pair).  Index [side] selects the row (0) or column (1) basis.
// Launch choices the autotuner sets (the public dh2_tuning, validated): one
// table per process, read when a compression prepares its launches.
struct TuneTable {
  int32_t jacobi_tpp[5];     // factor classes (<= 32, 40, 48, 64 rows, more): most threads per Jacobi column pair
  int32_t jacobi_narrow[4];  // mixed mode leaf classes: Jacobi CTAs of ~4 (0), ~2 (1) or ~1 (2) x rows threads
  int32_t rq_ctas_per_sm;    // leaf R kernel: resident CTAs per SM (0: its occupancy limit)
  int32_t rq_tensor;         // mixed mode: leaf R on the tensor cores (1) or the FP32 pipes (0)
  int32_t level_seg_cols;    // non-leaf pairs wider than twice this: factored by column segments (0: never)
};
TuneTable tune_current();
// factor class of a pair kernel compiled for P_T rows
__host__ __device__ constexpr int factor_class(int P_T) {
  return P_T <= 32 ? 0 : P_T <= 40 ? 1 : P_T <= 48 ? 2 : P_T <= 64 ? 3 : 4;
}

template <typename T>
struct PairArgs {
  const int32_t* start[2];            // first row index of the pair's cluster
  const int32_t* m[2];                // leaf rows (cluster size)
  const int32_t* ncols[2];            // #F_tc
  const int64_t* cmoff[2];            // leaf column-map offsets
  const int32_t* gcol[2];             // leaf column map: index of G's other dimension
  const int32_t* gblk[2];             // leaf column map: block id
  const T* colw[2];                   // leaf column map: weight 1/omega of the column's block
  const int32_t* son[2];              // non-leaf: 2 son pairs
  const int32_t* sonoff[2];           // non-leaf: column offsets in the son pairs
  const int32_t* level[2];
  const int32_t* kcap[2];             // rank capacity = leading dimension of R
  const int32_t* rowcap[2];           // leading dimension of the stored Q / [E1;E2]
  const int64_t* Roff[2];
  const int64_t* Qoff[2];
  const C2<T>* G;
  int64_t ld;
  const double* invw;                 // per block 1/omega_b
  C2<T>* R[2];
  C2<T>* Q[2];
  double* sig[2];                     // per pair P values (descending)
  int32_t* rank[2];
  const double* eps2;                 // per level eps_l^2
  const float4* H;                    // mixed modes: leaf Gram matrices (see GramArgs)
  float4* L4;                         // mixed modes: leaf Cholesky factors, pair at L4 + its Gram offset (FP32 complex, ld p)
  const int64_t* hoff[2];             // mixed modes: per pair, first entry of its Gram matrix in H
  const int32_t* rank_ovr[2];         // per pair a rank replacing the truncation rule (< 0: the rule), or NULL
  int32_t max_sweeps;
  int32_t jacobi_tpp[5];              // per factor class: most threads per Jacobi column pair (TuneTable)
  // non-leaf pairs factored by column segments: per pair the first entry of
  // its segments' factors in seg_buf (p x p each, ld p, one after the other),
  // -1 if not split; seg_cols columns per segment
  const int64_t* seg_off[2];
  C2<T>* seg_buf;
  int32_t seg_cols;
  uint32_t* status;
  // matrix-free mode: entries generated from points (permuted order, 3 doubles
  // each) and, for the double layer, their normals (NULL for the single layer)
  const double* pts;
  const double* nrm;
  double kappa;
  double diag;
  int32_t gen;
};

// Entry G_ij generated from the points, with `diag` on the diagonal:
//  - nrm == NULL: the Helmholtz single layer of Eq. (helmholtz),
//    exp(i kappa r) / (4 pi r), r = |x_i - x_j|;
//  - otherwise the double layer of Section 7 ("DLP matrix"),
//    (1 - i kappa r) exp(i kappa r) / (4 pi r^3) <x_i - x_j, n(x_j)>, with
//    nrm the unit normals (3 doubles per point, same order as pts).
// Distances, <x_i - x_j, n_j> and the phase reduction are formed in FP64; the
// FP32 variant evaluates sin/cos of the reduced phase (|phase| <= pi) in FP32.
template <typename T>
__device__ __forceinline__ C2<T> kernel_entry(const double* pts, const double* nrm, int64_t i, int64_t j,
                                              double kappa, double diag) {
  if (i == j) return C2<T>{(T)diag, T(0)};
  const double dx = pts[3 * i] - pts[3 * j];
  const double dy = pts[3 * i + 1] - pts[3 * j + 1];
  const double dz = pts[3 * i + 2] - pts[3 * j + 2];
  const double r = sqrt(dx * dx + dy * dy + dz * dz);
  // single layer: scale 1/(4 pi r); double layer: <x_i - x_j, n_j>/(4 pi r^3)
  // times (1 - i kappa r)
  double scale;
  double kr = 0.0;
  if (nrm) {
    const double dn = dx * nrm[3 * j] + dy * nrm[3 * j + 1] + dz * nrm[3 * j + 2];
    scale = dn / (12.566370614359172 * r * r * r);
    kr = kappa * r;
  } else {
    scale = 1.0 / (12.566370614359172 * r);
  }
  if (sizeof(T) == 8) {
    double sn, cs;
    sincos(kappa * r, &sn, &cs);
    // (cs + i sn)(1 - i kr) = cs + kr sn + i (sn - kr cs)
    return C2<T>{(T)((cs + kr * sn) * scale), (T)((sn - kr * cs) * scale)};
  } else {
    double th = kappa * r * 0.31830988618379067;  // phase / pi
    th -= 2.0 * rint(0.5 * th);                    // reduced to [-1, 1]
    float sn, cs;
    sincospif((float)th, &sn, &cs);
    const float krf = (float)kr, sc = (float)scale;
    return C2<T>{(T)((cs + krf * sn) * sc), (T)((sn - krf * cs) * sc)};
  }
}

// One CTA per launch code: args_dev holds one PairArgs per problem (device
// memory); P is the row capacity of the shared-memory factor (even).  With
// `count` (device int) the launch is sized at capacity nblocks and CTAs at or
// past *count return at once, so a list whose length is known only on the
// device needs no read-back.  Returns false, launching nothing, if the shared
// memory the launch needs exceeds the device's per-block limit.  With `segs`
// (non-leaf pairs only; codes unused) each CTA takes an entry code << 32 |
// segment and forms that column segment's LQ factor into the pair's slot of
// the segment buffer.
template <typename T>
bool launch_pair_kernel(const PairArgs<T>* args_dev, const uint32_t* codes, int nblocks, int P, bool from_r,
                        cudaStream_t st, const int* count = nullptr, const uint64_t* segs = nullptr);

// The leaf factorisation of the mixed modes: the pair kernel with steps 1
// and 1b replaced by the pivoted Cholesky of the leaf's Gram matrix H
// (launch_gram before it); leaves of at most 64 rows.
bool launch_pair_kernel_gram(const PairArgs<float>* args_dev, const uint32_t* codes, int nblocks, int P,
                             cudaStream_t st);

// R = Q^* A for the pairs of a pair-kernel launch, after it, by tiles of 32
// columns, tiles[i] = launch code << 32 | first column (P as for the pair
// kernel).  Leaf tiles of a stored G (gen false) go to a persistent kernel
// that keeps the next tile's loads in flight; the others get one CTA per tile.
template <typename T>
bool launch_rq_kernel(const PairArgs<T>* args_dev, const uint64_t* tiles, int ntiles, int P, bool from_r, bool gen,
                      cudaStream_t st);

// Non-leaf codes of one level split by the row count of their Ghat (from the
// sons' ranks): out = 4 segments of n codes, counts[4] zeroed by the caller.
template <typename T>
void launch_classify(const PairArgs<T>* args_dev, const uint32_t* codes, int n, uint32_t* out, int* counts,
                     cudaStream_t st);
// the same for segment entries (code << 32 | segment)
template <typename T>
void launch_classify_seg(const PairArgs<T>* args_dev, const uint64_t* segs, int n, uint64_t* out, int* counts,
                         cudaStream_t st);

// Arguments of the leaf Gram kernel of the mixed modes (one per problem).
// Index [side] selects the row (0) or column (1) basis.
struct GramArgs {
  const int32_t* start[2];   // first row index of the pair's cluster
  const int32_t* m[2];       // leaf rows
  const int32_t* ncols[2];   // #F_tc
  const int64_t* cmoff[2];   // leaf column-map offsets
  const int32_t* gcol[2];    // leaf column map: index of G's other dimension
  const float* colw[2];      // leaf column map: weight 1/omega of the column's block
  const int64_t* hoff[2];    // per pair: first entry of its Gram in H (mp x mp, mp = m rounded up to 8)
  const int64_t* seg_begin[2];  // per pair: its blocks of F_tc as a range of column-map segments
  const int32_t* seg_blk[2];    // per segment: block id
  const int32_t* bt;         // per block: row cluster
  const int32_t* bs;         // per block: column cluster
  const int32_t* cstart;     // per cluster: first index
  const int32_t* csize;      // per cluster: size
  const double* invw;        // per block: 1/omega_b
  const float* bmax;         // per admissible block: largest |re|, |im| per row, then per column
  const int64_t* bmax_off;
  const C2<float>* G;
  int64_t ld;
  float4* H;                 // Gram matrices: (re hi, re lo, im hi, im lo) double-float, column-major, ld mp
  uint32_t* status;
  uint32_t spin_limit;       // polls of a wait for a tensor-core batch (0: default)
};
// Columns of one exact accumulation window of the Gram kernel.
constexpr int kGramWindow = 448;

// H = A A^* for the leaf pairs of a launch list (leaves of at most maxm <= 64
// rows) on the tensor cores; false if the launch cannot run.
bool launch_gram(const GramArgs* args_dev, const uint32_t* codes, int n, int maxm, cudaStream_t st);

// R = Q^* A of the mixed mode's leaf pairs on the tensor cores, over a list of
// R tiles of kRTile columns (all leaf classes; a 128-column tile starts at
// every entry whose first column is a multiple of 128); false if it cannot run.
bool launch_rq_tc(const PairArgs<float>* args_dev, const uint64_t* tiles, int64_t ntiles, uint32_t spin_limit,
                  cudaStream_t st);

// Phase cycle counters of the pair kernel (only with -DDH2_PROFILE); 17 values.
void prof_reset_pair();
bool prof_read_pair(unsigned long long* out17);
// Phase cycle counters of the Gram kernels (only with -DDH2_PROFILE): 10
// values of the one-stage form, then 12 of the pipelined form.
void prof_reset_gram();
bool prof_read_gram(unsigned long long* out22);

}  // namespace dh2
