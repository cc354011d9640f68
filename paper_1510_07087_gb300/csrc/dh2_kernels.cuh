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
template <typename T>
struct PairArgs {
  const int32_t* order;               // (side << 30) | pair, launch order
  const int32_t* start[2];            // first row index of the pair's cluster
  const int32_t* m[2];                // leaf rows (cluster size)
  const int32_t* ncols[2];            // #F_tc
  const int64_t* cmoff[2];            // leaf column-map offsets
  const int32_t* gcol[2];             // leaf column map: index of G's other dimension
  const int32_t* gblk[2];             // leaf column map: block id (weight)
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
  int32_t P;                          // rows of the shared-memory factor (even)
  int32_t max_sweeps;
  uint32_t* status;
};

template <typename T>
void launch_pair_kernel(const PairArgs<T>& a, int nblocks, bool from_r, cudaStream_t st);

// Phase cycle counters of the pair kernel (only with -DDH2_PROFILE).
void prof_reset_pair();
bool prof_read_pair(unsigned long long* out8);

}  // namespace dh2
