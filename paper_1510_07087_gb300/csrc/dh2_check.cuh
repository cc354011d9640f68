// Optional device-side bounds checks (compiled in with -DDH2_CHECK).  A failed
// check records where it happened and skips the access; the host reads the
// record after the launch sequence.  Without DH2_CHECK every check is `true`.
#pragma once

#include <cstdint>

namespace dh2 {

struct CheckLimits {
  int64_t G, R[2], Q[2], X[2], S, near, nblocks, npairs[2], ncol[2], seg;
};

struct CheckRecord {
  int32_t count;
  int32_t where;
  int32_t item;
  int32_t pad;
  int64_t index;
  int64_t limit;
};

// one setter / reader per translation unit (each holds its own copies)
void check_set_limits_pair(const CheckLimits& l);
void check_set_limits_ops(const CheckLimits& l);
bool check_read_pair(CheckRecord* out);
bool check_read_ops(CheckRecord* out);

}  // namespace dh2

#ifdef DH2_CHECK
#define DH2_CHECK_DECLS                                                                        \
  __constant__ dh2::CheckLimits c_lim;                                                         \
  __device__ dh2::CheckRecord g_chk;                                                           \
  __device__ __noinline__ bool dh2_in(int64_t idx, int64_t lim, int where, int item) {         \
    if (idx >= 0 && idx < lim) return true;                                                    \
    if (atomicAdd(&g_chk.count, 1) == 0) {                                                     \
      g_chk.where = where;                                                                     \
      g_chk.item = item;                                                                       \
      g_chk.index = idx;                                                                       \
      g_chk.limit = lim;                                                                       \
    }                                                                                          \
    return false;                                                                              \
  }
#define DH2_IN(idx, lim, where, item) dh2_in((int64_t)(idx), (int64_t)(lim), (where), (item))
#else
#define DH2_CHECK_DECLS
#define DH2_IN(idx, lim, where, item) true
#endif
