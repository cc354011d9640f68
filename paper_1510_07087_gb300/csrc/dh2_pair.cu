// Per-(cluster, direction) factorisation kernel: the leaf step and the
// non-leaf step of procedure basis() (Section 6), one CTA per pair.
//
// For a pair (t, c) the kernel
//   1. streams the columns of its matrix A -- G^omega_tc restricted to the
//      rows of t for a leaf (Section 6 leaf step, weights of Remark "Error
//      control"), or Ghat_tc = [R_t1c'|F_tc ; R_t2c'|F_tc] for a non-leaf
//      (Eq. hatQ_hatG) -- in chunks of C columns held in registers (one row
//      of the chunk per group of LPR threads) and reduces it to a p x p
//      lower-triangular factor L with A = L Omega, Omega with orthonormal
//      rows: an LQ factorisation by Householder reflections applied chunk by
//      chunk, so the Gram matrix A A^* is never formed and singular values
//      are not squared;
//   2. runs one-sided (Hestenes) Jacobi on the columns of L held in shared
//      memory, one column pair per group of 8 threads and all pairs of a
//      round at once: L J = U Sigma, so the normalised columns are the left
//      singular vectors of A and their norms its singular values;
//   3. chooses the rank k = min{k : sum_{i>k} sigma_i^2 <= eps_l^2} with the
//      tail sums formed in FP64;
//   4. writes Q = first k left singular vectors (Q_tc for a leaf, the stacked
//      transfer matrices [E_t1c; E_t2c] for a non-leaf), the singular values
//      and k.
// rq_kernel then streams A once more to form R_tc = Q^* A (Section 6, R
// recursion) for all pairs of the launch at once.
#include <cfloat>
#include <cstdlib>
#include <type_traits>

#include "dh2_check.cuh"
#include "dh2_internal.h"
#include "dh2_kernels.cuh"

namespace dh2 {

namespace {

DH2_CHECK_DECLS

#ifdef DH2_PROFILE
// summed over CTAs: cycles of LQ, Jacobi, rank+Q, R; sweeps; pairs; p; K;
// cycles of the LQ staging; chunks; LQ steps; cycles from a step's start to
// the end of its own work, summed over the warps (10: the warp forming the
// next reflection, 11: all warps), and cycles to the formed reflection (13),
// split (14-16) into step start -> update of row i+1 -> its norm reduced ->
// reflection formed, as seen by the thread that forms it
__device__ unsigned long long g_prof[17];
#define DH2_PROF_T(v) const long long v = clock64()
#define DH2_PROF_ADD(i, v) \
  if (threadIdx.x == 0) atomicAdd(&g_prof[i], (unsigned long long)(v))
#define DH2_PROF_ON 1
#else
#define DH2_PROF_T(v)
#define DH2_PROF_ADD(i, v)
#define DH2_PROF_ON 0
#endif

template <typename T>
__device__ __forceinline__ C2<T> czero() { return C2<T>{T(0), T(0)}; }
template <typename T>
__device__ __forceinline__ C2<T> cadd(C2<T> a, C2<T> b) { return C2<T>{a.re + b.re, a.im + b.im}; }
template <typename T>
__device__ __forceinline__ C2<T> csub(C2<T> a, C2<T> b) { return C2<T>{a.re - b.re, a.im - b.im}; }
template <typename T>
__device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
  return C2<T>{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// a * conj(b)
template <typename T>
__device__ __forceinline__ C2<T> cmulc(C2<T> a, C2<T> b) {
  return C2<T>{a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im};
}
template <typename T>
__device__ __forceinline__ T cnorm2(C2<T> a) { return a.re * a.re + a.im * a.im; }
// Accumulating forms as fused multiply-adds (the compiler may not reassociate
// acc + (x*y + z*w) into them itself): acc + a conj(b), c - t x, acc + |a|^2.
template <typename T>
__device__ __forceinline__ C2<T> cmacc(C2<T> acc, C2<T> a, C2<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.im, b.re, acc.im);
  acc.im = fma(-a.re, b.im, acc.im);
  return acc;
}
// acc + a b, with the same fused multiply-adds in the same order as
// cmacc(acc, a, conj(b)) (the negations are exact), so either form of a
// product gives the same bits
template <typename T>
__device__ __forceinline__ C2<T> cmac_nc(C2<T> acc, C2<T> a, C2<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.im, b.re, acc.im);
  acc.im = fma(a.re, b.im, acc.im);
  return acc;
}
template <typename T>
__device__ __forceinline__ C2<T> cnmac(C2<T> c, C2<T> t, C2<T> x) {
  c.re = fma(-t.re, x.re, c.re);
  c.re = fma(t.im, x.im, c.re);
  c.im = fma(-t.re, x.im, c.im);
  c.im = fma(-t.im, x.re, c.im);
  return c;
}
template <typename T>
__device__ __forceinline__ T nmac(T acc, C2<T> a) {
  return fma(a.im, a.im, fma(a.re, a.re, acc));
}

template <typename T>
struct Eps;
// u: unit roundoff; tiny: squared norms below it are treated as zero (far
// below any weighted entry, and far enough above the underflow threshold that
// 1/tiny and the Householder scale factors stay finite).
template <>
struct Eps<float> {
  static constexpr float u = 5.9604645e-08f;
  static constexpr float tiny = 1e-30f;
};
template <>
struct Eps<double> {
  static constexpr double u = 1.1102230246251565e-16;
  static constexpr double tiny = 1e-280;
};

// Reciprocal square root and quotient for the rotation and reflector scalars:
// hardware approximations in FP32 (a few ulp; the rotations and reflections
// stay unitary to that level), correctly rounded in FP64.
__device__ __forceinline__ float frsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double frsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }

// Asynchronous global -> shared copies (cp.async): not held up by CTA
// barriers; completed by cp_async_wait_all in the issuing thread.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Two consecutive complex entries from a 16-byte aligned shared-memory
// address (one 16-byte load in FP32).
template <typename T>
__device__ __forceinline__ void load_c2x2(const C2<T>* p, C2<T>& a, C2<T>& b) {
  a = p[0];
  b = p[1];
}
template <>
__device__ __forceinline__ void load_c2x2<float>(const C2<float>* p, C2<float>& a, C2<float>& b) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = C2<float>{v.x, v.y};
  b = C2<float>{v.z, v.w};
}

template <typename T>
__device__ __forceinline__ void store_c2x2(C2<T>* p, C2<T> a, C2<T> b) {
  p[0] = a;
  p[1] = b;
}
template <>
__device__ __forceinline__ void store_c2x2<float>(C2<float>* p, C2<float> a, C2<float> b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.re, a.im, b.re, b.im);
}

// Walk e = start, start + step, ... < slow_n * fast_n over a (slow, fast)
// index pair, e = slow * fast_n + fast, with one division at set-up.
struct Walk2 {
  int f, g, df, dg, fn;
  __device__ __forceinline__ Walk2(int start, int step, int fast_n)
      : f(start % fast_n), g(start / fast_n), df(step % fast_n), dg(step / fast_n), fn(fast_n) {}
  __device__ __forceinline__ void next() {
    f += df;
    g += dg;
    if (f >= fn) {
      f -= fn;
      ++g;
    }
  }
};

// Element (r, j) of the pair's matrix A (row r of the factor, column j of F_tc).
template <typename T, bool FROM_R>
struct Source {
  int side, pid;
  // leaf
  const C2<T>* G;
  int64_t ld;
  int r0;
  const int32_t* gcol;
  const T* colw;
  int64_t cmo;
  const double* pts;  // matrix-free mode
  const double* nrm;  // double layer: normals (NULL: single layer)
  double kappa, diag;
  int gen;
  // non-leaf
  const C2<T>* R0;
  const C2<T>* R1;
  int64_t roff0, roff1;
  int k1, off0, off1, ld0, ld1;
  bool segsrc = false;  // R0 is the segments' factors [L_1 ... L_S] (bounds of the segment buffer)

  // leaf: global column index and weight 1/omega_b of column j of F_tc
  __device__ __forceinline__ void colinfo(int j, int& gc, T& w) const {
    gc = 0;
    w = T(0);
    if (!DH2_IN(cmo + j, c_lim.ncol[side], 3, pid)) return;
    gc = gcol[j];
    w = colw[j];
  }
  // leaf: address of G's entry behind element (r, j) of A given column j's
  // global index gc (NULL if out of range: checked builds only)
  __device__ __forceinline__ const C2<T>* leaf_ptr(int r, int gc) const {
    const int64_t e = side == 0 ? (int64_t)gc * ld + r0 + r : (int64_t)(r0 + r) * ld + gc;
    if (!DH2_IN(e, c_lim.G, side == 0 ? 5 : 7, pid)) return nullptr;
    return G + e;
  }
  // non-leaf: address of element (r, j) of Ghat in the sons' R (NULL as above)
  __device__ __forceinline__ const C2<T>* sons_ptr(int r, int j) const {
    if (r < k1) {
      const int64_t e = (int64_t)(off0 + j) * ld0 + r;
      if (!DH2_IN(roff0 + e, segsrc ? c_lim.seg : c_lim.R[side], 1, pid)) return nullptr;
      return R0 + e;
    }
    const int64_t e = (int64_t)(off1 + j) * ld1 + (r - k1);
    if (!DH2_IN(roff1 + e, c_lim.R[side], 2, pid)) return nullptr;
    return R1 + e;
  }
  // leaf: element (r, j) given column j's global index gc and weight w
  __device__ __forceinline__ C2<T> leaf_at(int r, int gc, T w) const {
    if (gen) {
      C2<T> g = side == 0 ? kernel_entry<T>(pts, nrm, r0 + r, gc, kappa, diag)
                          : kernel_entry<T>(pts, nrm, gc, r0 + r, kappa, diag);
      return C2<T>{g.re * w, side == 0 ? g.im * w : -g.im * w};
    }
    if (side == 0) {
      const int64_t e = (int64_t)gc * ld + r0 + r;
      if (!DH2_IN(e, c_lim.G, 5, pid)) return czero<T>();
      const C2<T> g = G[e];
      return C2<T>{g.re * w, g.im * w};
    }
    // column basis: the same procedure on G^*; row r of A is column r0+r of G
    const int64_t e = (int64_t)(r0 + r) * ld + gc;
    if (!DH2_IN(e, c_lim.G, 7, pid)) return czero<T>();
    const C2<T> g = G[e];
    return C2<T>{g.re * w, -g.im * w};
  }

  __device__ __forceinline__ C2<T> get(int r, int j) const {
    if (FROM_R) {
      if (r < k1) {
        const int64_t e = (int64_t)(off0 + j) * ld0 + r;
        if (!DH2_IN(roff0 + e, segsrc ? c_lim.seg : c_lim.R[side], 1, pid)) return czero<T>();
        return R0[e];
      }
      const int64_t e = (int64_t)(off1 + j) * ld1 + (r - k1);
      if (!DH2_IN(roff1 + e, c_lim.R[side], 2, pid)) return czero<T>();
      return R1[e];
    } else {
      int gc;
      T w;
      colinfo(j, gc, w);
      return leaf_at(r, gc, w);
    }
  }
};

// Column table of columns j0 .. j0+cwid-1 of a leaf pair: global index and
// weight 1/omega_b (read first, so that the element loads do not wait on the
// column map).
template <typename T, bool FROM_R, int NT>
__device__ __forceinline__ void stage_table(const Source<T, FROM_R>& src, int j0, int cwid, int* cgc, T* cwt) {
  if (FROM_R) return;
  for (int jj = threadIdx.x; jj < cwid; jj += NT) {
    int gc;
    T w;
    src.colinfo(j0 + jj, gc, w);
    cgc[jj] = gc;
    cwt[jj] = w;
  }
}

// Columns j0 .. j0+ncols-1 of the pair's matrix A (zero from column cwid on)
// into dst, column jj at dst[jj * ld]: 8 loads in flight per thread,
// consecutive threads on the contiguous direction of the source (the rows of
// A for G and for the sons' R, the columns of A for G^*).  A leaf needs the
// column table of stage_table, visible to every thread.
template <typename T, bool FROM_R, int NT>
__device__ __forceinline__ void stage_cols(const Source<T, FROM_R>& src, int p, int j0, int cwid, int ncols,
                                           C2<T>* dst, int ld, const int* cgc, const T* cwt) {
  const int tid = threadIdx.x;
  const bool down = FROM_R || src.side == 0;
  const int tot = ncols * p;
  for (int e0 = 0; e0 < tot; e0 += 8 * NT) {
    C2<T> v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + tid + u * NT;
      const int r = down ? e % p : e / ncols;
      const int jj = down ? e / p : e % ncols;
      v[u] = czero<T>();
      if (e < tot && jj < cwid) v[u] = FROM_R ? src.get(r, j0 + jj) : src.leaf_at(r, cgc[jj], cwt[jj]);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + tid + u * NT;
      const int r = down ? e % p : e / ncols;
      const int jj = down ? e / p : e % ncols;
      if (e < tot) dst[jj * ld + r] = v[u];
    }
  }
}

// ---------------------------------------------------------------- double-float arithmetic
// A value hi + lo of two floats (|lo| <= ulp(hi)/2, about 48 significant
// bits), with the error-free sum of Knuth and the error-free product from a
// fused multiply-add (Dekker's double-length arithmetic in FP32 registers).
struct Df {
  float hi, lo;
};
__device__ __forceinline__ Df df_fast_sum(float s, float e) {  // |s| >= |e|
  const float h = s + e;
  return Df{h, e - (h - s)};
}
__device__ __forceinline__ Df df_add(Df x, Df y) {
  const float s = x.hi + y.hi;
  const float bb = s - x.hi;
  const float e = (x.hi - (s - bb)) + (y.hi - bb) + x.lo + y.lo;
  return df_fast_sum(s, e);
}
__device__ __forceinline__ Df df_neg(Df x) { return Df{-x.hi, -x.lo}; }
__device__ __forceinline__ Df df_mul(Df x, Df y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return df_fast_sum(p, e);
}
// one Newton step from the FP32 square root / reciprocal
__device__ __forceinline__ Df df_sqrt(Df x) {
  const float r = sqrtf(x.hi);
  const float p = r * r;
  const float e = fmaf(r, r, -p);
  const float d = ((x.hi - p) - e) + x.lo;  // x - r^2
  return df_fast_sum(r, d / (2.f * r));
}
__device__ __forceinline__ Df df_recip(Df x) {
  const float q = 1.f / x.hi;
  const Df xq = df_mul(x, Df{q, 0.f});
  const Df rest = df_add(Df{1.f, 0.f}, df_neg(xq));  // 1 - x q
  return df_fast_sum(q, rest.hi * q);
}
__device__ __forceinline__ Df df_shfl_xor(Df x, int o) {
  return Df{__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
}

// ---------------------------------------------------------------- 1'. pivoted Cholesky of a Gram matrix
// H = A A^* of a leaf pair from the tensor-core Gram kernel (double-float,
// column-major, ld mp = p rounded up to 8) is factored by left-looking
// Cholesky with diagonal pivoting in double-float arithmetic:
// H = L L^* + (Schur complement), stopping at the first K whose Schur
// complement has trace E_K <= tau (= drop eps_l^2).  Since L L^* = A A^*, the
// K columns of L span the same subspace, and E_K is the same energy, as the
// K leading columns of the row-pivoted LQ of A (steps 1 and 1b), so the
// Jacobi, rank and Q steps that follow are shared.  H is first scaled by an
// even power of two 2^s that brings its largest diagonal entry near 1 (exact;
// keeps the low halves of the products clear of underflow); L is scaled back
// by 2^(-s/2) as it is written to Lm in FP32, and E_K by 2^-s.
// Column j of L (double-float) replaces H's column of the j-th pivot, which is
// read only when that pivot is chosen; in FP32 it goes to Lg (global, ld p;
// the pair's Gram slot itself unless the Gram matrices are kept: H has been
// read into shared memory first).
// Rows: LPR threads per row.
template <typename T, int NT, int LPR>
__device__ void gram_cholesky(const PairArgs<T>& a, int side, int pid, int p, int P, int row, int q,
                              bool live, double tau, C2<T>* Lg, float4* Hs, float* dhi, float* dlo, int* piv,
                              int* pcol, int& K, double& E_K) {
  const int tid = threadIdx.x, lane = tid & 31;
  const int mp = (p + 7) & ~7;
  DH2_PROF_T(t_h0);
  const float4* Hin = a.H + a.hoff[side][pid];
  // the scale from the largest diagonal entry (warp 0), then H is read,
  // scaled (a power of two: exact) and stored in one pass that also fills the
  // Schur diagonal
  __shared__ int sh_se;
  if ((tid >> 5) == 0) {
    float hmax = 0.f;
    for (int r = lane; r < p; r += 32) hmax = fmaxf(hmax, Hin[r + (int64_t)r * mp].x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) hmax = fmaxf(hmax, __shfl_xor_sync(0xffffffffu, hmax, o));
    int eh = 0;
    if (hmax > 0.f) frexpf(hmax, &eh);
    if (lane == 0) sh_se = -2 * (eh >> 1);  // even
  }
  if (tid < p) pcol[tid] = -1;
  __syncthreads();
  const int se = sh_se;
  const float sc = ldexpf(1.f, se);  // 2^se, se in [-128, 126]: exact (subnormal at the low end)
#pragma unroll 4
  for (int idx = tid; idx < p * p; idx += NT) {
    const int r = idx % p, c = idx / p;
    const float4 h = __ldg(Hin + r + (int64_t)c * mp);
    const float4 hs = make_float4(h.x * sc, h.y * sc, h.z * sc, h.w * sc);
    Hs[r + c * P] = hs;
    if (r == c) {
      dhi[r] = hs.x;
      dlo[r] = hs.y;
    }
  }
  __syncthreads();
  // the stopping threshold in the scaled units, as a double-float (the loop
  // runs on the FP32 pipes only: GB300's FP64 pipe is narrow)
  const double tau_d = ldexp(tau, se);
  const Df tau_s{(float)tau_d, (float)(tau_d - (double)(float)tau_d)};
  const float back = ldexpf(1.f, -se / 2);
  DH2_PROF_T(t_h1);
  DH2_PROF_ADD(8, t_h1 - t_h0);  // H staged and scaled
#if DH2_PROF_ON
  long long pc_n = 0, pc_piv = 0, pc_col = 0;  // columns, cycles of the pivot searches and of the columns
#endif
  K = p;
  E_K = 0.0;
  __shared__ int sh_pv;
  __shared__ float sh_piv[4];  // sqrt(d_pv) and 1/sqrt(d_pv), double-float
  __shared__ double sh_e;
  for (int j = 0; j < p; ++j) {
#if DH2_PROF_ON
    ++pc_n;
#endif
    DH2_PROF_T(t_c0);
    // warp 0: Schur trace of the unchosen rows (double-float), the pivot
    // (largest diagonal, lowest row on ties) and its scalars; -1 = stop
    if ((tid >> 5) == 0) {
      Df e{0.f, 0.f};
      float best = -1.f;
      int pv = p;
      for (int r = lane; r < p; r += 32)
        if (pcol[r] < 0) {
          e = df_add(e, Df{dhi[r], dlo[r]});
          if (dhi[r] > best) {
            best = dhi[r];
            pv = r;
          }
        }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        e = df_add(e, df_shfl_xor(e, o));
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, pv, o);
        if (ob > best || (ob == best && oi < pv)) {
          best = ob;
          pv = oi;
        }
      }
      const Df gap = df_add(e, df_neg(tau_s));  // e - tau
      const bool stop = !(gap.hi > 0.f) || pv >= p || !(best > 0.f);
      if (lane == 0) {
        sh_pv = stop ? -1 : pv;
        sh_e = (double)e.hi + (double)e.lo;
        if (!stop) {
          const Df sq = df_sqrt(Df{dhi[pv], dlo[pv]});
          const Df inv = df_recip(sq);
          sh_piv[0] = sq.hi;
          sh_piv[1] = sq.lo;
          sh_piv[2] = inv.hi;
          sh_piv[3] = inv.lo;
        }
      }
    }
    __syncthreads();
    DH2_PROF_T(t_c1);
#if DH2_PROF_ON
    pc_piv += t_c1 - t_c0;  // pivot search and its broadcast
#endif
    const int pv = sh_pv;
    if (pv < 0) {
      K = j;
      // the Schur diagonal is formed by subtraction: a trace below zero is
      // rounding (|e| at most a few units of 2^-48 of the largest diagonal)
      const double ed = sh_e;
      E_K = ed != ed ? ed : ldexp(fmax(ed, 0.0), -se);
      break;
    }
    const Df sq{sh_piv[0], sh_piv[1]};
    const Df inv{sh_piv[2], sh_piv[3]};
    // column j: l_r = (H[r][pv] - sum_{i<j} L[r][i] conj(L[pv][i])) / sqrt(d_pv)
    const bool act = live && row != pv && pcol[row] < 0;
    Df sre{0.f, 0.f}, sim{0.f, 0.f};
    float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
    if (act) {
      for (int i = q; i < j; i += LPR) {
        const int c = piv[i];
        const float4 x = Hs[row + c * P], y = Hs[pv + c * P];
        const Df xr{x.x, x.y}, xi{x.z, x.w}, yr{y.x, y.y}, yi{y.z, y.w};
        // x conj(y) = (xr yr + xi yi) + i (xi yr - xr yi)
        sre = df_add(sre, df_add(df_mul(xr, yr), df_mul(xi, yi)));
        sim = df_add(sim, df_add(df_mul(xi, yr), df_neg(df_mul(xr, yi))));
      }
      h = Hs[row + pv * P];
    }
#pragma unroll
    for (int o = 1; o < LPR; o <<= 1) {
      sre = df_add(sre, df_shfl_xor(sre, o));
      sim = df_add(sim, df_shfl_xor(sim, o));
    }
    const Df lr = df_mul(df_add(Df{h.x, h.y}, df_neg(sre)), inv);
    const Df li = df_mul(df_add(Df{h.z, h.w}, df_neg(sim)), inv);
    __syncthreads();  // column pv of H has been read by every row
    DH2_PROF_T(t_c2);
#if DH2_PROF_ON
    pc_col += t_c2 - t_c1;  // the column's entries
#endif
    if (live && q == 0) {
      if (row == pv) {
        Hs[pv + pv * P] = make_float4(sq.hi, sq.lo, 0.f, 0.f);
        Lg[(int64_t)j * p + pv] = C2<T>{(T)((sq.hi + sq.lo) * back), T(0)};
        pcol[pv] = j;
        piv[j] = pv;
      } else if (pcol[row] < 0) {
        Hs[row + pv * P] = make_float4(lr.hi, lr.lo, li.hi, li.lo);
        Lg[(int64_t)j * p + row] = C2<T>{(T)((lr.hi + lr.lo) * back), (T)((li.hi + li.lo) * back)};
        const Df d = df_add(Df{dhi[row], dlo[row]}, df_neg(df_add(df_mul(lr, lr), df_mul(li, li))));
        dhi[row] = d.hi;
        dlo[row] = d.lo;
      } else {
        Hs[row + pv * P] = make_float4(0.f, 0.f, 0.f, 0.f);  // chosen earlier: L[row][j] = 0
        Lg[(int64_t)j * p + row] = C2<T>{T(0), T(0)};
      }
    }
    __syncthreads();
  }
#if DH2_PROF_ON
  DH2_PROF_ADD(12, pc_n);
  DH2_PROF_ADD(13, pc_piv);
  DH2_PROF_ADD(14, pc_col);
#endif
}

// P_T: largest factor size of the instantiation (32, 48, 64 or 128 rows).
// NT: threads per CTA: 4 per row of P_T for the leaf sizes (128, 192, 256),
// 256 for P_T = 128.  Every thread holds 16 chunk entries, so the chunk is
// 64 columns wide for the three leaf sizes.
#ifndef DH2_PAIR_MINB
#define DH2_PAIR_MINB 3  // CTAs per SM at 256 threads (FP32)
#endif
#ifndef DH2_PAIR_MINB192
#define DH2_PAIR_MINB192 4  // at 192 threads
#endif
#ifndef DH2_PAIR_MINB160
#define DH2_PAIR_MINB160 5  // at 160 threads
#endif
#ifndef DH2_PAIR_MINB128
#define DH2_PAIR_MINB128 6  // at 128 threads
#endif
#ifndef DH2_LQT
#define DH2_LQT 8  // threads per row in the streamed LQ (4 or 8)
#endif
// Steps 2-4 of a pair (Jacobi on the K leading columns of L in shared memory,
// the rank from the tail sums, Q), shared by pair_kernel and
// gram_jacobi_kernel.
template <typename T, int P_T, int NT>
__device__ __forceinline__ void jacobi_rank_q(const PairArgs<T>& a, int side, int pid, int p, int LDL, int K,
                                              double E_K, int kcap, int lvl, C2<T>* Lm, double* sig2, int* ord,
                                              int32_t* rank_out, double* sig_out, long long t_b) {
  const int tid = threadIdx.x, warp = tid >> 5;
  __shared__ int sh_rot[2];
  __shared__ unsigned sh_off[2];  // per sweep parity: largest |gamma| / sqrt(alpha beta) rotated (float bits)
  __shared__ int sh_k;
  (void)t_b;
  // ---------------------------------------------------------------- 2. Jacobi
  // one column pair per group of tpp threads (at most the tuning table's
  // width for this class, fewer where the pe/2 pairs of a round need more
  // groups; 4..32); round-robin ordering over pe columns
  const int pe = K + (K & 1);
  const T tol = T(p) * Eps<T>::u;
  constexpr int JH = (P_T / 2 + NT / 4 - 1) / (NT / 4);  // pairs per group at most
  int tpp = a.jacobi_tpp[factor_class(P_T)];
  while (tpp > 4 && tpp * (pe / 2) > NT) tpp >>= 1;
  const int jng = NT / tpp;
  const int jg = tid / tpp, jl = tid & (tpp - 1);
  if (tid == 0) {
    sh_rot[0] = 0;
    sh_rot[1] = 0;
    sh_off[0] = 0u;
    sh_off[1] = 0u;
  }
  __syncthreads();
  bool conv = pe < 2;
  int nsweeps = 0;
  for (int sweep = 0; sweep < a.max_sweeps && pe >= 2; ++sweep) {
    ++nsweeps;
    const int sp = sweep & 1;
    // round-robin positions of this group's pairs in round 0; each round
    // moves every position but the fixed one (index 0) by one place
    int ia[JH], ib[JH];
#pragma unroll
    for (int h = 0; h < JH; ++h) {
      const int kk = jg + h * jng;
      ia[h] = kk;
      ib[h] = pe - 1 - kk;
    }
    for (int rd = 0; rd < pe - 1; ++rd) {
#pragma unroll
      for (int h = 0; h < JH; ++h) {
        const int kk = jg + h * jng;
        // warps with an active group run the reductions converged (full mask)
        if ((warp * 32) / tpp + h * jng < pe / 2) {
          const bool act = kk < pe / 2;
          C2<T>* ca = Lm + (act ? ia[h] : 0) * LDL;
          C2<T>* cb = Lm + (act ? ib[h] : 0) * LDL;
          T al = T(0), be = T(0);
          C2<T> ga = czero<T>();
          if (act)
            for (int r = jl; r < p; r += tpp) {
              const C2<T> xa = ca[r], xb = cb[r];
              al = nmac(al, xa);
              be = nmac(be, xb);
              ga = cmacc(ga, xb, xa);  // + conj(xa) * xb
            }
          for (int o = 1; o < tpp; o <<= 1) {
            al += __shfl_xor_sync(0xffffffffu, al, o);
            be += __shfl_xor_sync(0xffffffffu, be, o);
            ga.re += __shfl_xor_sync(0xffffffffu, ga.re, o);
            ga.im += __shfl_xor_sync(0xffffffffu, ga.im, o);
          }
          const T g2 = cnorm2(ga);
          // rotate unless the pair is orthogonal to tol (relative)
          // rotation scalars from reciprocal square roots and one quotient
          // (hardware approximations in FP32, a few ulp): c^2 + s^2 = 1 to
          // that level, far inside the convergence test's tol = p u
          const T rg = frsqrt(g2);
          const T off = g2 * rg * frsqrt(al) * frsqrt(be);  // |gamma| / sqrt(alpha beta)
          if (act && al > Eps<T>::tiny && be > Eps<T>::tiny && g2 > T(0) && off > tol) {
            const T zt = (be - al) * T(0.5) * rg;
            const T az = fabs(zt);
            const T q1 = T(1) + zt * zt;
            const T t = (zt >= T(0) ? T(1) : T(-1)) *
                        (az > T(1e15) ? fdiv(T(0.5), az) : fdiv(T(1), az + q1 * frsqrt(q1)));
            const T c = frsqrt(T(1) + t * t);
            const T s = t * c;
            if (s != T(0)) {
              const C2<T> e = C2<T>{ga.re * rg, -ga.im * rg};  // e^{-i arg gamma}
              for (int r = jl; r < p; r += tpp) {
                const C2<T> xa = ca[r];
                const C2<T> eb = cmul(e, cb[r]);
                ca[r] = C2<T>{c * xa.re - s * eb.re, c * xa.im - s * eb.im};
                cb[r] = C2<T>{s * xa.re + c * eb.re, s * xa.im + c * eb.im};
              }
              if (jl == 0) {
                sh_rot[sp] = 1;
                atomicMax(&sh_off[sp], __float_as_uint((float)off));
              }
            }
          }
          if (act) {
            if (kk > 0) ia[h] = ia[h] == pe - 1 ? 1 : ia[h] + 1;
            ib[h] = ib[h] == pe - 1 ? 1 : ib[h] + 1;
          }
        }
      }
      __syncthreads();
      if (rd == 0 && tid == 0) {
        sh_rot[sp ^ 1] = 0;
        sh_off[sp ^ 1] = 0u;
      }
    }
    const int rot = sh_rot[sp];
    // quadratic convergence: once the largest rotated off-diagonal ratio of a
    // sweep is below sqrt(tol) / 4, the next sweep's ratios stay below tol,
    // so that confirming sweep is not run
    const T offmax = (T)__uint_as_float(sh_off[sp]);
    __syncthreads();
    if (rot == 0 || offmax * offmax * T(16) <= tol) {
      conv = true;
      break;
    }
  }
  if (!conv && tid == 0) atomicOr(a.status, kStatusNoConv);
  DH2_PROF_T(t_c);
  DH2_PROF_ADD(1, t_c - t_b);
  DH2_PROF_ADD(4, nsweeps);
  DH2_PROF_ADD(5, 1);
  DH2_PROF_ADD(6, p);
  DH2_PROF_ADD(7, K);
  (void)nsweeps;

  // ---------------------------------------------------------------- 3. rank
  const int grp = tid >> 3, gl = tid & 7;
  for (int jb = 0; jb < K; jb += NT / 8) {
    const int j = jb + grp;
    T s = T(0);
    if (j < K)
      for (int r = gl; r < p; r += 8) s = nmac(s, Lm[j * LDL + r]);
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (j < K && gl == 0) sig2[j] = (double)s;
  }
  __syncthreads();
  // non-finite values (only from non-finite input) are ranked as zero and
  // reported; ord stays a permutation of 0..p-1 in every case
  if (tid < K) {
    ord[tid] = tid;
    if (!(sig2[tid] >= 0.0 && sig2[tid] <= 1.0e300)) {
      sig2[tid] = 0.0;
      atomicOr(a.status, kStatusNaN);
    }
  }
  __syncthreads();
  int rk = -1;
  if (tid < K) {
    const double v = sig2[tid];
    rk = 0;
    for (int i = 0; i < K; ++i) {
      const double u = sig2[i];
      rk += (u > v) || (u == v && i < tid);
    }
  }
  __syncthreads();
  if (rk >= 0 && rk < K) ord[rk] = tid;
  __syncthreads();
  if (tid == 0) {
    const double e2 = a.eps2[lvl];
    double tail = E_K;
    int k = K;
    for (int r = K - 1; r >= 0; --r) {
      const double v = sig2[ord[r]];
      if (tail + v <= e2) {
        tail += v;
        k = r;
      } else {
        break;
      }
    }
    if (a.rank_ovr[side] && a.rank_ovr[side][pid] >= 0) k = min(a.rank_ovr[side][pid], K);
    if (k > kcap) k = kcap;
    sh_k = k;
    *rank_out = k;
  }
  for (int r = tid; r < kSigValues; r += NT) sig_out[r] = r < K ? sqrt(sig2[ord[r]]) : 0.0;
  if (tid == 0) {
    sig_out[kSigValues] = (double)K;    // singular values resolved individually
    sig_out[kSigValues + 1] = E_K;      // energy of the rest (sum of their squares)
  }
  __syncthreads();
  const int k = sh_k;

  // ---------------------------------------------------------------- 4. Q
  C2<T>* Qout = a.Q[side] + a.Qoff[side][pid];
  const int ldq = a.rowcap[side][pid];
  for (int qq = grp; qq < k; qq += NT / 8) {
    const int j = ord[qq];
    const T inv = frsqrt((T)sig2[j]);
    for (int r = gl; r < p; r += 8) {
      const C2<T> v = Lm[j * LDL + r];
      if (DH2_IN(a.Qoff[side][pid] + r + (int64_t)qq * ldq, c_lim.Q[side], 10, pid))
        Qout[r + (int64_t)qq * ldq] = C2<T>{v.re * inv, v.im * inv};
    }
  }
  DH2_PROF_T(t_d);
  DH2_PROF_ADD(2, t_d - t_c);
}

// CTAs per SM of the pivoted Cholesky of a Gram matrix (pair_kernel with
// GRAM): its shared memory is H alone (P x P double-float complex), so the
// register file sets the limit for the classes up to 48 rows.  8 / 7 / 5 CTAs
// (64 / 56 / 64 registers, no spills) against the 6 / 5 / 4 of the LQ pair
// kernel: the Cholesky waits on a barrier per pivot step, and more pairs per
// SM fill those waits (measured: factor phase 4.50 -> 4.19 ms at n = 32768)
#ifndef DH2_GRAM_MINB128
#define DH2_GRAM_MINB128 8
#endif
#ifndef DH2_GRAM_MINB160
#define DH2_GRAM_MINB160 7
#endif
#ifndef DH2_GRAM_MINB192
#define DH2_GRAM_MINB192 5
#endif
template <int NT>
constexpr int gram_min_blocks() {
  return NT >= 256 ? 3 : NT >= 192 ? DH2_GRAM_MINB192 : NT >= 160 ? DH2_GRAM_MINB160 : DH2_GRAM_MINB128;
}

template <int NT, typename T>
constexpr int pair_min_blocks() {
  return sizeof(T) == 4 ? (NT >= 256   ? DH2_PAIR_MINB
                           : NT >= 192 ? DH2_PAIR_MINB192
                           : NT >= 160 ? DH2_PAIR_MINB160
                                       : DH2_PAIR_MINB128)
                        : (NT >= 160 ? 1 : 2);
}

template <typename T, int P_T, bool FROM_R, int NT, bool GRAM = false>
__global__ void __launch_bounds__(NT, (GRAM ? gram_min_blocks<NT>() : pair_min_blocks<NT, T>()))
    pair_kernel(const PairArgs<T>* __restrict__ args, const uint32_t* __restrict__ codes, const int P,
                const int* __restrict__ count, const uint64_t* __restrict__ segs) {
  constexpr int LPR = NT / P_T;      // threads per row in the pivoted LQ (rows in place)
  constexpr int LQT = DH2_LQT;       // threads per row in the streamed LQ
  constexpr int GPW = 32 / LQT;      // rows per warp and per block of rows
  constexpr int NW = NT / 32;        // warps
  constexpr int S = P_T / (NT / LQT);  // rows per group of LQT threads
  constexpr int E = 16 / S;          // chunk entries per thread and row
  constexpr int C = LQT * E;         // chunk width (16 * NT / P_T)
  static_assert(LPR >= 1 && LPR <= 32 && S >= 1 && S * E == 16, "16 chunk entries per thread");
  constexpr int XTRA = GRAM ? 0 : C;  // columns after L: the staged chunk of A (none from a Gram matrix)
  static_assert(!GRAM || (!FROM_R && sizeof(T) == 4), "Gram factors: FP32 leaf pairs");
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ C2<T> sh_v0[2];
  __shared__ T sh_tau[2];
  __shared__ int sh_skip[2];
  // leaf column table of the chunk being staged: global index, weight
  __shared__ int cgc[64];
  __shared__ T cwt[64];
  static_assert(C <= 64, "chunk column table");

  const int LDL = P + 1;              // column-major L: element (r, c) at c * LDL + r
  C2<T>* Lm = reinterpret_cast<C2<T>*>(smem);  // (Gram factors: L goes to global memory)
  size_t soff = GRAM ? 0 : ((size_t)(P + XTRA) * LDL * sizeof(C2<T>) + 15) & ~(size_t)15;
  C2<T>* vbuf = reinterpret_cast<C2<T>*>(smem + soff);  // 2 x C reflection vectors
  soff += GRAM ? 0 : 2 * C * sizeof(C2<T>);
  double* sig2 = reinterpret_cast<double*>(smem + soff);
  soff += (size_t)P * sizeof(double);
  int* ord = reinterpret_cast<int*>(smem + soff);
  soff += (size_t)P * sizeof(int);
  int* pcol = reinterpret_cast<int*>(smem + soff);  // pivot step of each row in the pivoted LQ
  soff += (size_t)P * sizeof(int);
  T* nu = reinterpret_cast<T*>(smem + soff);         // residual row norms (Gram factors: Schur diagonal, hi)
  soff += (size_t)P * sizeof(T);
  soff = (soff + 15) & ~(size_t)15;
  float4* Hs = reinterpret_cast<float4*>(smem + soff);  // Gram factors: H, then L column by column
  soff += GRAM ? (size_t)P * P * sizeof(float4) : 0;
  float* dlo = reinterpret_cast<float*>(smem + soff);  // Gram factors: Schur diagonal, lo
  soff += GRAM ? (size_t)P * sizeof(float) : 0;
  int* piv = reinterpret_cast<int*>(smem + soff);      // Gram factors: row chosen at each step

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (count && (int)blockIdx.x >= *count) return;  // launched at capacity: slots past the list's length
  // segs: entries (code << 32 | segment) of non-leaf pairs factored by column
  // segments; this CTA forms one segment's LQ factor only
  const uint32_t code = segs ? (uint32_t)(segs[blockIdx.x] >> 32) : codes[blockIdx.x];
  const int seg = segs ? (int)(uint32_t)segs[blockIdx.x] : -1;
  const int prob = (int)(code >> kCodeProbShift);
  const int side = (int)((code >> kCodeSideShift) & 1u);
  const int pid = (int)(code & kCodePairMask);
  const PairArgs<T>& a = args[prob];
  if (!DH2_IN(pid, c_lim.npairs[side], 9, pid)) return;
  int N = a.ncols[side][pid];
  const int kcap = a.kcap[side][pid];
  const int lvl = a.level[side][pid];

  Source<T, FROM_R> src;
  src.side = side;
  src.pid = pid;
  int p = 0;
  if (FROM_R) {
    const int s0 = a.son[side][2 * pid], s1 = a.son[side][2 * pid + 1];
    if (!DH2_IN(s0, c_lim.npairs[side], 12, pid) || !DH2_IN(s1, c_lim.npairs[side], 13, pid)) return;
    src.k1 = a.rank[side][s0];
    p = src.k1 + a.rank[side][s1];
    src.off0 = a.sonoff[side][2 * pid];
    src.off1 = a.sonoff[side][2 * pid + 1];
    src.ld0 = a.kcap[side][s0];
    src.ld1 = a.kcap[side][s1];
    src.roff0 = a.Roff[side][s0];
    src.roff1 = a.Roff[side][s1];
    src.R0 = a.R[side] + src.roff0;
    src.R1 = a.R[side] + src.roff1;
  } else {
    p = a.m[side][pid];
    src.r0 = a.start[side][pid];
    src.cmo = a.cmoff[side][pid];
    src.gcol = a.gcol[side] + src.cmo;
    src.colw = a.colw[side] + src.cmo;
    src.G = a.G;
    src.ld = a.ld;
    src.pts = a.pts;
    src.nrm = a.nrm;
    src.kappa = a.kappa;
    src.diag = a.diag;
    src.gen = a.gen;
  }
  // column segments of a wide non-leaf pair (Section 6's Ghat_tc = [L_1 Q_1,
  // ..., L_S Q_S] has the singular values and left singular vectors of
  // [L_1 ... L_S]): a segment CTA factors its columns; the pair's own CTA
  // then factors the segments' factors instead of Ghat_tc
  C2<T>* seg_out = nullptr;
  if (FROM_R) {
    const int64_t so = a.seg_off[side] ? a.seg_off[side][pid] : -1;
    if (seg >= 0) {
      if (so < 0 || p > P || p > P_T || p == 0) return;  // reported by the pair's own CTA
      const int c0 = seg * a.seg_cols;
      N = min(a.seg_cols, N - c0);
      src.off0 += c0;
      src.off1 += c0;
      seg_out = a.seg_buf + so + (int64_t)seg * p * p;
      if (N <= 0) {
        for (int i = tid; i < p * p; i += NT) seg_out[i] = czero<T>();
        return;
      }
    } else if (so >= 0 && p > 0) {
      const int nseg = (N + a.seg_cols - 1) / a.seg_cols;
      src.R0 = a.seg_buf + so;
      src.roff0 = so;
      src.k1 = p;
      src.ld0 = p;
      src.off0 = 0;
      src.segsrc = true;
      N = nseg * p;
    }
  }
  int32_t* rank_out = a.rank[side] + pid;
  double* sig_out = a.sig[side] + (int64_t)pid * kSigStride;
  if (p > P || p > P_T) {
    if (tid == 0) {
      atomicOr(a.status, kStatusTooLarge);
      *rank_out = 0;
    }
    return;
  }
  if (p == 0 || N == 0) {
    if (tid == 0) *rank_out = 0;
    for (int r = tid; r < kSigStride; r += NT) sig_out[r] = 0.0;
    return;
  }

  if constexpr (!GRAM)
    for (int i = tid; i < P * LDL; i += NT) Lm[i] = czero<T>();  // L; the staging columns need none
  DH2_PROF_T(t_a);
  const int row = tid / LPR, q = tid % LPR;  // row mapping of the pivoted steps (1b / 1')
  const bool live = row < p;
  const double drop = sizeof(T) == 4 ? 1e-2 : 1e-10;
  int K = p;         // columns kept for the Jacobi step
  double E_K = 0.0;  // energy left out of them
  long long t_b = 0;  // start of the Jacobi step (profile build)
  if constexpr (GRAM) {
    gram_cholesky<T, NT, LPR>(a, side, pid, p, P, row, q, live, drop * a.eps2[lvl],
                              reinterpret_cast<C2<T>*>(a.L4 + a.hoff[side][pid]), Hs, nu, dlo, piv, pcol, K, E_K);
#if DH2_PROF_ON
    t_b = clock64();
#endif
    DH2_PROF_ADD(0, t_b - t_a);
  } else {

  // ---------------------------------------------------------------- 1. LQ
  // Rows go to groups of LQT threads in blocks of GPW = 32/LQT consecutive
  // rows (one row per group of a warp), the blocks dealt round-robin over the
  // warps.  Each thread keeps E entries of each of its S rows of the current
  // chunk in registers (S = 1 for LQT = 4 in the classes up to 64 rows); the
  // chunk is first staged through shared memory with coalesced loads.  Step i
  // applies reflection i (row i) to the rows below it; the warp owning row
  // i+1 updates that row's block first and forms reflection i+1, then updates
  // its other blocks; one barrier per step.  The reductions over a row run on
  // its group alone (measured faster than running every group converged with
  // the full mask).
  const int lq = lane & (LQT - 1);
  const int lgrp = lane / LQT;
  // row of slot s of this thread: block warp + NW * s, row `lgrp` in it
  auto lrow = [&](int s) { return GPW * (warp + NW * s) + lgrp; };
  // does slot s of this warp hold a row r > j (r < p)?
  auto slot_live = [&](int s, int j) { return min(GPW * (warp + NW * s) + GPW - 1, p - 1) > j; };
  // chunk column of entry u of a thread: pairs of adjacent columns, so that
  // the reflection vector moves in 16-byte words
  auto ccol = [&](int u) { return 2 * lq + (u & 1) + (u >> 1) * 2 * LQT; };
  C2<T>* Xs = Lm + (int64_t)P * LDL;  // staged chunk: column jj at Xs[jj * LDL]
  C2<T> ch[S][E];

  // Householder reflection of row r from the right: the row becomes
  // (beta, 0, ..., 0) on the columns {r} u chunk, beta = -e^{i arg alpha} |x|;
  // the chunk part x is the reflection's vector (vbuf[slot]).  Called by a
  // whole warp; only the quarter holding row r (mine) works.
  auto publish = [&](int r, const C2<T> (&x)[E], bool mine, int slot) {
    if (!mine) return;
    const unsigned qmask = ((1u << LQT) - 1u) << (lane & (32 - LQT));
    // the diagonal entry and its phase do not depend on the row norm: form
    // them while the norm is reduced
    const C2<T> al = Lm[r * LDL + r];
    const T an2 = cnorm2(al);
    const T ra = an2 > Eps<T>::tiny ? frsqrt(an2) : T(0);
    const T an = an2 * ra;
    const C2<T> ph = an2 > Eps<T>::tiny ? C2<T>{al.re * ra, al.im * ra} : C2<T>{T(1), T(0)};
#pragma unroll
    for (int u = 0; u < E; u += 2) store_c2x2(vbuf + slot * C + ccol(u), x[u], x[u + 1]);
    T s0 = T(0), s1 = T(0);
#pragma unroll
    for (int u = 0; u < E; u += 2) {
      s0 = nmac(s0, x[u]);
      if (u + 1 < E) s1 = nmac(s1, x[u + 1]);
    }
    s0 += s1;
#pragma unroll
    for (int o = 1; o < LQT; o <<= 1) s0 += __shfl_xor_sync(qmask, s0, o);
    if (lq == 0) {
      if (!(s0 > Eps<T>::tiny)) {
        sh_skip[slot] = 1;
      } else {
        const T xn2 = s0 + an2;
        const T xn = xn2 * frsqrt(xn2);
        Lm[r * LDL + r] = C2<T>{-ph.re * xn, -ph.im * xn};
        sh_v0[slot] = C2<T>{ph.re * (an + xn), -ph.im * (an + xn)};
        sh_tau[slot] = fdiv(T(1), xn * (xn + an));
        sh_skip[slot] = 0;
      }
    }
  };

  // apply reflection j (vector x, scalars v0, tau) to this thread's row r of a
  // slot (entries c); called by a whole warp, rows other than j < r < p are
  // left unchanged (their quarters return at once)
  auto apply = [&](C2<T> (&c)[E], int r, int j, const C2<T>* xs, C2<T> v0, T tau_j) {
    const bool act = r > j && r < p;
    if (!act) return;
    const unsigned qmask = ((1u << LQT) - 1u) << (lane & (32 - LQT));
    const T tau = tau_j;
    const C2<T> lrj = Lm[j * LDL + r];
    C2<T> x[E];
#pragma unroll
    for (int u = 0; u < E; u += 2) load_c2x2(xs + ccol(u), x[u], x[u + 1]);
    C2<T> wa[4] = {czero<T>(), czero<T>(), czero<T>(), czero<T>()};
#pragma unroll
    for (int u = 0; u < E; ++u) wa[u & 3] = cmacc(wa[u & 3], c[u], x[u]);
    C2<T> w = cadd(cadd(wa[0], wa[1]), cadd(wa[2], wa[3]));
#pragma unroll
    for (int o = 1; o < LQT; o <<= 1) {
      w.re += __shfl_xor_sync(qmask, w.re, o);
      w.im += __shfl_xor_sync(qmask, w.im, o);
    }
    w = cadd(w, cmul(lrj, v0));
    const C2<T> tw = C2<T>{tau * w.re, tau * w.im};
#pragma unroll
    for (int u = 0; u < E; ++u) c[u] = cnmac(c[u], tw, x[u]);
    if (lq == 0) Lm[j * LDL + r] = csub(lrj, cmulc(tw, v0));
  };

  auto stage = [&](int j0, int cwid, int ncols, C2<T>* dst) {
    stage_table<T, FROM_R, NT>(src, j0, cwid, cgc, cwt);
    if (!FROM_R) __syncthreads();
    stage_cols<T, FROM_R, NT>(src, p, j0, cwid, ncols, dst, LDL, cgc, cwt);
  };

  // Asynchronous staging of the next chunk while the steps of the current one
  // run (all but the matrix-free mode, whose entries are computed): the
  // column table (leaf) at step 0, the entries at step 2 once the table is
  // visible, the weights and the conjugation of G^* applied after the last
  // step.  Xs is free during the steps: the chunk is in registers.
  const bool async_ok = FROM_R || !src.gen;
  auto issue_table = [&](int j0n, int cwn) {
    for (int jj = tid; jj < cwn; jj += NT) {
      if (DH2_IN(src.cmo + j0n + jj, c_lim.ncol[side], 3, pid)) {
        cp_async<4>(&cgc[jj], src.gcol + j0n + jj);
        cp_async<sizeof(T)>(&cwt[jj], src.colw + j0n + jj);
      } else {
        cgc[jj] = 0;
        cwt[jj] = T(0);
      }
    }
    cp_async_commit();
  };
  const bool down = FROM_R || side == 0;  // consecutive threads on the contiguous direction
  auto issue_cols = [&](int j0n, int cwn) {
    for (Walk2 it(tid, NT, down ? p : C); it.g < (down ? C : p); it.next()) {
      const int r = down ? it.f : it.g;
      const int jj = down ? it.g : it.f;
      C2<T>* d = Xs + jj * LDL + r;
      const C2<T>* g = nullptr;
      if (jj < cwn) g = FROM_R ? src.sons_ptr(r, j0n + jj) : src.leaf_ptr(r, cgc[jj]);
      if (g) cp_async<sizeof(C2<T>)>(d, g);
      else *d = czero<T>();
    }
    cp_async_commit();
  };
  auto finish_cols = [&](int cwn) {
    if (FROM_R) return;
    for (Walk2 it(tid, NT, down ? p : C); it.g < (down ? C : p); it.next()) {
      const int r = down ? it.f : it.g;
      const int jj = down ? it.g : it.f;
      if (jj < cwn) {
        C2<T>* d = Xs + jj * LDL + r;
        const C2<T> g = *d;
        const T w = cwt[jj];
        *d = C2<T>{g.re * w, side == 0 ? g.im * w : -g.im * w};
      }
    }
  };

  {
    DH2_PROF_T(t_s0);
    stage(0, min(C, N), C, Xs);
    __syncthreads();
    DH2_PROF_T(t_s1);
    DH2_PROF_ADD(8, t_s1 - t_s0);
  }
#if DH2_PROF_ON
  long long pw_all = 0, pw_crit = 0, pw_pub = 0, pw_steps = 0;
  long long pq_a = 0, pq_b = 0, pq_c = 0;
#endif
  for (int j0 = 0; j0 < N; j0 += C) {
    DH2_PROF_ADD(9, 1);
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int r = lrow(s);
#pragma unroll
      for (int u = 0; u < E; ++u) ch[s][u] = r < p ? Xs[ccol(u) * LDL + r] : czero<T>();
    }
    if (warp == 0) publish(0, ch[0], lrow(0) == 0, 0);
    __syncthreads();
    const int j0n = j0 + C;
    const int cwn = min(C, N - j0n);
    const bool pre = async_ok && j0n < N;
    bool issued = false;
    for (int i = 0; i < p; ++i) {
#if DH2_PROF_ON
      const long long ts0 = clock64();
      long long tsp = ts0;
#endif
      const int sl = i & 1;
      // a skipped reflection (zero chunk part) is the identity: tau = 0
      const bool skip = sh_skip[sl] != 0;
      const C2<T>* x = vbuf + sl * C;
      const C2<T> v0 = skip ? czero<T>() : sh_v0[sl];
      const T tau = skip ? T(0) : sh_tau[sl];
      const int b1 = (i + 1) / GPW;  // block of row i+1
      const int cs = i + 1 < p && (b1 % NW) == warp ? b1 / NW : -1;
#if DH2_PROF_ON
      const long long tsa = clock64();
#endif
      // slots in increasing order: for the owner of row i+1 that row's slot is
      // its lowest live one, so the next reflection is formed first
#pragma unroll
      for (int s = 0; s < S; ++s) {
        if (!slot_live(s, i)) continue;
        apply(ch[s], lrow(s), i, x, v0, tau);
        if (s == cs) {
#if DH2_PROF_ON
          const long long tsb = clock64();
#endif
          publish(i + 1, ch[s], lrow(s) == i + 1, sl ^ 1);
#if DH2_PROF_ON
          if (lrow(s) == i + 1 && lq == 0) {
            const long long tsc = clock64();
            pq_a += tsa - ts0;
            pq_b += tsb - tsa;
            pq_c += tsc - tsb;
          }
          __syncwarp();
          tsp = clock64();
#endif
        }
      }
#if DH2_PROF_ON
      __syncwarp();
      {
        const long long ts1 = clock64();
        pw_all += ts1 - ts0;
        if (cs >= 0) {
          pw_crit += ts1 - ts0;
          pw_pub += tsp - ts0;
        }
        ++pw_steps;
      }
#endif
      if (pre) {
        if (FROM_R) {
          if (i == 0) {
            issue_cols(j0n, cwn);
            issued = true;
          }
        } else if (i == 0) {
          issue_table(j0n, cwn);
        } else if (i == 1) {
          cp_async_wait_all();  // the table, visible to all after this step's barrier
        } else if (i == 2) {
          issue_cols(j0n, cwn);
          issued = true;
        }
      }
      __syncthreads();
    }
    if (j0n < N) {
      DH2_PROF_T(t_s0);
      cp_async_wait_all();
      if (issued) {
        finish_cols(cwn);
      } else {
        stage(j0n, cwn, C, Xs);  // short pair or matrix-free mode
      }
      __syncthreads();  // next chunk staged
      DH2_PROF_T(t_s1);
      DH2_PROF_ADD(8, t_s1 - t_s0);
    }
  }

#if DH2_PROF_ON
  t_b = clock64();
#endif
  DH2_PROF_ADD(0, t_b - t_a);
#if DH2_PROF_ON
  if (lane == 0) {
    atomicAdd(&g_prof[10], (unsigned long long)pw_crit);
    atomicAdd(&g_prof[11], (unsigned long long)pw_all);
    atomicAdd(&g_prof[13], (unsigned long long)pw_pub);
  }
  if (tid == 0) atomicAdd(&g_prof[12], (unsigned long long)pw_steps);
  if (pq_a + pq_b + pq_c) {
    atomicAdd(&g_prof[14], (unsigned long long)pq_a);
    atomicAdd(&g_prof[15], (unsigned long long)pq_b);
    atomicAdd(&g_prof[16], (unsigned long long)pq_c);
  }
#endif

  if (seg_out) {  // a segment: its factor L (p x p, ld p) for the pair's CTA
    for (int i = tid; i < p * p; i += NT) seg_out[i] = Lm[(i / p) * LDL + i % p];
    return;
  }

  // ---------------------------------------------------------------- 1b. pivoted LQ of L
  // Rank-revealing step: L Omega' = L' by Householder reflections from the
  // right with row pivoting (the row of largest residual norm first).  Rows
  // stay in place: pcol[r] records the step at which row r was chosen (-1
  // while it has not been), so L' is lower triangular up to a row
  // permutation.  The step stops at the first K whose remaining rows have
  // residual energy E_K <= drop * eps_l^2 over columns K..p-1; that energy is
  // added to every tail sum below (an upper bound on the residual of the
  // chosen subspace), and the Jacobi step works on the K leading columns only.
  // Two barriers per step: the pivot search is repeated by every warp on the
  // shared residual norms, so it needs none of its own.
  const T tau_drop_t = (T)(drop * a.eps2[lvl]);
  // (shuffles run converged over whole warps with the full mask; the row
  // predicates only gate the memory accesses)
  {
    T s = T(0);
    if (live)
      for (int c = q; c < p; c += LPR) s = nmac(s, Lm[c * LDL + row]);
#pragma unroll
    for (int o = 1; o < LPR; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (live && q == 0) {
      nu[row] = s;
      pcol[row] = -1;
    }
  }
  __syncthreads();
  for (int i = 0; i < p; ++i) {
    // residual energy of the unchosen rows and the pivot (lowest row on ties);
    // the butterfly leaves the same values in every lane of every warp
    T e = T(0);
    T best = T(-1);
    int pv = p;
    for (int r = lane; r < p; r += 32) {
      if (pcol[r] < 0) {
        const T v = nu[r];
        e += v;
        if (v > best) {
          best = v;
          pv = r;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e += __shfl_xor_sync(0xffffffffu, e, o);
      const T ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, pv, o);
      if (ob > best || (ob == best && oi < pv)) {
        best = ob;
        pv = oi;
      }
    }
    if (e <= tau_drop_t || pv >= p) {
      K = i;
      E_K = (double)e;
      break;
    }
    if (warp == pv / (32 / LPR)) {
      // reflector of row pv over columns i..p-1: the row becomes beta e_i
      T s = T(0);
      if (row == pv)
        for (int c = i + 1 + q; c < p; c += LPR) s = nmac(s, Lm[c * LDL + pv]);
#pragma unroll
      for (int o = 1; o < LPR; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (row == pv && q == 0) {
        if (!(s > Eps<T>::tiny)) {
          sh_skip[0] = 1;
        } else {
          const C2<T> al = Lm[i * LDL + pv];
          const T an2 = cnorm2(al);
          const T ra = an2 > Eps<T>::tiny ? frsqrt(an2) : T(0);
          const T an = an2 * ra;
          const T xn2 = s + an2;
          const T xn = xn2 * frsqrt(xn2);
          const C2<T> ph = an2 > Eps<T>::tiny ? C2<T>{al.re * ra, al.im * ra} : C2<T>{T(1), T(0)};
          Lm[i * LDL + pv] = C2<T>{-ph.re * xn, -ph.im * xn};
          sh_v0[0] = C2<T>{ph.re * (an + xn), -ph.im * (an + xn)};
          sh_tau[0] = fdiv(T(1), xn * (xn + an));
          sh_skip[0] = 0;
        }
      }
    }
    __syncthreads();
    // apply to the unchosen rows and refresh their residual norms (columns > i);
    // pcol[pv] is set only here, after every warp's pivot search has read it
    if (row == pv && q == 0) pcol[pv] = i;
    if (warp * (32 / LPR) < p) {  // warps holding rows
      const bool act = live && row != pv && pcol[row] < 0;
      const bool skip = sh_skip[0] != 0;
      T s = T(0);
      C2<T> w = czero<T>();
      if (act && !skip) {
        if (q == 0) w = cmul(Lm[i * LDL + row], sh_v0[0]);
        for (int c = i + 1 + q; c < p; c += LPR) w = cmacc(w, Lm[c * LDL + row], Lm[c * LDL + pv]);
      }
      if (!skip) {
#pragma unroll
        for (int o = 1; o < LPR; o <<= 1) {
          w.re += __shfl_xor_sync(0xffffffffu, w.re, o);
          w.im += __shfl_xor_sync(0xffffffffu, w.im, o);
        }
      }
      if (act) {
        if (!skip) {
          const C2<T> v0 = sh_v0[0];
          const T tau = sh_tau[0];
          const C2<T> tw = C2<T>{tau * w.re, tau * w.im};
          for (int c = i + 1 + q; c < p; c += LPR) {
            const C2<T> x = cnmac(Lm[c * LDL + row], tw, Lm[c * LDL + pv]);
            Lm[c * LDL + row] = x;
            s = nmac(s, x);
          }
          if (q == 0) Lm[i * LDL + row] = csub(Lm[i * LDL + row], cmulc(tw, v0));
        } else {
          for (int c = i + 1 + q; c < p; c += LPR) s = nmac(s, Lm[c * LDL + row]);
        }
      }
#pragma unroll
      for (int o = 1; o < LPR; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (act && q == 0) nu[row] = s;
    }
    __syncthreads();
  }
  }  // LQ steps (1, 1b)
  if (!(E_K >= 0.0 && E_K <= 1.0e300)) {  // only from non-finite input
    if (tid == 0) atomicOr(a.status, kStatusNaN);
    E_K = 0.0;
  }
  if constexpr (GRAM) {
    // L (columns < K) is in the factor buffer; a zero column pads it to
    // even width; K and E_K go to the singular-value record, and
    // gram_jacobi_kernel takes it from there
    C2<T>* Lg = reinterpret_cast<C2<T>*>(a.L4 + a.hoff[side][pid]);
    if (K & 1)
      for (int i = tid; i < p; i += NT) Lg[(int64_t)K * p + i] = czero<T>();
    if (tid == 0) {
      sig_out[kSigValues] = (double)K;
      sig_out[kSigValues + 1] = E_K;
    }
    return;
  }
  // chosen rows keep their reflector vectors right of their pivot column and
  // unchosen rows their residual right of column K: clear what the Jacobi step
  // reads (columns < pe, pe = K rounded up to even)
  {
    const int pe0 = K + (K & 1);
    if (live) {
      const int from = pcol[row] >= 0 ? pcol[row] + 1 : K;
      for (int c = from + q; c < pe0; c += LPR) Lm[c * LDL + row] = czero<T>();
    }
  }
  __syncthreads();
  jacobi_rank_q<T, P_T, NT>(a, side, pid, p, LDL, K, E_K, kcap, lvl, Lm, sig2, ord, rank_out, sig_out, t_b);
}

// Steps 2-4 of the leaf pairs of a mixed-mode launch list, after the
// pivoted Cholesky of their Gram matrices (pair_kernel<..., GRAM>): L (p x K,
// ld p, columns < K rounded up to even) from the factor buffer L4, K and E_K
// from its singular-value record.  Only L is held in shared memory, so that
// more pairs run side by side than in the Cholesky, whose shared memory holds
// all of H.
template <int P_T, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    gram_jacobi_kernel(const PairArgs<float>* __restrict__ args, const uint32_t* __restrict__ codes, const int P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int LDL = P + 1;
  C2<float>* Lm = reinterpret_cast<C2<float>*>(smem);
  size_t soff = ((size_t)P * LDL * sizeof(C2<float>) + 15) & ~(size_t)15;
  double* sig2 = reinterpret_cast<double*>(smem + soff);
  soff += (size_t)P * sizeof(double);
  int* ord = reinterpret_cast<int*>(smem + soff);
  const int tid = threadIdx.x;
  const uint32_t code = codes[blockIdx.x];
  const PairArgs<float>& a = args[code >> kCodeProbShift];
  const int side = (int)((code >> kCodeSideShift) & 1u);
  const int pid = (int)(code & kCodePairMask);
  if (!DH2_IN(pid, c_lim.npairs[side], 14, pid)) return;
  const int p = a.m[side][pid];
  const int N = a.ncols[side][pid];
  if (p > P || p > P_T || p == 0 || N == 0) return;  // rank and record already written by the Cholesky launch
  int32_t* rank_out = a.rank[side] + pid;
  double* sig_out = a.sig[side] + (int64_t)pid * kSigStride;
  const int K = (int)sig_out[kSigValues];
  const double E_K = sig_out[kSigValues + 1];
  const int pe = K + (K & 1);
  const C2<float>* Lg = reinterpret_cast<const C2<float>*>(a.L4 + a.hoff[side][pid]);
  for (int i = tid; i < pe * p; i += NT) Lm[(i / p) * LDL + i % p] = Lg[i];
  __syncthreads();
  long long t_b = 0;
#if DH2_PROF_ON
  t_b = clock64();
#endif
  jacobi_rank_q<float, P_T, NT>(a, side, pid, p, LDL, K, E_K, a.kcap[side][pid], a.level[side][pid], Lm, sig2, ord,
                                rank_out, sig_out, t_b);
}

// R_tc = Q^* A for the pairs of one launch (Section 6, R recursion: R_tc =
// V_tc^* G_tc for a leaf, [E_t1c; E_t2c]^* Ghat_tc for a non-leaf), after
// pair_kernel has written Q and the rank.  One CTA of 128 threads per tile of
// TW = 32 columns of one pair (tile = launch code << 32 | first column), so
// that the loads of many tiles are in flight at once.  The leaf column table
// is read first; the entries of A and the block of Q then arrive together by
// cp.async, and the weights and the conjugation of G^* are applied in shared
// memory.  Each thread forms 2 x 2 outputs of the k x TW tile of R.
template <typename T, bool FROM_R>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 6 : 2)
    rq_kernel(const PairArgs<T>* __restrict__ args, const uint64_t* __restrict__ tiles, const int P) {
  constexpr int NT = 128;
  constexpr int QB = 32;
  constexpr int TW = kRTile;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int cgc[TW];
  __shared__ T cwt[TW];
  // row-major tiles, row r of Q's block at Qs[r * LQ] and of A's tile at
  // As[r * LA] (padded rows of 16-byte multiples)
  constexpr int LQ = QB + 2, LA = TW + 2;
  C2<T>* Qs = reinterpret_cast<C2<T>*>(smem);
  C2<T>* As = Qs + P * LQ;
  const int tid = threadIdx.x;
  const uint64_t tile = tiles[blockIdx.x];
  const uint32_t code = (uint32_t)(tile >> 32);
  const int j0 = (int)(uint32_t)tile;
  const int prob = (int)(code >> kCodeProbShift);
  const int side = (int)((code >> kCodeSideShift) & 1u);
  const int pid = (int)(code & kCodePairMask);
  const PairArgs<T>& a = args[prob];
  if (!DH2_IN(pid, c_lim.npairs[side], 9, pid)) return;
  const int N = a.ncols[side][pid];
  const int k = a.rank[side][pid];
  if (k <= 0 || j0 >= N) return;
  Source<T, FROM_R> src;
  src.side = side;
  src.pid = pid;
  int p = 0;
  if (FROM_R) {
    const int s0 = a.son[side][2 * pid], s1 = a.son[side][2 * pid + 1];
    if (!DH2_IN(s0, c_lim.npairs[side], 12, pid) || !DH2_IN(s1, c_lim.npairs[side], 13, pid)) return;
    src.k1 = a.rank[side][s0];
    p = src.k1 + a.rank[side][s1];
    src.off0 = a.sonoff[side][2 * pid];
    src.off1 = a.sonoff[side][2 * pid + 1];
    src.ld0 = a.kcap[side][s0];
    src.ld1 = a.kcap[side][s1];
    src.roff0 = a.Roff[side][s0];
    src.roff1 = a.Roff[side][s1];
    src.R0 = a.R[side] + src.roff0;
    src.R1 = a.R[side] + src.roff1;
  } else {
    p = a.m[side][pid];
    src.r0 = a.start[side][pid];
    src.cmo = a.cmoff[side][pid];
    src.gcol = a.gcol[side] + src.cmo;
    src.colw = a.colw[side] + src.cmo;
    src.G = a.G;
    src.ld = a.ld;
    src.pts = a.pts;
    src.nrm = a.nrm;
    src.kappa = a.kappa;
    src.diag = a.diag;
    src.gen = a.gen;
  }
  if (p <= 0 || p > P) return;  // reported by pair_kernel
  const bool gen = !FROM_R && src.gen;
  const bool down = FROM_R || side == 0;  // consecutive threads on the contiguous direction
  const int cw = min(TW, N - j0);
  const C2<T>* Qin = a.Q[side] + a.Qoff[side][pid];
  const int ldq = a.rowcap[side][pid];
  C2<T>* Rout = a.R[side] + a.Roff[side][pid];
  const int kcap = a.kcap[side][pid];
  if (!FROM_R) {
    stage_table<T, FROM_R, NT>(src, j0, cw, cgc, cwt);
    __syncthreads();
  }
  for (int qb = 0; qb < k; qb += QB) {
    const int kb = min(QB, k - qb);
    if (qb > 0) __syncthreads();  // the previous block's products are done with Qs
    for (Walk2 it(tid, NT, p); it.g < kb; it.next()) {
      const int r = it.f, qq = it.g;
      const int64_t e = r + (int64_t)(qb + qq) * ldq;
      if (DH2_IN(a.Qoff[side][pid] + e, c_lim.Q[side], 14, pid)) cp_async<sizeof(C2<T>)>(Qs + r * LQ + qq, Qin + e);
      else Qs[r * LQ + qq] = czero<T>();
    }
    if (qb == 0) {
      for (Walk2 it(tid, NT, down ? p : cw); it.g < (down ? cw : p); it.next()) {
        const int r = down ? it.f : it.g;
        const int jj = down ? it.g : it.f;
        C2<T>* d = As + r * LA + jj;
        if (gen) {
          *d = src.leaf_at(r, cgc[jj], cwt[jj]);
        } else {
          const C2<T>* g = FROM_R ? src.sons_ptr(r, j0 + jj) : src.leaf_ptr(r, cgc[jj]);
          if (g) cp_async<sizeof(C2<T>)>(d, g);
          else *d = czero<T>();
        }
      }
    }
    cp_async_commit();
    cp_async_wait_all();
    if (qb == 0 && !FROM_R && !gen) {
      // weights 1/omega_b and, for the column basis, the conjugation of G^*
      for (Walk2 it(tid, NT, down ? p : cw); it.g < (down ? cw : p); it.next()) {
        const int r = down ? it.f : it.g;
        const int jj = down ? it.g : it.f;
        C2<T>* d = As + r * LA + jj;
        const C2<T> g = *d;
        const T w = cwt[jj];
        *d = C2<T>{g.re * w, side == 0 ? g.im * w : -g.im * w};
      }
    }
    __syncthreads();
    // 2 x 2 output tiles
    const int nqt = (kb + 1) >> 1, njt = (cw + 1) >> 1;
    for (int t = tid; t < nqt * njt; t += NT) {
      const int q0 = 2 * (t % nqt), jb = 2 * (t / nqt);
      // entries past kb or cw are read (finite or not) but never stored
      const C2<T>* qp = Qs + q0;
      const C2<T>* ap = As + jb;
      C2<T> c00 = czero<T>(), c01 = czero<T>(), c10 = czero<T>(), c11 = czero<T>();
#pragma unroll 2
      for (int r = 0; r < p; ++r, qp += LQ, ap += LA) {
        C2<T> x0, x1, y0, y1;
        load_c2x2(qp, x0, x1);
        load_c2x2(ap, y0, y1);
        c00 = cmacc(c00, y0, x0);
        c01 = cmacc(c01, y1, x0);
        c10 = cmacc(c10, y0, x1);
        c11 = cmacc(c11, y1, x1);
      }
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        const int qq = q0 + (d >> 1), jj = jb + (d & 1);
        const C2<T> v = d == 0 ? c00 : d == 1 ? c01 : d == 2 ? c10 : c11;
        const int64_t e = (qb + qq) + (int64_t)(j0 + jj) * kcap;
        if (qq < kb && jj < cw && DH2_IN(a.Roff[side][pid] + e, c_lim.R[side], 11, pid)) Rout[e] = v;
      }
    }
  }
}

// One tile of the leaf R = Q^* A: pair, columns and the addresses its loads
// and stores need (live = false for a tile past the list or with rank 0).
template <typename T>
struct RqLeafTile {
  const C2<T>* G;
  const int32_t* gcol;  // column map of the pair, from its first column
  const T* colw;
  const C2<T>* Q;
  C2<T>* R;
  int64_t ld, cmo, qoff, roff;
  int side, pid, r0, p, k, cw, j0, ldq, kcap;
  bool live;
};

template <typename T>
__device__ __forceinline__ RqLeafTile<T> rq_leaf_tile(const PairArgs<T>* __restrict__ args,
                                                      const uint64_t* __restrict__ tiles, int64_t t,
                                                      int64_t ntiles, int P) {
  RqLeafTile<T> x;
  x.live = false;
  x.side = x.pid = x.r0 = x.p = x.k = x.cw = x.j0 = x.ldq = x.kcap = 0;
  x.ld = x.cmo = x.qoff = x.roff = 0;
  x.G = x.Q = nullptr;
  x.R = nullptr;
  x.gcol = nullptr;
  x.colw = nullptr;
  if (t >= ntiles) return x;
  const uint64_t tile = tiles[t];
  const uint32_t code = (uint32_t)(tile >> 32);
  x.j0 = (int)(uint32_t)tile;
  const int prob = (int)(code >> kCodeProbShift);
  x.side = (int)((code >> kCodeSideShift) & 1u);
  x.pid = (int)(code & kCodePairMask);
  const PairArgs<T>& a = args[prob];
  if (!DH2_IN(x.pid, c_lim.npairs[x.side], 9, x.pid)) return x;
  const int sd = x.side, pid = x.pid;
  const int N = a.ncols[sd][pid];
  x.k = a.rank[sd][pid];
  x.p = a.m[sd][pid];
  if (x.k <= 0 || x.j0 >= N || x.p <= 0 || x.p > P) return x;  // p > P: reported by pair_kernel
  x.cw = min(kRTile, N - x.j0);
  x.r0 = a.start[sd][pid];
  x.cmo = a.cmoff[sd][pid];
  x.gcol = a.gcol[sd] + x.cmo;
  x.colw = a.colw[sd] + x.cmo;
  x.G = a.G;
  x.ld = a.ld;
  x.qoff = a.Qoff[sd][pid];
  x.Q = a.Q[sd] + x.qoff;
  x.ldq = a.rowcap[sd][pid];
  x.roff = a.Roff[sd][pid];
  x.R = a.R[sd] + x.roff;
  x.kcap = a.kcap[sd][pid];
  x.live = true;
  return x;
}

// R_tc = Q^* A for the leaf pairs (Section 6, R_tc = V_tc^* G_tc), the
// dense-matrix modes.  A persistent kernel: CTA b takes tiles b, b + grid,
// ... of the tile list.  While it forms the products of one tile, the next
// tile's entries and Q block and the column table of the tile after that are
// in flight (cp.async), in a second shared-memory stage and a third table
// slot, so that the load latency of a tile hides behind the arithmetic of the
// one before.  The weight 1/omega_b and the conjugation of G^* are applied to
// the outputs: for the row basis R = w sum_r conj(Q) G, for the column basis
// R = w conj(sum_r Q G') with G' the stored entries of G.
#ifndef DH2_RQ_MINB
#define DH2_RQ_MINB 3  // FP32 leaf R kernel: register cap for this many CTAs per SM
#endif
template <typename T>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? DH2_RQ_MINB : 2)
    rq_leaf_kernel(const PairArgs<T>* __restrict__ args, const uint64_t* __restrict__ tiles, const int64_t ntiles,
                   const int P) {
  constexpr int NT = 128;
  constexpr int QB = 16;  // ranks per pass (leaf ranks are mostly below 16): a smaller Q stage, more CTAs per SM
  constexpr int TW = kRTile;
  constexpr int LQ = QB + 2, LA = TW + 2;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int cgc[3][TW];
  __shared__ T cwt[3][TW];
  C2<T>* const base = reinterpret_cast<C2<T>*>(smem);
  auto stQ = [&](int s) { return base + (size_t)s * P * (LQ + LA); };
  auto stA = [&](int s) { return base + (size_t)s * P * (LQ + LA) + (size_t)P * LQ; };
  const int tid = threadIdx.x;
  const int64_t stride = gridDim.x;

  auto issue_table = [&](const RqLeafTile<T>& x, int slot) {
    if (!x.live) return;
    for (int jj = tid; jj < x.cw; jj += NT) {
      if (DH2_IN(x.cmo + x.j0 + jj, c_lim.ncol[x.side], 3, x.pid)) {
        cp_async<4>(&cgc[slot][jj], x.gcol + x.j0 + jj);
        cp_async<sizeof(T)>(&cwt[slot][jj], x.colw + x.j0 + jj);
      } else {
        cgc[slot][jj] = 0;
        cwt[slot][jj] = T(0);
      }
    }
  };
  // entries of the tile (needs its table) and block qb of Q
  auto issue_q = [&](const RqLeafTile<T>& x, int s, int qb) {
    C2<T>* Qs = stQ(s);
    const int kb = min(QB, x.k - qb);
    for (Walk2 it(tid, NT, x.p); it.g < kb; it.next()) {
      const int r = it.f, qq = it.g;
      const int64_t e = r + (int64_t)(qb + qq) * x.ldq;
      if (DH2_IN(x.qoff + e, c_lim.Q[x.side], 14, x.pid)) cp_async<sizeof(C2<T>)>(Qs + r * LQ + qq, x.Q + e);
      else Qs[r * LQ + qq] = czero<T>();
    }
  };
  auto issue_a = [&](const RqLeafTile<T>& x, int s, int slot) {
    if (!x.live) return;
    C2<T>* As = stA(s);
    const bool down = x.side == 0;  // consecutive threads on the contiguous direction
    for (Walk2 it(tid, NT, down ? x.p : x.cw); it.g < (down ? x.cw : x.p); it.next()) {
      const int r = down ? it.f : it.g;
      const int jj = down ? it.g : it.f;
      const int gc = cgc[slot][jj];
      const int64_t e = x.side == 0 ? (int64_t)gc * x.ld + x.r0 + r : (int64_t)(x.r0 + r) * x.ld + gc;
      if (DH2_IN(e, c_lim.G, x.side == 0 ? 5 : 7, x.pid)) cp_async<sizeof(C2<T>)>(As + r * LA + jj, x.G + e);
      else As[r * LA + jj] = czero<T>();
    }
    issue_q(x, s, 0);
  };
  // 2 x 2 output tiles of block qb; entries past kb or cw are read (finite or
  // not) but never stored
  auto products = [&](const RqLeafTile<T>& x, int s, int slot, int qb) {
    const C2<T>* Qs = stQ(s);
    const C2<T>* As = stA(s);
    const int kb = min(QB, x.k - qb);
    const int nqt = (kb + 1) >> 1, njt = (x.cw + 1) >> 1;
    const T sg = x.side == 0 ? T(1) : T(-1);  // conj(Q) for the row basis, Q for the column basis
    for (int u = tid; u < nqt * njt; u += NT) {
      const int q0 = 2 * (u % nqt), jb = 2 * (u / nqt);
      C2<T> c00 = czero<T>(), c01 = czero<T>(), c10 = czero<T>(), c11 = czero<T>();
      // the row loop once per basis (no sign multiply per entry of Q): the
      // products with conj(Q) (row basis) or Q (column basis)
      auto rows = [&](auto conj_q) {
        const C2<T>* qp = Qs + q0;
        const C2<T>* ap = As + jb;
#pragma unroll 2
        for (int r = 0; r < x.p; ++r, qp += LQ, ap += LA) {
          C2<T> x0, x1, y0, y1;
          load_c2x2(qp, x0, x1);
          load_c2x2(ap, y0, y1);
          if constexpr (decltype(conj_q)::value) {
            c00 = cmacc(c00, y0, x0);
            c01 = cmacc(c01, y1, x0);
            c10 = cmacc(c10, y0, x1);
            c11 = cmacc(c11, y1, x1);
          } else {
            c00 = cmac_nc(c00, y0, x0);
            c01 = cmac_nc(c01, y1, x0);
            c10 = cmac_nc(c10, y0, x1);
            c11 = cmac_nc(c11, y1, x1);
          }
        }
      };
      if (x.side == 0) rows(std::true_type{});
      else rows(std::false_type{});
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        const int qq = q0 + (d >> 1), jj = jb + (d & 1);
        if (qq < kb && jj < x.cw) {
          const C2<T> v = d == 0 ? c00 : d == 1 ? c01 : d == 2 ? c10 : c11;
          const T w = cwt[slot][jj];
          const int64_t e = (qb + qq) + (int64_t)(x.j0 + jj) * x.kcap;
          if (DH2_IN(x.roff + e, c_lim.R[x.side], 11, x.pid)) x.R[e] = C2<T>{v.re * w, sg * v.im * w};
        }
      }
    }
  };

  int64_t t = blockIdx.x;
  RqLeafTile<T> cur = rq_leaf_tile(args, tiles, t, ntiles, P);
  RqLeafTile<T> nxt = rq_leaf_tile(args, tiles, t + stride, ntiles, P);
  issue_table(cur, 0);
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  issue_a(cur, 0, 0);
  issue_table(nxt, 1);
  cp_async_commit();
  for (int i = 0; t < ntiles; ++i, t += stride) {
    const int s = i & 1, slot = i % 3;
    const RqLeafTile<T> nn = rq_leaf_tile(args, tiles, t + 2 * stride, ntiles, P);
    cp_async_wait_all();
    __syncthreads();  // this tile's stage and the next tile's table have landed; stage s^1 is free
    issue_a(nxt, s ^ 1, (i + 1) % 3);
    issue_table(nn, (i + 2) % 3);
    cp_async_commit();
    if (cur.live) {
      products(cur, s, slot, 0);
      for (int qb = QB; qb < cur.k; qb += QB) {  // ranks above 32: further Q blocks, loaded in place
        __syncthreads();
        issue_q(cur, s, qb);
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        products(cur, s, slot, qb);
      }
    }
    cur = nxt;
    nxt = nn;
  }
  cp_async_wait_all();
}

// Dynamic shared memory of `smem` bytes for kern, checked against the
// device's opt-in limit (false: the launch cannot run, nothing was launched).
template <typename K>
bool set_smem(K kern, size_t smem) {
  int dev = 0, maxopt = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      smem > (size_t)maxopt || cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

template <typename T, int P_T, bool FROM_R, int NT, bool GRAM = false>
bool launch_one(const PairArgs<T>* args, const uint32_t* codes, int nblocks, int P, cudaStream_t st,
                const int* count = nullptr, const uint64_t* segs = nullptr) {
  constexpr int C = 16 * (NT / P_T);
  constexpr int XTRA = GRAM ? 0 : C;
  const int LDL = P + 1;
  size_t smem = (GRAM ? 0 : (((size_t)(P + XTRA) * LDL * sizeof(C2<T>) + 15) & ~(size_t)15) + 2 * C * sizeof(C2<T>)) +
                (size_t)P * sizeof(double) + 2 * (size_t)P * sizeof(int) + (size_t)P * sizeof(T);
  if (GRAM) smem = ((smem + 15) & ~(size_t)15) + (size_t)P * P * sizeof(float4) + (size_t)P * (sizeof(float) + sizeof(int));
  auto kern = pair_kernel<T, P_T, FROM_R, NT, GRAM>;
#ifdef DH2_PROFILE
  // DH2_PROFILE_SOLO=1: one CTA per SM, so the phase counters show latency
  // without the contention of co-resident pairs
  if (const char* solo = getenv("DH2_PROFILE_SOLO"))
    if (solo[0] == '1' && smem < 120 * 1024) smem = 120 * 1024;
#endif
  if (!set_smem(kern, smem)) return false;
  kern<<<nblocks, NT, smem, st>>>(args, codes, P, count, segs);
  return true;
}

}  // namespace

void check_set_limits_pair(const CheckLimits& l) {
#ifdef DH2_CHECK
  cudaMemcpyToSymbol(c_lim, &l, sizeof(l));
  CheckRecord z{};
  cudaMemcpyToSymbol(g_chk, &z, sizeof(z));
#else
  (void)l;
#endif
}

bool check_read_pair(CheckRecord* out) {
#ifdef DH2_CHECK
  cudaMemcpyFromSymbol(out, g_chk, sizeof(*out));
  return out->count != 0;
#else
  (void)out;
  return false;
#endif
}

void prof_reset_pair() {
#ifdef DH2_PROFILE
  unsigned long long z[17] = {};
  cudaMemcpyToSymbol(g_prof, z, sizeof(z));
#endif
}

bool prof_read_pair(unsigned long long* out17) {
#ifdef DH2_PROFILE
  cudaMemcpyFromSymbol(out17, g_prof, 17 * sizeof(unsigned long long));
  return true;
#else
  (void)out17;
  return false;
#endif
}

// Non-leaf pairs of one level by row count p = k_t1c' + k_t2c' (known only
// once the sons' ranks are): class 0..3 for p <= 32, <= 48, <= 64, more.
// out holds 4 segments of n codes; counts[c] the class sizes.
template <typename T>
__global__ void classify_kernel(const PairArgs<T>* __restrict__ args, const uint32_t* __restrict__ codes, int n,
                                uint32_t* __restrict__ out, int* __restrict__ counts) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t code = codes[i];
  const PairArgs<T>& a = args[code >> kCodeProbShift];
  const int side = (int)((code >> kCodeSideShift) & 1u);
  const int pid = (int)(code & kCodePairMask);
  const int p = a.rank[side][a.son[side][2 * pid]] + a.rank[side][a.son[side][2 * pid + 1]];
  const int cls = p <= 32 ? 0 : p <= 48 ? 1 : p <= 64 ? 2 : 3;
  out[(int64_t)cls * n + atomicAdd(&counts[cls], 1)] = code;
}

// the same classes for the segment entries (code << 32 | segment) of wide pairs
template <typename T>
__global__ void classify_seg_kernel(const PairArgs<T>* __restrict__ args, const uint64_t* __restrict__ segs, int n,
                                    uint64_t* __restrict__ out, int* __restrict__ counts) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t e = segs[i];
  const uint32_t code = (uint32_t)(e >> 32);
  const PairArgs<T>& a = args[code >> kCodeProbShift];
  const int side = (int)((code >> kCodeSideShift) & 1u);
  const int pid = (int)(code & kCodePairMask);
  const int p = a.rank[side][a.son[side][2 * pid]] + a.rank[side][a.son[side][2 * pid + 1]];
  const int cls = p <= 32 ? 0 : p <= 48 ? 1 : p <= 64 ? 2 : 3;
  out[(int64_t)cls * n + atomicAdd(&counts[cls], 1)] = e;
}

template <typename T, bool FROM_R>
bool launch_rq(const PairArgs<T>* args, const uint64_t* tiles, int ntiles, int P, cudaStream_t st) {
  const size_t smem = (size_t)(32 + 2 + kRTile + 2) * P * sizeof(C2<T>);  // row-major Q block and A tile
  auto kern = rq_kernel<T, FROM_R>;
  if (!set_smem(kern, smem)) return false;
  kern<<<ntiles, 128, smem, st>>>(args, tiles, P);
  return true;
}

template <typename T>
bool launch_rq_leaf(const PairArgs<T>* args, const uint64_t* tiles, int ntiles, int P, cudaStream_t st) {
  constexpr int QB = 16, LQ = QB + 2, LA = kRTile + 2;
  const size_t smem = 2 * (size_t)(LQ + LA) * P * sizeof(C2<T>);  // two stages of Q block and A tile
  auto kern = rq_leaf_kernel<T>;
  if (!set_smem(kern, smem)) return false;
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, smem);
  const int cap = tune_current().rq_ctas_per_sm;  // the tuning table's choice, within the occupancy limit
  if (cap > 0 && cap < per_sm) per_sm = cap;
  const int grid = (int)std::min<int64_t>(ntiles, (int64_t)std::max(1, nsm) * std::max(1, per_sm));
  kern<<<grid, 128, smem, st>>>(args, tiles, (int64_t)ntiles, P);
  return true;
}

template <typename T>
bool launch_rq_kernel(const PairArgs<T>* args, const uint64_t* tiles, int ntiles, int P, bool from_r, bool gen,
                      cudaStream_t st) {
  if (ntiles <= 0) return true;
  if (from_r) return launch_rq<T, true>(args, tiles, ntiles, P, st);
  if (gen) return launch_rq<T, false>(args, tiles, ntiles, P, st);
  return launch_rq_leaf<T>(args, tiles, ntiles, P, st);
}
template <typename T>
void launch_classify(const PairArgs<T>* args, const uint32_t* codes, int n, uint32_t* out, int* counts,
                     cudaStream_t st) {
  if (n > 0) classify_kernel<T><<<(n + 255) / 256, 256, 0, st>>>(args, codes, n, out, counts);
}
template <typename T>
void launch_classify_seg(const PairArgs<T>* args, const uint64_t* segs, int n, uint64_t* out, int* counts,
                         cudaStream_t st) {
  if (n > 0) classify_seg_kernel<T><<<(n + 255) / 256, 256, 0, st>>>(args, segs, n, out, counts);
}
template void launch_classify_seg<float>(const PairArgs<float>*, const uint64_t*, int, uint64_t*, int*, cudaStream_t);
template void launch_classify_seg<double>(const PairArgs<double>*, const uint64_t*, int, uint64_t*, int*,
                                          cudaStream_t);
template void launch_classify<float>(const PairArgs<float>*, const uint32_t*, int, uint32_t*, int*, cudaStream_t);
template void launch_classify<double>(const PairArgs<double>*, const uint32_t*, int, uint32_t*, int*, cudaStream_t);

template bool launch_rq_kernel<float>(const PairArgs<float>*, const uint64_t*, int, int, bool, bool, cudaStream_t);
template bool launch_rq_kernel<double>(const PairArgs<double>*, const uint64_t*, int, int, bool, bool, cudaStream_t);

template <typename T>
bool launch_pair_kernel(const PairArgs<T>* args, const uint32_t* codes, int nblocks, int P, bool from_r,
                        cudaStream_t st, const int* count, const uint64_t* segs) {
  if (nblocks <= 0) return true;
  if (!from_r) {
    if (P <= 32) return launch_one<T, 32, false, 128>(args, codes, nblocks, P, st, count);
    if (P <= 40) return launch_one<T, 40, false, 160>(args, codes, nblocks, P, st, count);
    if (P <= 48) return launch_one<T, 48, false, 192>(args, codes, nblocks, P, st, count);
    if (P <= 64) return launch_one<T, 64, false, 256>(args, codes, nblocks, P, st, count);
    return launch_one<T, 128, false, 256>(args, codes, nblocks, P, st, count);
  }
  if (P <= 32) return launch_one<T, 32, true, 128>(args, codes, nblocks, P, st, count, segs);
  if (P <= 48) return launch_one<T, 48, true, 192>(args, codes, nblocks, P, st, count, segs);
  if (P <= 64) return launch_one<T, 64, true, 256>(args, codes, nblocks, P, st, count, segs);
  return launch_one<T, 128, true, 256>(args, codes, nblocks, P, st, count, segs);
}

// The Jacobi launch of a class: NT = 4 x rows threads per CTA, or (the
// tuning table's narrow choices) NTN, a multiple of 32 near 2 x rows, or NTM
// near 1 x rows, with the same threads per SM (about twice or four times the
// CTAs, so more pairs at once; at most 32 CTAs per SM).
template <int P_T, int NT, int NTN, int NTM>
bool launch_gram_factor(const PairArgs<float>* args, const uint32_t* codes, int nblocks, int P, cudaStream_t st) {
  static_assert(NT % 32 == 0 && NTN % 32 == 0 && NTM % 32 == 0 && NTM >= P_T,
                "whole warps (the Jacobi reductions run converged), one thread per column of the rank step");
  if (!launch_one<float, P_T, false, NT, true>(args, codes, nblocks, P, st)) return false;
  const size_t smem = (((size_t)P * (P + 1) * sizeof(C2<float>) + 15) & ~(size_t)15) + (size_t)P * sizeof(double) +
                      (size_t)P * sizeof(int);
  constexpr int MINB = 2048 / NT - 4;
  const int narrow = tune_current().jacobi_narrow[factor_class(P_T)];
  if (narrow == 2) {
    constexpr int MB = NT * MINB / NTM < 32 ? NT * MINB / NTM : 32;
    auto kern = gram_jacobi_kernel<P_T, NTM, MB>;
    if (!set_smem(kern, smem)) return false;
    kern<<<nblocks, NTM, smem, st>>>(args, codes, P);
  } else if (narrow == 1) {
    auto kern = gram_jacobi_kernel<P_T, NTN, NT * MINB / NTN>;
    if (!set_smem(kern, smem)) return false;
    kern<<<nblocks, NTN, smem, st>>>(args, codes, P);
  } else {
    auto kern = gram_jacobi_kernel<P_T, NT, MINB>;
    if (!set_smem(kern, smem)) return false;
    kern<<<nblocks, NT, smem, st>>>(args, codes, P);
  }
  return true;
}

bool launch_pair_kernel_gram(const PairArgs<float>* args, const uint32_t* codes, int nblocks, int P, cudaStream_t st) {
  if (nblocks <= 0) return true;
  if (P <= 32) return launch_gram_factor<32, 128, 64, 32>(args, codes, nblocks, P, st);
  if (P <= 40) return launch_gram_factor<40, 160, 96, 64>(args, codes, nblocks, P, st);
  if (P <= 48) return launch_gram_factor<48, 192, 96, 64>(args, codes, nblocks, P, st);
  if (P <= 64) return launch_gram_factor<64, 256, 128, 64>(args, codes, nblocks, P, st);
  return false;
}

template bool launch_pair_kernel<float>(const PairArgs<float>*, const uint32_t*, int, int, bool, cudaStream_t,
                                        const int*, const uint64_t*);
template bool launch_pair_kernel<double>(const PairArgs<double>*, const uint32_t*, int, int, bool, cudaStream_t,
                                         const int*, const uint64_t*);

}  // namespace dh2
