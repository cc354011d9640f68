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
//      and k, and
//   5. streams A once more through shared memory to form R_tc = Q^* A
//      (Section 6, R recursion).
#include <cfloat>

#include "dh2_check.cuh"
#include "dh2_internal.h"
#include "dh2_kernels.cuh"

namespace dh2 {

namespace {

DH2_CHECK_DECLS

#ifdef DH2_PROFILE
// per-phase clock cycles summed over CTAs: LQ, Jacobi, rank+Q, R; sweeps; pairs
__device__ unsigned long long g_prof[8];
#define DH2_PROF_T(v) const long long v = clock64()
#define DH2_PROF_ADD(i, v) \
  if (threadIdx.x == 0) atomicAdd(&g_prof[i], (unsigned long long)(v))
#else
#define DH2_PROF_T(v)
#define DH2_PROF_ADD(i, v)
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

// Element (r, j) of the pair's matrix A (row r of the factor, column j of F_tc).
template <typename T, bool FROM_R>
struct Source {
  int side, pid;
  // leaf
  const C2<T>* G;
  int64_t ld;
  int r0;
  const int32_t* gcol;
  const int32_t* gblk;
  const double* invw;
  int64_t cmo;
  const double* pts;  // matrix-free mode
  double kappa, diag;
  int gen;
  // non-leaf
  const C2<T>* R0;
  const C2<T>* R1;
  int64_t roff0, roff1;
  int k1, off0, off1, ld0, ld1;

  __device__ __forceinline__ C2<T> get(int r, int j) const {
    if (FROM_R) {
      if (r < k1) {
        const int64_t e = (int64_t)(off0 + j) * ld0 + r;
        if (!DH2_IN(roff0 + e, c_lim.R[side], 1, pid)) return czero<T>();
        return R0[e];
      }
      const int64_t e = (int64_t)(off1 + j) * ld1 + (r - k1);
      if (!DH2_IN(roff1 + e, c_lim.R[side], 2, pid)) return czero<T>();
      return R1[e];
    } else {
      if (!DH2_IN(cmo + j, c_lim.ncol[side], 3, pid)) return czero<T>();
      const int gc = gcol[j];
      const int b = gblk[j];
      if (!DH2_IN(b, c_lim.nblocks, 4, pid)) return czero<T>();
      const T w = (T)invw[b];
      if (gen) {
        C2<T> g = side == 0 ? helmholtz_entry<T>(pts, r0 + r, gc, kappa, diag)
                            : helmholtz_entry<T>(pts, gc, r0 + r, kappa, diag);
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
  }
};

// P_T: largest factor size of the instantiation (64 or 128 rows).
template <typename T, int P_T, bool FROM_R>
#ifndef DH2_PAIR_MINB
#define DH2_PAIR_MINB 3
#endif
#ifndef DH2_LEAF_CHUNK
#define DH2_LEAF_CHUNK 64
#endif
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? DH2_PAIR_MINB : 1)
    pair_kernel(const PairArgs<T>* __restrict__ args, const uint32_t* __restrict__ codes, const int P) {
  constexpr int NT = 256;
  constexpr int LPR = NT / P_T;      // threads per row in the LQ
  constexpr int C = P_T == 64 ? DH2_LEAF_CHUNK : 32;
  constexpr int CPL = C / LPR;       // chunk entries per thread
  constexpr int XTRA = 16;           // spare L columns used to stage R chunks
  static_assert(C % LPR == 0, "chunk width must split over the threads of a row");
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ C2<T> sh_v0[2];
  __shared__ T sh_tau[2];
  __shared__ int sh_skip[2];
  __shared__ int sh_rot[2];
  __shared__ int sh_k;
  __shared__ int sh_piv;
  __shared__ double sh_E;

  const int LDL = P + 1;              // column-major L: element (r, c) at c * LDL + r
  C2<T>* Lm = reinterpret_cast<C2<T>*>(smem);
  size_t soff = ((size_t)(P + XTRA) * LDL * sizeof(C2<T>) + 15) & ~(size_t)15;
  C2<T>* vbuf = reinterpret_cast<C2<T>*>(smem + soff);  // 2 x C reflector rows
  soff += 2 * C * sizeof(C2<T>);
  double* sig2 = reinterpret_cast<double*>(smem + soff);
  soff += (size_t)P * sizeof(double);
  int* ord = reinterpret_cast<int*>(smem + soff);
  soff += (size_t)P * sizeof(int);
  int* perm = reinterpret_cast<int*>(smem + soff);  // row permutation of the pivoted LQ
  soff += (size_t)P * sizeof(int);
  T* nu = reinterpret_cast<T*>(smem + soff);         // residual row norms

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t code = codes[blockIdx.x];
  const int prob = (int)(code >> kCodeProbShift);
  const int side = (int)((code >> kCodeSideShift) & 1u);
  const int pid = (int)(code & kCodePairMask);
  const PairArgs<T>& a = args[prob];
  if (!DH2_IN(pid, c_lim.npairs[side], 9, pid)) return;
  const int N = a.ncols[side][pid];
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
    src.gblk = a.gblk[side] + src.cmo;
    src.G = a.G;
    src.ld = a.ld;
    src.invw = a.invw;
    src.pts = a.pts;
    src.kappa = a.kappa;
    src.diag = a.diag;
    src.gen = a.gen;
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

  for (int i = tid; i < (P + XTRA) * LDL; i += NT) Lm[i] = czero<T>();
  DH2_PROF_T(t_a);

  // ---------------------------------------------------------------- 1. LQ
  const int row = tid / LPR, q = tid % LPR;
  const unsigned gmask = (LPR == 32) ? 0xffffffffu : (((1u << LPR) - 1u) << (lane & ~(LPR - 1)));
  const bool live = row < p;
  C2<T> ch[CPL];

  // Householder reflection of row i (held by its LPR threads) from the right:
  // the row becomes (beta, 0, ..., 0) on the columns {i} u chunk,
  // beta = -e^{i arg alpha} |x|; the chunk part goes to vbuf[slot].
  auto make_reflector = [&](int i, int slot) {
    T s0 = T(0), s1 = T(0);
#pragma unroll
    for (int u = 0; u < CPL; u += 2) {
      s0 += cnorm2(ch[u]);
      s1 += cnorm2(ch[u + 1]);
      vbuf[slot * C + q + u * LPR] = ch[u];
      vbuf[slot * C + q + (u + 1) * LPR] = ch[u + 1];
    }
    T s = s0 + s1;
#pragma unroll
    for (int o = 1; o < LPR; o <<= 1) s += __shfl_xor_sync(gmask, s, o);
    if (q == 0) {
      if (!(s > Eps<T>::tiny)) {
        sh_skip[slot] = 1;
      } else {
        const C2<T> al = Lm[i * LDL + i];
        const T an2 = cnorm2(al);
        const T ra = an2 > Eps<T>::tiny ? frsqrt(an2) : T(0);
        const T an = an2 * ra;
        const T xn2 = s + an2;
        const T xn = xn2 * frsqrt(xn2);
        const C2<T> ph = an2 > Eps<T>::tiny ? C2<T>{al.re * ra, al.im * ra} : C2<T>{T(1), T(0)};
        Lm[i * LDL + i] = C2<T>{-ph.re * xn, -ph.im * xn};
        sh_v0[slot] = C2<T>{ph.re * (an + xn), -ph.im * (an + xn)};
        sh_tau[slot] = fdiv(T(1), xn * (xn + an));
        sh_skip[slot] = 0;
      }
    }
  };

  for (int j0 = 0; j0 < N; j0 += C) {
    const int cw = min(C, N - j0);
#pragma unroll
    for (int u = 0; u < CPL; ++u) {
      const int jj = q + u * LPR;
      ch[u] = (live && jj < cw) ? src.get(row, j0 + jj) : czero<T>();
    }
    __syncthreads();  // L zeroed / previous chunk's last reflector consumed
    if (row == 0) make_reflector(0, 0);
    __syncthreads();
    for (int i = 0; i < p; ++i) {
      const int sl = i & 1;
      if (!sh_skip[sl] && row > i && live) {
        const C2<T> v0 = sh_v0[sl];
        const T tau = sh_tau[sl];
        const C2<T>* xi = vbuf + sl * C;
        C2<T> w = czero<T>(), w1 = czero<T>();
        if (q == 0) w = cmul(Lm[i * LDL + row], v0);
#pragma unroll
        for (int u = 0; u < CPL; u += 2) {
          w = cadd(w, cmulc(ch[u], xi[q + u * LPR]));
          w1 = cadd(w1, cmulc(ch[u + 1], xi[q + (u + 1) * LPR]));
        }
        w = cadd(w, w1);
#pragma unroll
        for (int o = 1; o < LPR; o <<= 1) {
          w.re += __shfl_xor_sync(gmask, w.re, o);
          w.im += __shfl_xor_sync(gmask, w.im, o);
        }
        const C2<T> tw = C2<T>{tau * w.re, tau * w.im};
#pragma unroll
        for (int u = 0; u < CPL; ++u) ch[u] = csub(ch[u], cmul(tw, xi[q + u * LPR]));
        if (q == 0) Lm[i * LDL + row] = csub(Lm[i * LDL + row], cmulc(tw, v0));
      }
      if (row == i + 1 && live) make_reflector(i + 1, (i + 1) & 1);
      __syncthreads();
    }
  }

  DH2_PROF_T(t_b);
  DH2_PROF_ADD(0, t_b - t_a);

  // ---------------------------------------------------------------- 1b. pivoted LQ of L
  // Rank-revealing step: L = Pi^T L' Omega' by Householder reflections from
  // the right with row pivoting (largest residual row first).  It stops at the
  // first K whose remaining block L'(K:, K:) has energy E_K <= drop * eps_l^2;
  // that energy is added to every tail sum below (an upper bound on the
  // residual of the chosen subspace), and the Jacobi step works on the K
  // leading columns only.  Pi is kept in perm[].
  const double drop = sizeof(T) == 4 ? 1e-2 : 1e-10;
  const double tau_drop = drop * a.eps2[lvl];
  for (int r = tid; r < P; r += NT) perm[r] = r;
  int K = p;
  double E_K = 0.0;
  for (int i = 0; i < p; ++i) {
    // residual row norms over columns i..p-1 (row i-1 becomes final: zero its tail)
    if (i > 0 && row == i - 1)
      for (int c = i + q; c < p; c += LPR) Lm[c * LDL + row] = czero<T>();
    if (row >= i && live) {
      T s = T(0);
      for (int c = i + q; c < p; c += LPR) s += cnorm2(Lm[c * LDL + row]);
#pragma unroll
      for (int o = 1; o < LPR; o <<= 1) s += __shfl_xor_sync(gmask, s, o);
      if (q == 0) nu[row] = s;
    }
    __syncthreads();
    if (warp == 0) {
      double e = 0.0;
      T best = T(-1);
      int bi = i;
      for (int r = i + lane; r < p; r += 32) {
        const T v = nu[r];
        e += (double)v;
        if (v > best) {
          best = v;
          bi = r;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_xor_sync(0xffffffffu, e, o);
        const T ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (lane == 0) {
        sh_E = e;
        sh_piv = bi;
      }
    }
    __syncthreads();
    if (sh_E <= tau_drop) {
      K = i;
      E_K = sh_E;
      break;
    }
    const int pv = sh_piv;
    if (pv != i) {
      for (int c = tid; c < p; c += NT) {
        const C2<T> t0 = Lm[c * LDL + i];
        Lm[c * LDL + i] = Lm[c * LDL + pv];
        Lm[c * LDL + pv] = t0;
      }
      if (tid == 0) {
        const int t1 = perm[i];
        perm[i] = perm[pv];
        perm[pv] = t1;
      }
    }
    __syncthreads();
    if (row == i) {
      // reflector of row i over columns i..p-1
      T s = T(0);
      for (int c = i + 1 + q; c < p; c += LPR) s += cnorm2(Lm[c * LDL + i]);
#pragma unroll
      for (int o = 1; o < LPR; o <<= 1) s += __shfl_xor_sync(gmask, s, o);
      if (q == 0) {
        if (!(s > Eps<T>::tiny)) {
          sh_skip[0] = 1;
        } else {
          const C2<T> al = Lm[i * LDL + i];
          const T an2 = cnorm2(al);
          const T ra = an2 > Eps<T>::tiny ? frsqrt(an2) : T(0);
          const T an = an2 * ra;
          const T xn2 = s + an2;
          const T xn = xn2 * frsqrt(xn2);
          const C2<T> ph = an2 > Eps<T>::tiny ? C2<T>{al.re * ra, al.im * ra} : C2<T>{T(1), T(0)};
          Lm[i * LDL + i] = C2<T>{-ph.re * xn, -ph.im * xn};
          sh_v0[0] = C2<T>{ph.re * (an + xn), -ph.im * (an + xn)};
          sh_tau[0] = fdiv(T(1), xn * (xn + an));
          sh_skip[0] = 0;
        }
      }
    }
    __syncthreads();
    if (!sh_skip[0] && row > i && live) {
      const C2<T> v0 = sh_v0[0];
      const T tau = sh_tau[0];
      C2<T> w = czero<T>();
      if (q == 0) w = cmul(Lm[i * LDL + row], v0);
      for (int c = i + 1 + q; c < p; c += LPR) w = cadd(w, cmulc(Lm[c * LDL + row], Lm[c * LDL + i]));
#pragma unroll
      for (int o = 1; o < LPR; o <<= 1) {
        w.re += __shfl_xor_sync(gmask, w.re, o);
        w.im += __shfl_xor_sync(gmask, w.im, o);
      }
      const C2<T> tw = C2<T>{tau * w.re, tau * w.im};
      for (int c = i + 1 + q; c < p; c += LPR)
        Lm[c * LDL + row] = csub(Lm[c * LDL + row], cmul(tw, Lm[c * LDL + i]));
      if (q == 0) Lm[i * LDL + row] = csub(Lm[i * LDL + row], cmulc(tw, v0));
    }
    __syncthreads();
  }
  // the last processed row keeps its (already applied) tail: zero it; with K
  // odd, column K holds residual entries and is cleared for the pairing
  if (K > 0 && row == K - 1)
    for (int c = K + q; c < p; c += LPR) Lm[c * LDL + row] = czero<T>();
  __syncthreads();
  if ((K & 1) && K < P)
    for (int r = tid; r < p; r += NT) Lm[K * LDL + r] = czero<T>();
  __syncthreads();
  // ---------------------------------------------------------------- 2. Jacobi
  // one column pair per group of 8 threads; round-robin ordering over pe columns
  const int pe = K + (K & 1);
  const T tol = T(p) * Eps<T>::u;
  const int grp = tid >> 3, gl = tid & 7;
  const unsigned m8 = 0xffu << (lane & 24);
  if (tid == 0) {
    sh_rot[0] = 0;
    sh_rot[1] = 0;
  }
  __syncthreads();
  bool conv = pe < 2;
  int nsweeps = 0;
  for (int sweep = 0; sweep < a.max_sweeps && pe >= 2; ++sweep) {
    ++nsweeps;
    const int sp = sweep & 1;
    // round-robin positions of this group's pairs in round 0; each round
    // moves every position but the fixed one (index 0) by one place
    int ia[P_T / 64], ib[P_T / 64];
#pragma unroll
    for (int h = 0; h < P_T / 64; ++h) {
      const int kk = grp + h * (NT / 8);
      ia[h] = kk;
      ib[h] = pe - 1 - kk;
    }
    for (int rd = 0; rd < pe - 1; ++rd) {
#pragma unroll
      for (int h = 0; h < P_T / 64; ++h) {
        const int kk = grp + h * (NT / 8);
        if (kk < pe / 2) {
          C2<T>* ca = Lm + ia[h] * LDL;
          C2<T>* cb = Lm + ib[h] * LDL;
          T al = T(0), be = T(0);
          C2<T> ga = czero<T>();
          for (int r = gl; r < p; r += 8) {
            const C2<T> xa = ca[r], xb = cb[r];
            al += cnorm2(xa);
            be += cnorm2(xb);
            ga = cadd(ga, cmulc(xb, xa));  // conj(xa) * xb
          }
#pragma unroll
          for (int o = 1; o < 8; o <<= 1) {
            al += __shfl_xor_sync(m8, al, o);
            be += __shfl_xor_sync(m8, be, o);
            ga.re += __shfl_xor_sync(m8, ga.re, o);
            ga.im += __shfl_xor_sync(m8, ga.im, o);
          }
          const T g2 = cnorm2(ga);
          // rotate unless the pair is orthogonal to tol (relative)
          if (al > Eps<T>::tiny && be > Eps<T>::tiny && g2 > T(0) &&
              sqrt(g2) * frsqrt(al) * frsqrt(be) > tol) {
            const T rg = frsqrt(g2);
            const T zt = (be - al) * T(0.5) * rg;
            const T t = (zt >= T(0) ? T(1) : T(-1)) / (fabs(zt) + sqrt(T(1) + zt * zt));
            const T c = T(1) / sqrt(T(1) + t * t);
            const T s = t * c;
            if (s != T(0)) {
              const C2<T> e = C2<T>{ga.re * rg, -ga.im * rg};  // e^{-i arg gamma}
              for (int r = gl; r < p; r += 8) {
                const C2<T> xa = ca[r];
                const C2<T> eb = cmul(e, cb[r]);
                ca[r] = C2<T>{c * xa.re - s * eb.re, c * xa.im - s * eb.im};
                cb[r] = C2<T>{s * xa.re + c * eb.re, s * xa.im + c * eb.im};
              }
              if (gl == 0) sh_rot[sp] = 1;
            }
          }
          if (kk > 0) ia[h] = ia[h] == pe - 1 ? 1 : ia[h] + 1;
          ib[h] = ib[h] == pe - 1 ? 1 : ib[h] + 1;
        }
      }
      __syncthreads();
      if (rd == 0 && tid == 0) sh_rot[sp ^ 1] = 0;
    }
    const int rot = sh_rot[sp];
    __syncthreads();
    if (rot == 0) {
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
  for (int j = grp; j < K; j += NT / 8) {
    double s = 0.0;
    for (int r = gl; r < p; r += 8) {
      const C2<T> x = Lm[j * LDL + r];
      s += (double)x.re * (double)x.re + (double)x.im * (double)x.im;
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) s += __shfl_xor_sync(m8, s, o);
    if (gl == 0) sig2[j] = s;
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
    const T inv = (T)(1.0 / sqrt(sig2[j]));
    for (int r = gl; r < p; r += 8) {
      const C2<T> v = Lm[j * LDL + r];
      const int ro = perm[r];
      if (DH2_IN(a.Qoff[side][pid] + ro + (int64_t)qq * ldq, c_lim.Q[side], 10, pid))
        Qout[ro + (int64_t)qq * ldq] = C2<T>{v.re * inv, v.im * inv};
    }
  }
  if (k == 0) return;
  __syncthreads();
  // compact Q into L columns 0..k-1 (re-read from global, visible after the barrier)
  for (int idx = tid; idx < p * k; idx += NT) {
    const int r = idx % p, qq = idx / p;
    Lm[qq * LDL + r] = Qout[r + (int64_t)qq * ldq];
  }
  __syncthreads();

  DH2_PROF_T(t_d);
  DH2_PROF_ADD(2, t_d - t_c);
  // ---------------------------------------------------------------- 5. R = Q^* A
  C2<T>* Rout = a.R[side] + a.Roff[side][pid];
  const int CR = min(64, (P + XTRA - k)) & ~7;  // staged columns after Q
  C2<T>* Ast = Lm + (int64_t)k * LDL;
  for (int j0 = 0; j0 < N; j0 += CR) {
    const int cw = min(CR, N - j0);
    if (FROM_R || side == 0) {
      for (int jj = warp; jj < cw; jj += NT / 32)
        for (int r = lane; r < p; r += 32) Ast[jj * LDL + r] = src.get(r, j0 + jj);
    } else {
      for (int r = warp; r < p; r += NT / 32)
        for (int jj = lane; jj < cw; jj += 32) Ast[jj * LDL + r] = src.get(r, j0 + jj);
    }
    __syncthreads();
    for (int idx = tid; idx < k * cw; idx += NT) {
      const int qq = idx % k, jj = idx / k;
      const C2<T>* qc = Lm + qq * LDL;
      const C2<T>* ac = Ast + jj * LDL;
      C2<T> acc = czero<T>();
      for (int r = 0; r < p; ++r) acc = cadd(acc, cmulc(ac[r], qc[r]));
      if (DH2_IN(a.Roff[side][pid] + qq + (int64_t)(j0 + jj) * kcap, c_lim.R[side], 11, pid))
        Rout[qq + (int64_t)(j0 + jj) * kcap] = acc;
    }
    __syncthreads();
  }
  DH2_PROF_T(t_e);
  DH2_PROF_ADD(3, t_e - t_d);
}

template <typename T, int P_T, bool FROM_R>
void launch_one(const PairArgs<T>* args, const uint32_t* codes, int nblocks, int P, cudaStream_t st) {
  constexpr int C = P_T == 64 ? DH2_LEAF_CHUNK : 32;
  const int LDL = P + 1;
  size_t smem = (((size_t)(P + 16) * LDL * sizeof(C2<T>) + 15) & ~(size_t)15) + 2 * C * sizeof(C2<T>) +
                (size_t)P * sizeof(double) + 2 * (size_t)P * sizeof(int) + (size_t)P * sizeof(T);
  auto kern = pair_kernel<T, P_T, FROM_R>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kern<<<nblocks, 256, smem, st>>>(args, codes, P);
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
  unsigned long long z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  cudaMemcpyToSymbol(g_prof, z, sizeof(z));
#endif
}

bool prof_read_pair(unsigned long long* out8) {
#ifdef DH2_PROFILE
  cudaMemcpyFromSymbol(out8, g_prof, 8 * sizeof(unsigned long long));
  return true;
#else
  (void)out8;
  return false;
#endif
}

template <typename T>
void launch_pair_kernel(const PairArgs<T>* args, const uint32_t* codes, int nblocks, int P, bool from_r,
                        cudaStream_t st) {
  if (nblocks <= 0) return;
  if (!from_r) {
    if (P <= 64) launch_one<T, 64, false>(args, codes, nblocks, P, st);
    else launch_one<T, 128, false>(args, codes, nblocks, P, st);
  } else {
    if (P <= 64) launch_one<T, 64, true>(args, codes, nblocks, P, st);
    else launch_one<T, 128, true>(args, codes, nblocks, P, st);
  }
}

template void launch_pair_kernel<float>(const PairArgs<float>*, const uint32_t*, int, int, bool, cudaStream_t);
template void launch_pair_kernel<double>(const PairArgs<double>*, const uint32_t*, int, int, bool, cudaStream_t);

}  // namespace dh2
