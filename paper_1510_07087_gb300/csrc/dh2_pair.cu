// Per-(cluster, direction) factorisation kernel: the leaf step and the
// non-leaf step of procedure basis() (Section 6), one CTA per pair.
//
// For a pair (t, c) the kernel
//   1. streams the columns of its matrix A -- G^omega_tc restricted to the
//      rows of t for a leaf (Section 6 leaf step, weights of Remark "Error
//      control"), or Ghat_tc = [R_t1c'|F_tc ; R_t2c'|F_tc] for a non-leaf
//      (Eq. hatQ_hatG) -- through shared memory in chunks of C columns and
//      reduces it to a p x p lower-triangular factor L with A = L Omega,
//      Omega with orthonormal rows (an LQ factorisation by Householder
//      reflections applied chunk by chunk, so the Gram matrix A A^* is never
//      formed and singular values are not squared);
//   2. runs one-sided (Hestenes) Jacobi on the columns of L: L J = U Sigma,
//      so the normalised columns are the left singular vectors of A and their
//      norms its singular values;
//   3. chooses the rank k = min{k : sum_{i>k} sigma_i^2 <= eps_l^2} with the
//      tail sums formed in FP64;
//   4. writes Q = first k left singular vectors (Q_tc for a leaf, the stacked
//      transfer matrices [E_t1c; E_t2c] for a non-leaf), the singular values
//      and k, and
//   5. streams A once more to form R_tc = Q^* A (Section 6, R recursion).
#include <cfloat>

#include "dh2_check.cuh"
#include "dh2_internal.h"
#include "dh2_kernels.cuh"

namespace dh2 {

namespace {

DH2_CHECK_DECLS

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

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T, int C, int LPR, bool FROM_R>
__global__ void __launch_bounds__(256) pair_kernel(const PairArgs<T> a) {
  constexpr int NT = 256;
  constexpr int NW = NT / 32;
  constexpr int CPL = C / LPR;  // chunk columns per thread in the LQ updates
  static_assert(C % LPR == 0, "chunk width must split over the lanes of a row");
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ C2<T> sh_v0[2];
  __shared__ T sh_tau[2];
  __shared__ int sh_skip[2];
  __shared__ int sh_rot[2];
  __shared__ int sh_k;

  const int P = a.P;
  const int LDX = P + C + 1;
  C2<T>* X = reinterpret_cast<C2<T>*>(smem);
  size_t soff = ((size_t)P * LDX * sizeof(C2<T>) + 15) & ~(size_t)15;
  double* sig2 = reinterpret_cast<double*>(smem + soff);
  soff += (size_t)P * sizeof(double);
  int* ord = reinterpret_cast<int*>(smem + soff);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int code = a.order[blockIdx.x];
  const int side = code >> 30;
  const int pid = code & 0x3fffffff;
  const int N = a.ncols[side][pid];
  const int kcap = a.kcap[side][pid];
  const int lvl = a.level[side][pid];
  int p = 0, k1 = 0, off0 = 0, off1 = 0, ld0 = 1, ld1 = 1, r0 = 0;
  const C2<T>* R0 = nullptr;
  const C2<T>* R1 = nullptr;
  int64_t roff0 = 0, roff1 = 0;
  const int32_t* gcol = nullptr;
  const int32_t* gblk = nullptr;
  if (FROM_R) {
    const int s0 = a.son[side][2 * pid], s1 = a.son[side][2 * pid + 1];
    if (!DH2_IN(s0, c_lim.npairs[side], 12, pid) || !DH2_IN(s1, c_lim.npairs[side], 13, pid)) return;
    k1 = a.rank[side][s0];
    p = k1 + a.rank[side][s1];
    off0 = a.sonoff[side][2 * pid];
    off1 = a.sonoff[side][2 * pid + 1];
    ld0 = a.kcap[side][s0];
    ld1 = a.kcap[side][s1];
    roff0 = a.Roff[side][s0];
    roff1 = a.Roff[side][s1];
    R0 = a.R[side] + roff0;
    R1 = a.R[side] + roff1;
  } else {
    p = a.m[side][pid];
    r0 = a.start[side][pid];
    gcol = a.gcol[side] + a.cmoff[side][pid];
    gblk = a.gblk[side] + a.cmoff[side][pid];
  }
  const int64_t cmo = FROM_R ? 0 : a.cmoff[side][pid];
  (void)cmo;
  if (!DH2_IN(pid, c_lim.npairs[side], 9, pid)) return;
  int32_t* rank_out = a.rank[side] + pid;
  double* sig_out = a.sig[side] + (int64_t)pid * kSigStride;
  if (p > P || p > NT / LPR) {
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

  for (int i = tid; i < P * LDX; i += NT) X[i] = czero<T>();
  __syncthreads();

  // Columns j0 .. j0+C-1 of A into X[:, P .. P+C) (zero beyond N).
  auto load_chunk = [&](int j0) {
    const int cw = min(C, N - j0);
    if (FROM_R) {
      for (int jj = warp; jj < C; jj += NW) {
        const bool in = jj < cw;
        const C2<T>* c0 = R0 + (int64_t)(off0 + j0 + jj) * ld0;
        const C2<T>* c1 = R1 + (int64_t)(off1 + j0 + jj) * ld1;
        for (int r = lane; r < p; r += 32) {
          C2<T> v = czero<T>();
          if (in) {
            if (r < k1) {
              if (DH2_IN(roff0 + r + (int64_t)(off0 + j0 + jj) * ld0, c_lim.R[side], 1, pid)) v = c0[r];
            } else {
              if (DH2_IN(roff1 + (r - k1) + (int64_t)(off1 + j0 + jj) * ld1, c_lim.R[side], 2, pid)) v = c1[r - k1];
            }
          }
          X[r * LDX + P + jj] = v;
        }
      }
    } else if (side == 0) {
      // rows of t, columns from F_tc: contiguous runs down each G column
      for (int jj = warp; jj < C; jj += NW) {
        if (jj < cw && DH2_IN(cmo + j0 + jj, c_lim.ncol[side], 3, pid)) {
          const int gc = gcol[j0 + jj];
          const T w = DH2_IN(gblk[j0 + jj], c_lim.nblocks, 4, pid) ? (T)a.invw[gblk[j0 + jj]] : T(0);
          const C2<T>* col = a.G + (int64_t)gc * a.ld + r0;
          for (int r = lane; r < p; r += 32) {
            C2<T> g = czero<T>();
            if (DH2_IN((int64_t)gc * a.ld + r0 + r, c_lim.G, 5, pid)) g = col[r];
            X[r * LDX + P + jj] = C2<T>{g.re * w, g.im * w};
          }
        } else {
          for (int r = lane; r < p; r += 32) X[r * LDX + P + jj] = czero<T>();
        }
      }
    } else {
      // column basis: the same procedure on G^*; row r of A is column r0+r of G
      for (int r = warp; r < p; r += NW) {
        const C2<T>* col = a.G + (int64_t)(r0 + r) * a.ld;
        for (int jj = lane; jj < C; jj += 32) {
          C2<T> v = czero<T>();
          if (jj < cw && DH2_IN(cmo + j0 + jj, c_lim.ncol[side], 6, pid) &&
              DH2_IN((int64_t)(r0 + r) * a.ld + gcol[j0 + jj], c_lim.G, 7, pid) &&
              DH2_IN(gblk[j0 + jj], c_lim.nblocks, 8, pid)) {
            const C2<T> g = col[gcol[j0 + jj]];
            const T w = (T)a.invw[gblk[j0 + jj]];
            v = C2<T>{g.re * w, -g.im * w};
          }
          X[r * LDX + P + jj] = v;
        }
      }
    }
  };

  // ---------------------------------------------------------------- 1. LQ
  const int row = tid / LPR, q = tid % LPR;
  const unsigned gmask = (LPR == 32) ? 0xffffffffu : (((1u << LPR) - 1u) << (lane & ~(LPR - 1)));

  // Householder reflection of row i from the right: the row becomes
  // (beta, 0, ..., 0) on the columns {i} u chunk, beta = -e^{i arg alpha} |x|.
  auto make_reflector = [&](int i, int slot) {
    C2<T>* xr = X + i * LDX;
    T s = T(0);
#pragma unroll
    for (int u = 0; u < CPL; ++u) s += cnorm2(xr[P + q + u * LPR]);
#pragma unroll
    for (int o = 1; o < LPR; o <<= 1) s += __shfl_xor_sync(gmask, s, o);
    if (q == 0) {
      if (!(s > Eps<T>::tiny)) {
        sh_skip[slot] = 1;
      } else {
        const C2<T> al = xr[i];
        const T an = hypot(al.re, al.im);
        const T xn = sqrt(s + an * an);
        const C2<T> ph = an > T(0) ? C2<T>{al.re / an, al.im / an} : C2<T>{T(1), T(0)};
        xr[i] = C2<T>{-ph.re * xn, -ph.im * xn};
        sh_v0[slot] = C2<T>{ph.re * (an + xn), -ph.im * (an + xn)};
        sh_tau[slot] = T(1) / (xn * (xn + an));
        sh_skip[slot] = 0;
      }
    }
  };

  for (int j0 = 0; j0 < N; j0 += C) {
    load_chunk(j0);
    __syncthreads();
    if (row == 0) make_reflector(0, 0);
    __syncthreads();
    for (int i = 0; i < p; ++i) {
      const int sl = i & 1;
      if (!sh_skip[sl] && row > i && row < p) {
        const C2<T> v0 = sh_v0[sl];
        const T tau = sh_tau[sl];
        C2<T>* zr = X + row * LDX;
        const C2<T>* xi = X + i * LDX + P;
        C2<T> w = czero<T>();
        if (q == 0) w = cmul(zr[i], v0);
#pragma unroll
        for (int u = 0; u < CPL; ++u) {
          const int jj = q + u * LPR;
          w = cadd(w, cmulc(zr[P + jj], xi[jj]));
        }
#pragma unroll
        for (int o = 1; o < LPR; o <<= 1) {
          w.re += __shfl_xor_sync(gmask, w.re, o);
          w.im += __shfl_xor_sync(gmask, w.im, o);
        }
        const C2<T> tw = C2<T>{tau * w.re, tau * w.im};
#pragma unroll
        for (int u = 0; u < CPL; ++u) {
          const int jj = q + u * LPR;
          zr[P + jj] = csub(zr[P + jj], cmul(tw, xi[jj]));
        }
        if (q == 0) zr[i] = csub(zr[i], cmulc(tw, v0));
      }
      if (row == i + 1 && row < p) make_reflector(i + 1, (i + 1) & 1);
      __syncthreads();
    }
  }

  // ---------------------------------------------------------------- 2. Jacobi
  const int pe = p + (p & 1);
  const T tol = T(p) * Eps<T>::u;
  if (tid == 0) {
    sh_rot[0] = 0;
    sh_rot[1] = 0;
  }
  __syncthreads();
  bool conv = false;
  for (int sweep = 0; sweep < a.max_sweeps; ++sweep) {
    const int sp = sweep & 1;
    for (int rd = 0; rd < pe - 1; ++rd) {
      for (int kk = warp; kk < pe / 2; kk += NW) {
        const int ia = kk == 0 ? 0 : ((kk - 1 + rd) % (pe - 1)) + 1;
        const int ib = ((pe - 2 - kk + rd) % (pe - 1)) + 1;
        T al = T(0), be = T(0);
        C2<T> ga = czero<T>();
        for (int r = lane; r < p; r += 32) {
          const C2<T> xa = X[r * LDX + ia], xb = X[r * LDX + ib];
          al += cnorm2(xa);
          be += cnorm2(xb);
          ga = cadd(ga, cmulc(xb, xa));  // conj(xa) * xb
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga.re = warp_sum(ga.re);
        ga.im = warp_sum(ga.im);
        const T gabs = hypot(ga.re, ga.im);
        const T zt = (be - al) / (T(2) * gabs);
        const T t = (zt >= T(0) ? T(1) : T(-1)) / (fabs(zt) + hypot(T(1), zt));
        const T c = T(1) / sqrt(T(1) + t * t);
        const T s = t * c;
        if (al > Eps<T>::tiny && be > Eps<T>::tiny && gabs > tol * sqrt(al) * sqrt(be) && s != T(0)) {
          const C2<T> e = C2<T>{ga.re / gabs, -ga.im / gabs};  // e^{-i arg gamma}
          for (int r = lane; r < p; r += 32) {
            const C2<T> xa = X[r * LDX + ia];
            const C2<T> eb = cmul(e, X[r * LDX + ib]);
            X[r * LDX + ia] = C2<T>{c * xa.re - s * eb.re, c * xa.im - s * eb.im};
            X[r * LDX + ib] = C2<T>{s * xa.re + c * eb.re, s * xa.im + c * eb.im};
          }
          if (lane == 0) sh_rot[sp] = 1;
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

  // ---------------------------------------------------------------- 3. rank
  for (int j = warp; j < p; j += NW) {
    double s = 0.0;
    for (int r = lane; r < p; r += 32) {
      const C2<T> x = X[r * LDX + j];
      s += (double)x.re * (double)x.re + (double)x.im * (double)x.im;
    }
    s = warp_sum(s);
    if (lane == 0) sig2[j] = s;
  }
  __syncthreads();
  // non-finite values (only from non-finite input) are ranked as zero and
  // reported; ord stays a permutation of 0..p-1 in every case
  if (tid < p) {
    ord[tid] = tid;
    if (!(sig2[tid] >= 0.0 && sig2[tid] <= 1.0e300)) {
      sig2[tid] = 0.0;
      atomicOr(a.status, kStatusNaN);
    }
  }
  __syncthreads();
  int rk = -1;
  if (tid < p) {
    const double v = sig2[tid];
    rk = 0;
    for (int i = 0; i < p; ++i) {
      const double u = sig2[i];
      rk += (u > v) || (u == v && i < tid);
    }
  }
  __syncthreads();
  if (rk >= 0 && rk < p) ord[rk] = tid;
  __syncthreads();
  if (tid == 0) {
    const double e2 = a.eps2[lvl];
    double tail = 0.0;
    int k = p;
    for (int r = p - 1; r >= 0; --r) {
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
  for (int r = tid; r < kSigStride; r += NT) sig_out[r] = r < p ? sqrt(sig2[ord[r]]) : 0.0;
  __syncthreads();
  const int k = sh_k;

  // ---------------------------------------------------------------- 4. Q
  C2<T>* Qout = a.Q[side] + a.Qoff[side][pid];
  const int ldq = a.rowcap[side][pid];
  for (int qq = warp; qq < k; qq += NW) {
    const int j = ord[qq];
    const T inv = (T)(1.0 / sqrt(sig2[j]));
    for (int r = lane; r < p; r += 32) {
      C2<T> v = X[r * LDX + j];
      v = C2<T>{v.re * inv, v.im * inv};
      X[r * LDX + j] = v;
      if (DH2_IN(a.Qoff[side][pid] + r + (int64_t)qq * ldq, c_lim.Q[side], 10, pid)) Qout[r + (int64_t)qq * ldq] = v;
    }
  }
  __syncthreads();

  // ---------------------------------------------------------------- 5. R = Q^* A
  if (k == 0) return;
  C2<T>* Rout = a.R[side] + a.Roff[side][pid];
  for (int j0 = 0; j0 < N; j0 += C) {
    load_chunk(j0);
    __syncthreads();
    const int cw = min(C, N - j0);
    for (int idx = tid; idx < k * cw; idx += NT) {
      const int qq = idx % k, jj = idx / k;
      const int j = ord[qq];
      C2<T> acc = czero<T>();
      for (int r = 0; r < p; ++r) acc = cadd(acc, cmulc(X[r * LDX + P + jj], X[r * LDX + j]));
      if (DH2_IN(a.Roff[side][pid] + qq + (int64_t)(j0 + jj) * kcap, c_lim.R[side], 11, pid))
        Rout[qq + (int64_t)(j0 + jj) * kcap] = acc;
    }
    __syncthreads();
  }
}

template <typename T, int C, int LPR, bool FROM_R>
void launch_one(const PairArgs<T>& a, int nblocks, cudaStream_t st) {
  const int P = a.P;
  const int LDX = P + C + 1;
  size_t smem = (((size_t)P * LDX * sizeof(C2<T>) + 15) & ~(size_t)15) + (size_t)P * sizeof(double) +
                (size_t)P * sizeof(int);
  auto kern = pair_kernel<T, C, LPR, FROM_R>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kern<<<nblocks, 256, smem, st>>>(a);
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

template <typename T>
void launch_pair_kernel(const PairArgs<T>& a, int nblocks, bool from_r, cudaStream_t st) {
  if (nblocks <= 0) return;
  constexpr bool f32 = sizeof(T) == 4;
  if (!from_r) {
    if (a.P <= 64) launch_one<T, f32 ? 64 : 32, 4, false>(a, nblocks, st);
    else launch_one<T, f32 ? 32 : 16, 2, false>(a, nblocks, st);
  } else {
    if (a.P <= 64) launch_one<T, f32 ? 64 : 32, 4, true>(a, nblocks, st);
    else launch_one<T, f32 ? 32 : 16, 2, true>(a, nblocks, st);
  }
}

template void launch_pair_kernel<float>(const PairArgs<float>&, int, bool, cudaStream_t);
template void launch_pair_kernel<double>(const PairArgs<double>&, int, bool, cudaStream_t);

}  // namespace dh2
