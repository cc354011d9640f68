// Kernels around the per-pair factorisation: block norms and nearfield copy,
// basis expansion by Eq. (nested), the projection S_b, the matrix-vector
// product of Section 4 and the blockwise error.
#include "dh2_check.cuh"
#include "dh2_internal.h"
#include "dh2_ops.cuh"

namespace dh2 {

namespace {

DH2_CHECK_DECLS

template <typename T>
__device__ __forceinline__ C2<T> czero() { return C2<T>{T(0), T(0)}; }
template <typename T>
__device__ __forceinline__ C2<T> cadd(C2<T> a, C2<T> b) { return C2<T>{a.re + b.re, a.im + b.im}; }
template <typename T>
__device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
  return C2<T>{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T>
__device__ __forceinline__ C2<T> cmulc(C2<T> a, C2<T> b) {  // a * conj(b)
  return C2<T>{a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im};
}
template <typename T>
__device__ __forceinline__ C2<T> cconj(C2<T> a) { return C2<T>{a.re, -a.im}; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum of one double (256 threads)
__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;  // valid in thread 0
}

// Expanded basis of a pair: a leaf's stored Q (ld = cluster size) or the
// expansion buffer of a non-leaf pair (ld = cluster size).
template <typename T>
__device__ __forceinline__ const C2<T>* xbasis(const SideView<T>& S, int pid) {
  return S.leaf[pid] ? S.Q + S.Qoff[pid] : S.X + S.Xoff[pid];
}

// ---------------------------------------------------------------- norms / nearfield
// acc + |g|^2 with a fixed rounding sequence (no contraction left to the
// compiler), so that every kernel summing a piece gets the same bits
__device__ __forceinline__ float sq_add(float acc, C2<float> g) {
  return __fadd_rn(acc, __fmaf_rn(g.re, g.re, __fmul_rn(g.im, g.im)));
}
__device__ __forceinline__ double sq_add(double acc, C2<double> g) {
  return __dadd_rn(acc, __fma_rn(g.re, g.re, __dmul_rn(g.im, g.im)));
}

// |G_b|_F^2 of an admissible block as the admissible blocks' pass forms it:
// pieces of 32 rows by kNormCols columns in slab-major order, each a warp sum
// (in double) of per-lane sums over the piece's columns in order, added in
// piece order; one warp.
template <typename T>
__device__ double block_norm2_pieces(const NormsArgs<T>& a, int b, int64_t t0, int64_t s0, int mt, int ms, int lane) {
  double tot = 0.0;
  for (int sl = 0; sl * 32 < mt; ++sl) {
    const int r = sl * 32 + lane;
    for (int c0 = 0; c0 < ms; c0 += kNormCols) {
      const int c1 = min(ms, c0 + kNormCols);
      T acc = T(0);
      for (int j0 = c0; j0 < c1; j0 += 8) {
        C2<T> g[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          g[u] = czero<T>();
          if (r < mt && j0 + u < c1) {
            const int64_t gi = (s0 + j0 + u) * a.ld + t0 + r;
            if (DH2_IN(gi, c_lim.G, 20, b)) g[u] = a.G[gi];
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) acc = sq_add(acc, g[u]);
      }
      tot += warp_sum((double)acc);
    }
  }
  return tot;
}
// One warp per block of the block tree: |G_b|_F for an admissible block
// (weight omega_b = |G_b|_F zeta^-level(t), Remark "Error control"); a copy of
// G_b into the nearfield buffer for an inadmissible one.  Each warp walks the
// block column by column (contiguous runs of the row cluster).
template <typename T>
__global__ void __launch_bounds__(256) norms_near_kernel(const NormsArgs<T>* __restrict__ args,
                                                          const uint32_t* __restrict__ codes, int n) {
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const uint32_t code = codes ? codes[w] : (uint32_t)w;
  const NormsArgs<T>& a = args[code >> 26];
  const int b = (int)(code & ((1u << 26) - 1u));
  const int t = a.bt[b], s = a.bs[b];
  const int mt = a.csize[t], ms = a.csize[s];
  const int64_t t0 = a.cstart[t], s0 = a.cstart[s];
  if (a.gen) {
    // matrix-free: generate the block's entries from the points
    if (a.badm[b]) {
      double acc = 0.0;
      for (int64_t e = lane; e < (int64_t)mt * ms; e += 32) {
        const int r = (int)(e % mt), j = (int)(e / mt);
        const C2<T> g = kernel_entry<T>(a.pts, a.nrm, t0 + r, s0 + j, a.kappa, a.diag);
        acc += (double)g.re * g.re + (double)g.im * g.im;
      }
      const double tot = warp_sum(acc);
      if (lane == 0 && DH2_IN(b, c_lim.nblocks, 23, b))
        a.invw[b] = tot > 0.0 ? 1.0 / (sqrt(tot) * a.zpow[a.clevel[t]]) : 1.0;
    if (lane == 0 && a.bnorm2) a.bnorm2[b] = tot;
    } else if (a.copy) {
      C2<T>* out = a.near + a.near_off[b];
      for (int64_t e = lane; e < (int64_t)mt * ms; e += 32) {
        const int r = (int)(e % mt), j = (int)(e / mt);
        if (DH2_IN(a.near_off[b] + e, c_lim.near, 21, b))
          out[e] = kernel_entry<T>(a.pts, a.nrm, t0 + r, s0 + j, a.kappa, a.diag);
      }
    }
    return;
  }
  // dense input: the block is walked as a flat column-major index space,
  // 8 independent loads in flight per lane
  const int total = mt * ms;
  if (a.badm[b] && a.bmax) {
    // mixed modes: besides the norm, the largest |re|, |im| of every row and
    // every column of the block (the row scales of the leaf Gram slices).
    // Lanes take 32 consecutive rows, 8 columns in flight; a column's maximum
    // is a warp reduction, merged over the row slabs by lane 0.
    float* rmx = a.bmax + a.bmax_off[b];
    float* cmx = rmx + mt;
    for (int rs = 0; rs < mt; rs += 32) {
      const int r = rs + lane;
      float rm = 0.f;
      for (int j0 = 0; j0 < ms; j0 += 8) {
        C2<T> g[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          g[u] = czero<T>();
          if (r < mt && j0 + u < ms) {
            const int64_t gi = (s0 + j0 + u) * a.ld + t0 + r;
            if (DH2_IN(gi, c_lim.G, 20, b)) g[u] = a.G[gi];
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          float v = fmaxf(fabsf((float)g[u].re), fabsf((float)g[u].im));
          rm = fmaxf(rm, v);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
          // the first row slab stores the column maximum, later slabs merge
          // into it without waiting for a read (non-negative floats order as
          // their bit patterns)
          if (lane == 0 && j0 + u < ms) {
            if (rs == 0) cmx[j0 + u] = v;
            else atomicMax(reinterpret_cast<int*>(cmx + j0 + u), __float_as_int(v));
          }
        }
      }
      if (r < mt) rmx[r] = rm;
    }
    const double tot = block_norm2_pieces(a, b, t0, s0, mt, ms, lane);
    if (lane == 0 && DH2_IN(b, c_lim.nblocks, 23, b))
      a.invw[b] = tot > 0.0 ? 1.0 / (sqrt(tot) * a.zpow[a.clevel[t]]) : 1.0;
    if (lane == 0 && a.bnorm2) a.bnorm2[b] = tot;
  } else if (a.badm[b]) {
    const double tot = block_norm2_pieces(a, b, t0, s0, mt, ms, lane);
    if (lane == 0 && DH2_IN(b, c_lim.nblocks, 23, b))
      a.invw[b] = tot > 0.0 ? 1.0 / (sqrt(tot) * a.zpow[a.clevel[t]]) : 1.0;
    if (lane == 0 && a.bnorm2) a.bnorm2[b] = tot;
  } else if (a.copy) {
    C2<T>* out = a.near + a.near_off[b];
    for (int e0 = 0; e0 < total; e0 += 256) {
      C2<T> g[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + lane + 32 * u;
        g[u] = czero<T>();
        if (e < total) {
          const int r = e % mt, j = e / mt;
          const int64_t gi = (s0 + j) * a.ld + t0 + r;
          if (DH2_IN(gi, c_lim.G, 22, b)) g[u] = a.G[gi];
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + lane + 32 * u;
        if (e < total && DH2_IN(a.near_off[b] + e, c_lim.near, 21, b)) out[e] = g[u];
      }
    }
  }
}

// ---------------------------------------------------------------- expansion
// X_tc = [X_t1c' E_t1c ; X_t2c' E_t2c] (Eq. nested), one CTA per non-leaf pair.
template <typename T>
__global__ void __launch_bounds__(256) expand_kernel(SideView<T> S, const int32_t* pairs) {
  const int pid = pairs[blockIdx.x];
  const int k = S.rank[pid];
  if (k == 0) return;
  const int ldq = S.rowcap[pid];
  const C2<T>* E = S.Q + S.Qoff[pid];
  C2<T>* out = S.X + S.Xoff[pid];
  const int ldo = S.csize[S.cluster[pid]];
  int rowoff = 0, eoff = 0;
  for (int j = 0; j < 2; ++j) {
    const int sp = S.son[2 * pid + j];
    if (!DH2_IN(sp, c_lim.npairs[S.side], 34, pid)) return;
    const int kj = S.rank[sp];
    const int mj = S.csize[S.cluster[sp]];
    const C2<T>* W = xbasis(S, sp);
    for (int idx = threadIdx.x; idx < mj * k; idx += blockDim.x) {
      const int i = idx % mj, qq = idx / mj;
      C2<T> acc = czero<T>();
      for (int l = 0; l < kj; ++l) {
        const bool okw = S.leaf[sp] ? DH2_IN(S.Qoff[sp] + i + (int64_t)l * mj, c_lim.Q[S.side], 30, pid)
                                    : DH2_IN(S.Xoff[sp] + i + (int64_t)l * mj, c_lim.X[S.side], 31, pid);
        const bool oke = DH2_IN(S.Qoff[pid] + eoff + l + (int64_t)qq * ldq, c_lim.Q[S.side], 32, pid);
        if (okw && oke) acc = cadd(acc, cmul(W[i + (int64_t)l * mj], E[eoff + l + (int64_t)qq * ldq]));
      }
      if (DH2_IN(S.Xoff[pid] + rowoff + i + (int64_t)qq * ldo, c_lim.X[S.side], 33, pid))
        out[rowoff + i + (int64_t)qq * ldo] = acc;
    }
    rowoff += mj;
    eoff += kj;
  }
}

// ---------------------------------------------------------------- projection
// S_b = omega_b R_tc|_b W_sc: R_tc|_b = V_tc^* G_b / omega_b is the block's
// own column range of R_tc (Section 6), W_sc the expanded column basis.
// One warp per admissible block.  For ranks up to KS the warp stages chunks
// of JC columns of R_tc|_b and rows of W_sc in its own shared memory
// (coalesced) and each lane forms a 2 x 4 tile of S_b; larger ranks take the
// generic path, which reads R and W through L1.
template <typename T>
__device__ __forceinline__ C2<T> cmac(C2<T> acc, C2<T> x, C2<T> y) {  // acc + x y
  acc.re = fma(x.re, y.re, acc.re);
  acc.re = fma(-x.im, y.im, acc.re);
  acc.im = fma(x.re, y.im, acc.im);
  acc.im = fma(x.im, y.re, acc.im);
  return acc;
}

namespace {
// global -> shared copy of BYTES (4, 8 or 16; both addresses aligned to it)
// without a register round trip, and the wait for this thread's copies
template <int BYTES>
__device__ __forceinline__ void proj_cp_async(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src),
               "n"(BYTES)
               : "memory");
}
__device__ __forceinline__ void proj_cp_async_wait() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}
}  // namespace

#ifndef DH2_PROJ_MINB
#define DH2_PROJ_MINB 5  // FP32 projection: register cap for this many CTAs per SM (96 registers, no spills)
#endif
template <typename T>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? DH2_PROJ_MINB : 1) project_kernel(ProjArgs<T> a, int nadm) {
  constexpr int KS = 32;
  constexpr int JC = sizeof(T) == 4 ? 16 : 8;
  __shared__ C2<T> sR[4][KS * JC];  // R chunk: kt x jc, column-major, ld KS
  __shared__ C2<T> sW[4][JC * KS];  // W chunk: jc x ks, column-major, ld JC
  const int wl = threadIdx.x >> 5;
  const int wid = blockIdx.x * (blockDim.x >> 5) + wl;
  const int lane = threadIdx.x & 31;
  if (wid >= nadm) return;
  const int b = a.adm_list[wid];
  const int Pt = a.bpair_row[b], Ps = a.bpair_col[b];
  if (!DH2_IN(Pt, c_lim.npairs[0], 44, b) || !DH2_IN(Ps, c_lim.npairs[1], 45, b)) return;
  const int off = a.boff_row[b];
  const int kt = a.V.rank[Pt], ks = a.W.rank[Ps];
  C2<T>* Sout = a.S + a.Soff[b];
  if (kt == 0 || ks == 0) return;
  const int ms = a.csize[a.bs[b]];
  const int ldr = a.V.kcap[Pt];
  const int64_t rbase = a.V.Roff[Pt] + (int64_t)off * ldr;
  const C2<T>* R = a.V.R + rbase;
  const bool wleaf = a.W.leaf[Ps];
  const int64_t wbase = wleaf ? a.W.Qoff[Ps] : a.W.Xoff[Ps];
  const C2<T>* W = xbasis(a.W, Ps);
  const T w = (T)(1.0 / a.invw[b]);
  if (kt <= KS && ks <= KS) {
    C2<T>* r_s = sR[wl];
    C2<T>* w_s = sW[wl];
    const int nqt = (kt + 1) >> 1, nct = (ks + 3) >> 2, ntile = nqt * nct;
    for (int t0 = 0; t0 < ntile; t0 += 32) {
      const int t = t0 + lane;
      const bool act = t < ntile;
      const int q0 = act ? 2 * (t % nqt) : 0, c0 = act ? 4 * (t / nqt) : 0;
      C2<T> acc[2][4];
#pragma unroll
      for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = czero<T>();
      for (int j0 = 0; j0 < ms; j0 += JC) {
        const int jc = min(JC, ms - j0);
        __syncwarp();
        // the chunk's entries by asynchronous copies with fixed trip counts,
        // all in flight together (one load latency per chunk, not one per
        // entry): R rows q < kt (lane q) of columns j0 + jj, jj < jc; W rows
        // j0 + jj (lane % JC) of columns c < ks
#pragma unroll
        for (int jj = 0; jj < JC; ++jj)
          if (lane < kt && jj < jc) {
            const int64_t ri = lane + (int64_t)(j0 + jj) * ldr;
            if (DH2_IN(rbase + ri, c_lim.R[0], 40, b)) proj_cp_async<sizeof(C2<T>)>(r_s + lane + jj * KS, R + ri);
            else r_s[lane + jj * KS] = czero<T>();
          }
        constexpr int WU = KS * JC / 32;  // W entries per lane
#pragma unroll
        for (int u = 0; u < WU; ++u) {
          const int jj = lane % JC, c = u * (32 / JC) + lane / JC;
          if (jj < jc && c < ks) {
            const int64_t wi = (j0 + jj) + (int64_t)c * ms;
            const bool ok = wleaf ? DH2_IN(wbase + wi, c_lim.Q[1], 41, b) : DH2_IN(wbase + wi, c_lim.X[1], 42, b);
            if (ok) proj_cp_async<sizeof(C2<T>)>(w_s + jj + c * JC, W + wi);
            else w_s[jj + c * JC] = czero<T>();
          }
        }
        proj_cp_async_wait();
        __syncwarp();
        if (act)
          for (int jj = 0; jj < jc; ++jj) {
            // rows past kt and columns past ks read unwritten entries whose
            // products are never stored
            const C2<T> x0 = r_s[q0 + jj * KS], x1 = r_s[q0 + 1 + jj * KS];
#pragma unroll
            for (int y = 0; y < 4; ++y) {
              const C2<T> wy = w_s[jj + (c0 + y) * JC];
              acc[0][y] = cmac(acc[0][y], x0, wy);
              acc[1][y] = cmac(acc[1][y], x1, wy);
            }
          }
      }
      if (act)
#pragma unroll
        for (int x = 0; x < 2; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            const int qq = q0 + x, cc = c0 + y;
            const int o = qq + cc * kt;  // column-major, ld = kt
            if (qq < kt && cc < ks && DH2_IN(a.Soff[b] + o, c_lim.S, 43, b))
              Sout[o] = C2<T>{w * acc[x][y].re, w * acc[x][y].im};
          }
    }
    return;
  }
  const int nout = kt * ks;
  for (int o0 = 0; o0 < nout; o0 += 32 * 8) {
    C2<T> acc[8];
    int qq[8], cc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      acc[u] = czero<T>();
      const int o = o0 + lane + 32 * u;
      qq[u] = o % kt;
      cc[u] = o / kt;
    }
    for (int j = 0; j < ms; ++j) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (o0 + lane + 32 * u < nout) {
          const int64_t ri = qq[u] + (int64_t)j * ldr;
          const int64_t wi = j + (int64_t)cc[u] * ms;
          const bool ok = DH2_IN(rbase + ri, c_lim.R[0], 40, b) &&
                          (wleaf ? DH2_IN(wbase + wi, c_lim.Q[1], 41, b) : DH2_IN(wbase + wi, c_lim.X[1], 42, b));
          if (ok) acc[u] = cmac(acc[u], R[ri], W[wi]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int o = o0 + lane + 32 * u;
      if (o < nout && DH2_IN(a.Soff[b] + o, c_lim.S, 43, b))
        Sout[o] = C2<T>{w * acc[u].re, w * acc[u].im};  // column-major, ld = kt
    }
  }
}

// ---------------------------------------------------------------- matvec
// forward transformation, leaves: xh_sc = W_sc^* x|_s (Eq. mvm1)
template <typename T>
__global__ void mv_forward_leaf(SideView<T> W, const int32_t* pairs, const C2<T>* x, int nrhs, int64_t n,
                                C2<T>* xh, const int64_t* hoff) {
  const int pid = pairs[blockIdx.x];
  const int k = W.rank[pid];
  const int m = W.csize[W.cluster[pid]];
  const int64_t s0 = W.cstart[W.cluster[pid]];
  const C2<T>* Q = W.Q + W.Qoff[pid];
  for (int idx = threadIdx.x; idx < k * nrhs; idx += blockDim.x) {
    const int qq = idx % k, rh = idx / k;
    C2<T> acc = czero<T>();
    for (int i = 0; i < m; ++i) acc = cadd(acc, cmulc(x[s0 + i + rh * n], Q[i + (int64_t)qq * m]));
    xh[hoff[pid] * nrhs + qq + (int64_t)rh * k] = acc;
  }
}

// forward transformation, non-leaves: xh_sc = sum_s' E_s'c^* xh_s'c'
template <typename T>
__global__ void mv_forward_up(SideView<T> W, const int32_t* pairs, int nrhs, C2<T>* xh, const int64_t* hoff) {
  const int pid = pairs[blockIdx.x];
  const int k = W.rank[pid];
  const int ldq = W.rowcap[pid];
  const C2<T>* E = W.Q + W.Qoff[pid];
  for (int idx = threadIdx.x; idx < k * nrhs; idx += blockDim.x) {
    const int qq = idx % k, rh = idx / k;
    C2<T> acc = czero<T>();
    int eoff = 0;
    for (int j = 0; j < 2; ++j) {
      const int sp = W.son[2 * pid + j];
      const int kj = W.rank[sp];
      const C2<T>* xs = xh + hoff[sp] * nrhs + (int64_t)rh * kj;
      for (int l = 0; l < kj; ++l) acc = cadd(acc, cmulc(xs[l], E[eoff + l + (int64_t)qq * ldq]));
      eoff += kj;
    }
    xh[hoff[pid] * nrhs + qq + (int64_t)rh * k] = acc;
  }
}

// coupling: yh_tc = sum over own blocks b of S_b xh_{s c} (Eq. mvm2)
template <typename T>
__global__ void mv_coupling(MvArgs<T> a, int nrhs) {
  const int pid = blockIdx.x;
  const int kt = a.V.rank[pid];
  for (int idx = threadIdx.x; idx < kt * nrhs; idx += blockDim.x) {
    const int qq = idx % kt, rh = idx / kt;
    C2<T> acc = czero<T>();
    for (int64_t e = a.own_ptr[pid]; e < a.own_ptr[pid + 1]; ++e) {
      const int b = a.own_blk[e];
      const int Ps = a.bpair_col[b];
      const int ks = a.W.rank[Ps];
      const C2<T>* S = a.S + a.Soff[b];
      const C2<T>* xs = a.xh + a.xhoff[Ps] * nrhs + (int64_t)rh * ks;
      for (int l = 0; l < ks; ++l) acc = cadd(acc, cmul(S[qq + (int64_t)l * kt], xs[l]));
    }
    a.yh[a.yhoff[pid] * nrhs + qq + (int64_t)rh * kt] = acc;
  }
}

// backward transformation: yh_t'c' += E_t'c yh_tc over the father pairs (t, c)
// with sd(c) = c', gathered per son pair (figure "Fast forward and backward
// transformation", right).
template <typename T>
__global__ void mv_backward_down(MvArgs<T> a, const int32_t* pairs, int nrhs) {
  const int pid = pairs[blockIdx.x];
  const int k = a.V.rank[pid];
  for (int idx = threadIdx.x; idx < k * nrhs; idx += blockDim.x) {
    const int qq = idx % k, rh = idx / k;
    C2<T> acc = a.yh[a.yhoff[pid] * nrhs + qq + (int64_t)rh * k];
    for (int64_t e = a.par_ptr[pid]; e < a.par_ptr[pid + 1]; ++e) {
      const int fp = a.par_pair[e];
      const int j = a.par_son[e];
      const int kf = a.V.rank[fp];
      const int ldq = a.V.rowcap[fp];
      const int eoff = j == 0 ? 0 : a.V.rank[a.V.son[2 * fp]];
      const C2<T>* E = a.V.Q + a.V.Qoff[fp];
      const C2<T>* yf = a.yh + a.yhoff[fp] * nrhs + (int64_t)rh * kf;
      for (int l = 0; l < kf; ++l) acc = cadd(acc, cmul(E[eoff + qq + (int64_t)l * ldq], yf[l]));
    }
    a.yh[a.yhoff[pid] * nrhs + qq + (int64_t)rh * k] = acc;
  }
}

template <typename T>
__device__ __forceinline__ void catomic_add(C2<T>* p, C2<T> v) {
  atomicAdd(&p->re, v.re);
  atomicAdd(&p->im, v.im);
}

// leaves: y|_t += V_tc yh_tc (Eq. mvm3)
template <typename T>
__global__ void mv_backward_leaf(MvArgs<T> a, const int32_t* pairs, int nrhs, C2<T>* y, int64_t n) {
  const int pid = pairs[blockIdx.x];
  const int k = a.V.rank[pid];
  if (k == 0) return;
  const int m = a.V.csize[a.V.cluster[pid]];
  const int64_t t0 = a.V.cstart[a.V.cluster[pid]];
  const C2<T>* Q = a.V.Q + a.V.Qoff[pid];
  for (int idx = threadIdx.x; idx < m * nrhs; idx += blockDim.x) {
    const int i = idx % m, rh = idx / m;
    const C2<T>* yh = a.yh + a.yhoff[pid] * nrhs + (int64_t)rh * k;
    C2<T> acc = czero<T>();
    for (int l = 0; l < k; ++l) acc = cadd(acc, cmul(Q[i + (int64_t)l * m], yh[l]));
    catomic_add(y + t0 + i + rh * n, acc);
  }
}

// nearfield: y|_t += G_b x|_s for inadmissible leaves
template <typename T>
__global__ void mv_near(MvArgs<T> a, const int32_t* blocks, int nrhs, const C2<T>* x, C2<T>* y, int64_t n) {
  const int b = blocks[blockIdx.x];
  const int t = a.bt[b], s = a.bs[b];
  const int mt = a.V.csize[t], ms = a.V.csize[s];
  const int64_t t0 = a.V.cstart[t], s0 = a.V.cstart[s];
  const C2<T>* Gb;
  int64_t ldb;
  if (a.near) {
    Gb = a.near + a.near_off[b];
    ldb = mt;
  } else {
    Gb = a.G + s0 * a.ld + t0;
    ldb = a.ld;
  }
  for (int idx = threadIdx.x; idx < mt * nrhs; idx += blockDim.x) {
    const int i = idx % mt, rh = idx / mt;
    C2<T> acc = czero<T>();
    for (int j = 0; j < ms; ++j) acc = cadd(acc, cmul(Gb[i + (int64_t)j * ldb], x[s0 + j + rh * n]));
    catomic_add(y + t0 + i + rh * n, acc);
  }
}

// ---------------------------------------------------------------- error
// sum over blocks of |G_ref - G~|_F^2 and |G_ref|_F^2 in FP64.
template <typename T, typename RT>
__device__ __forceinline__ C2<double> ref_entry(const ErrArgs<T>& a, const C2<RT>* Gref, int64_t ldr, int64_t i,
                                                int64_t j) {
  if (a.ref_gen) return kernel_entry<double>(a.pts, a.nrm, i, j, a.kappa, a.diag);
  const C2<RT> g = Gref[i + j * ldr];
  return C2<double>{(double)g.re, (double)g.im};
}

template <typename T, typename RT>
__global__ void __launch_bounds__(256) error_kernel(ErrArgs<T> a, const C2<RT>* Gref, int64_t ldr,
                                                    double* acc_out) {
  __shared__ double red[32];
  __shared__ C2<double> Ts[128][17];
  const int b = blockIdx.x;
  const int t = a.bt[b], s = a.bs[b];
  const int mt = a.csize[t], ms = a.csize[s];
  const int64_t t0 = a.cstart[t], s0 = a.cstart[s];
  double e2 = 0.0, r2 = 0.0;
  if (!a.badm[b]) {
    for (int idx = threadIdx.x; idx < mt * ms; idx += blockDim.x) {
      const int i = idx % mt, j = idx / mt;
      const C2<double> g = ref_entry<T, RT>(a, Gref, ldr, t0 + i, s0 + j);
      const C2<T> h = a.near ? a.near[a.near_off[b] + i + (int64_t)j * mt] : a.G[(t0 + i) + (s0 + j) * a.ld];
      const double dr = (double)g.re - (double)h.re, di = (double)g.im - (double)h.im;
      e2 += dr * dr + di * di;
      r2 += (double)g.re * g.re + (double)g.im * g.im;
    }
  } else {
    const int Pt = a.bpair_row[b], Ps = a.bpair_col[b];
    const int kt = a.V.rank[Pt], ks = a.W.rank[Ps];
    const C2<T>* Vt = xbasis(a.V, Pt);
    const C2<T>* Wsb = xbasis(a.W, Ps);
    const C2<T>* S = a.S + a.Soff[b];
    for (int j0 = 0; j0 < ms; j0 += 16) {
      const int cw = min(16, ms - j0);
      __syncthreads();
      // T = S W^* for columns j0..j0+cw (kt <= 128)
      for (int idx = threadIdx.x; idx < kt * cw; idx += blockDim.x) {
        const int qq = idx % kt, jj = idx / kt;
        double ar = 0.0, ai = 0.0;
        for (int l = 0; l < ks; ++l) {
          const C2<T> sv = S[qq + (int64_t)l * kt];
          const C2<T> wv = Wsb[j0 + jj + (int64_t)l * ms];
          // s * conj(w)
          ar += (double)sv.re * wv.re + (double)sv.im * wv.im;
          ai += (double)sv.im * wv.re - (double)sv.re * wv.im;
        }
        Ts[qq][jj] = C2<double>{ar, ai};
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < mt * cw; idx += blockDim.x) {
        const int i = idx % mt, jj = idx / mt;
        double ar = 0.0, ai = 0.0;
        for (int qq = 0; qq < kt; ++qq) {
          const C2<T> v = Vt[i + (int64_t)qq * mt];
          const C2<double> tv = Ts[qq][jj];
          ar += (double)v.re * tv.re - (double)v.im * tv.im;
          ai += (double)v.re * tv.im + (double)v.im * tv.re;
        }
        const C2<double> g = ref_entry<T, RT>(a, Gref, ldr, t0 + i, s0 + j0 + jj);
        const double dr = (double)g.re - ar, di = (double)g.im - ai;
        e2 += dr * dr + di * di;
        r2 += (double)g.re * g.re + (double)g.im * g.im;
      }
    }
  }
  const double se = block_sum(e2, red);
  const double sr = block_sum(r2, red);
  if (threadIdx.x == 0) {
    atomicAdd(acc_out, se);
    atomicAdd(acc_out + 1, sr);
  }
}

// ---------------------------------------------------------------- adjoint product
// y = G~^* x: the forward transformation runs on the row basis V, the
// coupling applies S_b^* from row pairs to column pairs, the backward
// transformation runs on the column basis W (the roles of V and W in
// Section 4 exchanged), plus G_b^* on the nearfield.  The kernels of the
// product are reused with an MvArgs whose V and W, coefficient vectors and
// pair lists are those of the exchanged sides; coupling and nearfield need
// their own (conjugate-transposed) loops.
//
// coupling: yh_sc = sum over the column pair's blocks b of S_b^* xh_tc
template <typename T>
__global__ void mv_coupling_adj(MvArgs<T> a, int nrhs) {
  const int pid = blockIdx.x;
  const int kout = a.V.rank[pid];  // rank of this column pair
  for (int idx = threadIdx.x; idx < kout * nrhs; idx += blockDim.x) {
    const int qq = idx % kout, rh = idx / kout;
    C2<T> acc = czero<T>();
    for (int64_t e = a.own_ptr[pid]; e < a.own_ptr[pid + 1]; ++e) {
      const int b = a.own_blk[e];
      const int Pt = a.bpair_col[b];   // the block's row pair
      const int kin = a.W.rank[Pt];
      const C2<T>* S = a.S + a.Soff[b];  // kin x kout, column-major
      const C2<T>* xs = a.xh + a.xhoff[Pt] * nrhs + (int64_t)rh * kin;
      for (int l = 0; l < kin; ++l) acc = cadd(acc, cmul(cconj(S[l + (int64_t)qq * kin]), xs[l]));
    }
    a.yh[a.yhoff[pid] * nrhs + qq + (int64_t)rh * kout] = acc;
  }
}

// nearfield: y|_s += G_b^* x|_t for inadmissible leaves
template <typename T>
__global__ void mv_near_adj(MvArgs<T> a, const int32_t* blocks, int nrhs, const C2<T>* x, C2<T>* y, int64_t n) {
  const int b = blocks[blockIdx.x];
  const int t = a.bt[b], s = a.bs[b];
  const int mt = a.V.csize[t], ms = a.V.csize[s];
  const int64_t t0 = a.V.cstart[t], s0 = a.V.cstart[s];
  const C2<T>* Gb;
  int64_t ldb;
  if (a.near) {
    Gb = a.near + a.near_off[b];
    ldb = mt;
  } else {
    Gb = a.G + s0 * a.ld + t0;
    ldb = a.ld;
  }
  // one warp per column of the block: lanes over its rows
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int cj = wp; cj < ms * nrhs; cj += nw) {
    const int j = cj % ms, rh = cj / ms;
    C2<T> acc = czero<T>();
    for (int i = lane; i < mt; i += 32) acc = cadd(acc, cmul(cconj(Gb[i + (int64_t)j * ldb]), x[t0 + i + rh * n]));
    acc.re = warp_sum(acc.re);
    acc.im = warp_sum(acc.im);
    if (lane == 0) catomic_add(y + s0 + j + rh * n, acc);
  }
}

// ---------------------------------------------------------------- dense products with the reference
// y = G_ref x (trans = false) or y = G_ref^* x (trans = true), complex128
// vectors, FP64 accumulation; G_ref stored (column-major, ld) or generated
// from the points (matrix-free compression: gen != 0).
template <typename RT>
__device__ __forceinline__ C2<double> gref(const C2<RT>* G, int64_t ld, const ErrArgs<float>& g, int64_t i,
                                           int64_t j) {
  if (!G) return kernel_entry<double>(g.pts, g.nrm, i, j, g.kappa, g.diag);
  const C2<RT> v = G[i + j * ld];
  return C2<double>{(double)v.re, (double)v.im};
}

template <typename RT>
__global__ void __launch_bounds__(256) gemv_n_kernel(const C2<RT>* G, int64_t ld, ErrArgs<float> g, int64_t n,
                                                     const C2<double>* x, C2<double>* y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double ar = 0.0, ai = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    const C2<double> v = gref<RT>(G, ld, g, i, j);
    const C2<double> u = x[j];
    ar = fma(v.re, u.re, fma(-v.im, u.im, ar));
    ai = fma(v.re, u.im, fma(v.im, u.re, ai));
  }
  y[i] = C2<double>{ar, ai};
}

template <typename RT>
__global__ void __launch_bounds__(256) gemv_c_kernel(const C2<RT>* G, int64_t ld, ErrArgs<float> g, int64_t n,
                                                     const C2<double>* x, C2<double>* y) {
  const int64_t j = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= n) return;
  double ar = 0.0, ai = 0.0;
  for (int64_t i = lane; i < n; i += 32) {
    const C2<double> v = gref<RT>(G, ld, g, i, j);
    const C2<double> u = x[i];
    // conj(v) u
    ar = fma(v.re, u.re, fma(v.im, u.im, ar));
    ai = fma(v.re, u.im, fma(-v.im, u.re, ai));
  }
  ar = warp_sum(ar);
  ai = warp_sum(ai);
  if (lane == 0) y[j] = C2<double>{ar, ai};
}

// ---------------------------------------------------------------- closed-form error
// sum over admissible blocks of |G_b|_F^2 - |S_b|_F^2 (the squared error of
// the orthogonal projection, Section 6) and over all blocks of |G_b|_F^2
// (inadmissible blocks from the nearfield copy or the viewed G).
template <typename T>
__global__ void __launch_bounds__(256) closed_form_kernel(ErrArgs<T> a, const double* bnorm2, int nblocks,
                                                           double* acc_out) {
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= nblocks) return;
  double e = 0.0, r = 0.0;
  if (a.badm[b]) {
    const int kt = a.V.rank[a.bpair_row[b]], ks = a.W.rank[a.bpair_col[b]];
    const C2<T>* S = a.S + a.Soff[b];
    double s2 = 0.0;
    for (int i = lane; i < kt * ks; i += 32) s2 += (double)S[i].re * S[i].re + (double)S[i].im * S[i].im;
    s2 = warp_sum(s2);
    e = bnorm2[b] - s2;
    r = bnorm2[b];
  } else {
    const int t = a.bt[b], s = a.bs[b];
    const int mt = a.csize[t], ms = a.csize[s];
    double g2 = 0.0;
    for (int idx = lane; idx < mt * ms; idx += 32) {
      const int i = idx % mt, j = idx / mt;
      const C2<T> v = a.near ? a.near[a.near_off[b] + idx] : a.G[(a.cstart[t] + i) + (a.cstart[s] + j) * a.ld];
      g2 += (double)v.re * v.re + (double)v.im * v.im;
    }
    r = warp_sum(g2);
  }
  if (lane == 0) {
    atomicAdd(acc_out, e);
    atomicAdd(acc_out + 1, r);
  }
}

// ---------------------------------------------------------------- vector helpers of the power iteration
template <typename T>
__global__ void to_type_kernel(const C2<double>* __restrict__ v, C2<T>* __restrict__ o, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = C2<T>{(T)v[i].re, (T)v[i].im};
}
template <typename T>
__global__ void sub_kernel(C2<double>* __restrict__ u, const C2<T>* __restrict__ t, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    u[i] = C2<double>{u[i].re - (double)t[i].re, u[i].im - (double)t[i].im};
}

// Admissible blocks of a stored G in pieces of one 32-row slab by kNormCols
// columns, one warp per piece (piece = code << 32 | slab << 16 | column
// group), so that no block's size sets the kernel's tail: the piece's sum of
// squares goes to partial[piece]; in the mixed modes its rows' and columns'
// largest |re|, |im| are merged into the block's maxima (zeroed before) by
// atomic maxima (non-negative floats order as their bit patterns).
// norms_finish_kernel adds a block's pieces in their order (the result does
// not depend on the order in which pieces run) and forms the weights.
template <typename T>
__global__ void __launch_bounds__(256) norms_adm_kernel(const NormsArgs<T>* __restrict__ args,
                                                        const uint64_t* __restrict__ pieces, int64_t n,
                                                        double* __restrict__ partial) {
  const int64_t w = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const uint64_t pc = pieces[w];
  const uint32_t code = (uint32_t)(pc >> 32);
  const int slab = (int)((pc >> 16) & 0xFFFFu), grp = (int)(pc & 0xFFFFu);
  const NormsArgs<T>& a = args[code >> 26];
  const int b = (int)(code & ((1u << 26) - 1u));
  const int t = a.bt[b], s = a.bs[b];
  const int mt = a.csize[t], ms = a.csize[s];
  const int64_t t0 = a.cstart[t], s0 = a.cstart[s];
  const int r = slab * 32 + lane;
  const int c0 = grp * kNormCols, c1 = min(ms, c0 + kNormCols);
  float* rmx = a.bmax ? a.bmax + a.bmax_off[b] : nullptr;
  float* cmx = rmx ? rmx + mt : nullptr;
  T acc = T(0);
  float rm = 0.f;
  // 8 columns at a time, the next 8 in flight while these are summed
  auto load8 = [&](int j0, C2<T> (&d)[8]) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      d[u] = czero<T>();
      if (r < mt && j0 + u < c1) {
        const int64_t gi = (s0 + j0 + u) * a.ld + t0 + r;
        if (DH2_IN(gi, c_lim.G, 24, b)) d[u] = a.G[gi];
      }
    }
  };
  C2<T> g[8], gn[8];
  load8(c0, g);
  for (int j0 = c0; j0 < c1; j0 += 8) {
    if (j0 + 8 < c1) load8(j0 + 8, gn);
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      acc = sq_add(acc, g[u]);
      v[u] = fmaxf(fabsf((float)g[u].re), fabsf((float)g[u].im));
      rm = fmaxf(rm, v[u]);
    }
    if (cmx) {
      // the 8 columns' maxima over the warp's 32 rows in 9 shuffles: each
      // exchange halves the columns a lane holds (xor 16, 8, 4), then xor 2, 1;
      // lane l ends with column ((l >> 4) & 1) * 4 + ((l >> 3) & 1) * 2 + ((l >> 2) & 1)
      const bool b4 = (lane >> 4) & 1, b3 = (lane >> 3) & 1, b2 = (lane >> 2) & 1;
      float w4[4], w2[2];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float keep = b4 ? v[4 + i] : v[i], give = b4 ? v[i] : v[4 + i];
        w4[i] = fmaxf(keep, __shfl_xor_sync(0xffffffffu, give, 16));
      }
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const float keep = b3 ? w4[2 + i] : w4[i], give = b3 ? w4[i] : w4[2 + i];
        w2[i] = fmaxf(keep, __shfl_xor_sync(0xffffffffu, give, 8));
      }
      float w1 = fmaxf(b2 ? w2[1] : w2[0], __shfl_xor_sync(0xffffffffu, b2 ? w2[0] : w2[1], 4));
      w1 = fmaxf(w1, __shfl_xor_sync(0xffffffffu, w1, 2));
      w1 = fmaxf(w1, __shfl_xor_sync(0xffffffffu, w1, 1));
      const int u = (int)b4 * 4 + (int)b3 * 2 + (int)b2;
      if ((lane & 3) == 0 && j0 + u < c1) atomicMax(reinterpret_cast<int*>(cmx + j0 + u), __float_as_int(w1));
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) g[u] = gn[u];
  }
  if (rmx && r < mt) atomicMax(reinterpret_cast<int*>(rmx + r), __float_as_int(rm));
  const double tot = warp_sum((double)acc);
  if (lane == 0) partial[w] = tot;
}

// the admissible blocks' |G_b|_F^2 (their pieces pbegin[i] .. pbegin[i+1] - 1
// added in order) and weights 1/omega_b
template <typename T>
__global__ void norms_finish_kernel(const NormsArgs<T>* __restrict__ args, const uint32_t* __restrict__ codes,
                                    const int64_t* __restrict__ pbegin, const double* __restrict__ partial,
                                    int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t code = codes[i];
  const NormsArgs<T>& a = args[code >> 26];
  const int b = (int)(code & ((1u << 26) - 1u));
  double tot = 0.0;
  for (int64_t q = pbegin[i]; q < pbegin[i + 1]; ++q) tot += partial[q];
  if (a.bnorm2 && DH2_IN(b, c_lim.nblocks, 25, b)) a.bnorm2[b] = tot;
  a.invw[b] = tot > 0.0 ? 1.0 / (sqrt(tot) * a.zpow[a.clevel[a.bt[b]]]) : 1.0;
}

// |v|^2 summed into *acc (zeroed by the caller)
__global__ void norm2_kernel(const C2<double>* __restrict__ v, int64_t n, double* __restrict__ acc) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += v[i].re * v[i].re + v[i].im * v[i].im;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(acc, s);
}

// v = w / sqrt(*n2) (v may be w); nothing when *n2 is not positive
__global__ void normalize_kernel(C2<double>* __restrict__ v, const C2<double>* w, int64_t n,
                                 const double* __restrict__ n2) {
  const double t = *n2;
  if (!(t > 0.0)) return;
  const double sc = rsqrt(t);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = C2<double>{w[i].re * sc, w[i].im * sc};
}

// a seeded start vector: entry i from two splitmix64 draws of (seed, i), each in [-1/2, 1/2)
__global__ void seed_vector_kernel(C2<double>* __restrict__ v, int64_t n, uint64_t seed) {
  auto mix = [](uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t a = mix(seed ^ (2 * (uint64_t)i)), b = mix(seed ^ (2 * (uint64_t)i + 1));
    v[i] = C2<double>{(double)(a >> 11) * (1.0 / 9007199254740992.0) - 0.5,
                      (double)(b >> 11) * (1.0 / 9007199254740992.0) - 0.5};
  }
}

}  // namespace

void check_set_limits_ops(const CheckLimits& l) {
#ifdef DH2_CHECK
  cudaMemcpyToSymbol(c_lim, &l, sizeof(l));
  CheckRecord z{};
  cudaMemcpyToSymbol(g_chk, &z, sizeof(z));
#else
  (void)l;
#endif
}

bool check_read_ops(CheckRecord* out) {
#ifdef DH2_CHECK
  cudaMemcpyFromSymbol(out, g_chk, sizeof(*out));
  return out->count != 0;
#else
  (void)out;
  return false;
#endif
}

template <typename T>
void launch_norms_near(const NormsArgs<T>* args, const uint32_t* codes, int n, cudaStream_t st) {
  if (n > 0) norms_near_kernel<T><<<(n + 7) / 8, 256, 0, st>>>(args, codes, n);
}
template <typename T>
void launch_expand(const SideView<T>& S, const int32_t* pairs, int n, cudaStream_t st) {
  if (n > 0) expand_kernel<T><<<n, 256, 0, st>>>(S, pairs);
}
template <typename T>
void launch_project(const ProjArgs<T>& a, int nadm, cudaStream_t st) {
  if (nadm > 0) project_kernel<T><<<(nadm + 3) / 4, 128, 0, st>>>(a, nadm);
}
template <typename T>
void launch_mv_forward_leaf(const SideView<T>& W, const int32_t* pairs, int np, const C2<T>* x, int nrhs,
                            int64_t n, C2<T>* xh, const int64_t* hoff, cudaStream_t st) {
  if (np > 0) mv_forward_leaf<T><<<np, 128, 0, st>>>(W, pairs, x, nrhs, n, xh, hoff);
}
template <typename T>
void launch_mv_forward_up(const SideView<T>& W, const int32_t* pairs, int np, int nrhs, C2<T>* xh,
                          const int64_t* hoff, cudaStream_t st) {
  if (np > 0) mv_forward_up<T><<<np, 128, 0, st>>>(W, pairs, nrhs, xh, hoff);
}
template <typename T>
void launch_mv_coupling(const MvArgs<T>& a, int npairs_row, int nrhs, cudaStream_t st) {
  if (npairs_row > 0) mv_coupling<T><<<npairs_row, 128, 0, st>>>(a, nrhs);
}
template <typename T>
void launch_mv_backward_down(const MvArgs<T>& a, const int32_t* pairs, int np, int nrhs, cudaStream_t st) {
  if (np > 0) mv_backward_down<T><<<np, 128, 0, st>>>(a, pairs, nrhs);
}
template <typename T>
void launch_mv_backward_leaf(const MvArgs<T>& a, const int32_t* pairs, int np, int nrhs, C2<T>* y, int64_t n,
                             cudaStream_t st) {
  if (np > 0) mv_backward_leaf<T><<<np, 128, 0, st>>>(a, pairs, nrhs, y, n);
}
template <typename T>
void launch_mv_near(const MvArgs<T>& a, const int32_t* blocks, int nb, int nrhs, const C2<T>* x, C2<T>* y,
                    int64_t n, cudaStream_t st) {
  if (nb > 0) mv_near<T><<<nb, 128, 0, st>>>(a, blocks, nrhs, x, y, n);
}
template <typename T, typename RT>
void launch_error(const ErrArgs<T>& a, const C2<RT>* Gref, int64_t ldr, int nblocks, double* acc,
                  cudaStream_t st) {
  if (nblocks > 0) error_kernel<T, RT><<<nblocks, 256, 0, st>>>(a, Gref, ldr, acc);
}

template <typename T>
void launch_mv_coupling_adj(const MvArgs<T>& a, int npairs_col, int nrhs, cudaStream_t st) {
  if (npairs_col > 0) mv_coupling_adj<T><<<npairs_col, 128, 0, st>>>(a, nrhs);
}
template <typename T>
void launch_mv_near_adj(const MvArgs<T>& a, const int32_t* blocks, int nb, int nrhs, const C2<T>* x, C2<T>* y,
                        int64_t n, cudaStream_t st) {
  if (nb > 0) mv_near_adj<T><<<nb, 128, 0, st>>>(a, blocks, nrhs, x, y, n);
}
template <typename RT>
void launch_gemv(const C2<RT>* G, int64_t ld, const ErrArgs<float>& gen, int64_t n, bool trans, const C2<double>* x,
                 C2<double>* y, cudaStream_t st) {
  if (n <= 0) return;
  if (!trans) gemv_n_kernel<RT><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(G, ld, gen, n, x, y);
  else gemv_c_kernel<RT><<<(unsigned)((n + 7) / 8), 256, 0, st>>>(G, ld, gen, n, x, y);
}
template <typename T>
void launch_closed_form(const ErrArgs<T>& a, const double* bnorm2, int nblocks, double* acc, cudaStream_t st) {
  if (nblocks > 0) closed_form_kernel<T><<<(nblocks + 7) / 8, 256, 0, st>>>(a, bnorm2, nblocks, acc);
}
template <typename T>
void launch_to_type(const C2<double>* v, C2<T>* o, int64_t n, cudaStream_t st) {
  if (n > 0) to_type_kernel<T><<<(int)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, st>>>(v, o, n);
}
template <typename T>
void launch_norms_adm(const NormsArgs<T>* args_dev, const uint64_t* pieces, int64_t npieces, const uint32_t* codes,
                      const int64_t* pbegin, int64_t nblocks, double* partial, cudaStream_t st) {
  if (npieces > 0) norms_adm_kernel<T><<<(int)((npieces + 7) / 8), 256, 0, st>>>(args_dev, pieces, npieces, partial);
  if (nblocks > 0)
    norms_finish_kernel<T><<<(int)((nblocks + 255) / 256), 256, 0, st>>>(args_dev, codes, pbegin, partial, nblocks);
}

void launch_norm2(const C2<double>* v, int64_t n, double* acc, cudaStream_t st) {
  if (n > 0) norm2_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 4), 256, 0, st>>>(v, n, acc);
}
void launch_normalize(C2<double>* v, const C2<double>* w, int64_t n, const double* n2, cudaStream_t st) {
  if (n > 0) normalize_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, st>>>(v, w, n, n2);
}
void launch_seed_vector(C2<double>* v, int64_t n, uint64_t seed, cudaStream_t st) {
  if (n > 0) seed_vector_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, st>>>(v, n, seed);
}

template <typename T>
void launch_sub(C2<double>* u, const C2<T>* t, int64_t n, cudaStream_t st) {
  if (n > 0) sub_kernel<T><<<(int)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, st>>>(u, t, n);
}
template void launch_gemv<float>(const C2<float>*, int64_t, const ErrArgs<float>&, int64_t, bool, const C2<double>*,
                                 C2<double>*, cudaStream_t);
template void launch_gemv<double>(const C2<double>*, int64_t, const ErrArgs<float>&, int64_t, bool,
                                  const C2<double>*, C2<double>*, cudaStream_t);

// Column maps from their segments: one warp per segment writes the global
// column index and the block id of each of the segment's w columns.
__global__ void colmap_expand_kernel(const int64_t* __restrict__ dst, const int32_t* __restrict__ col0,
                                     const int32_t* __restrict__ w, const int32_t* __restrict__ blk, int64_t nseg,
                                     int32_t* __restrict__ gcol, int32_t* __restrict__ gblk) {
  const int64_t sg = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (sg >= nseg) return;
  const int64_t d = dst[sg];
  const int32_t c0 = col0[sg], b = blk[sg];
  for (int j = lane; j < w[sg]; j += 32) {
    gcol[d + j] = c0 + j;
    gblk[d + j] = b;
  }
}
void launch_colmap_expand(const int64_t* dst, const int32_t* col0, const int32_t* w, const int32_t* blk, int64_t nseg,
                          int32_t* gcol, int32_t* gblk, cudaStream_t st) {
  if (nseg > 0) colmap_expand_kernel<<<(unsigned)((nseg + 7) / 8), 256, 0, st>>>(dst, col0, w, blk, nseg, gcol, gblk);
}

// Per-column weights of a column map: colw[j] = 1/omega_b for the block b of
// column j (Remark "Error control"), so that the pair kernels read the weight
// of a column without the block-id indirection.
template <typename T>
__global__ void colw_kernel(const int32_t* __restrict__ gblk, const double* __restrict__ invw, T* __restrict__ colw,
                            int64_t n) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    colw[j] = (T)invw[gblk[j]];
}
template <typename T>
void launch_colw(const int32_t* gblk, const double* invw, T* colw, int64_t n, cudaStream_t st) {
  if (n > 0) colw_kernel<T><<<(int)std::min<int64_t>((n + 255) / 256, 152 * 8), 256, 0, st>>>(gblk, invw, colw, n);
}

#define DH2_INST(T)                                                                                         \
  template void launch_colw<T>(const int32_t*, const double*, T*, int64_t, cudaStream_t);                  \
  template void launch_norms_near<T>(const NormsArgs<T>*, const uint32_t*, int, cudaStream_t);            \
  template void launch_expand<T>(const SideView<T>&, const int32_t*, int, cudaStream_t);                   \
  template void launch_project<T>(const ProjArgs<T>&, int, cudaStream_t);                                  \
  template void launch_mv_forward_leaf<T>(const SideView<T>&, const int32_t*, int, const C2<T>*, int,      \
                                          int64_t, C2<T>*, const int64_t*, cudaStream_t);                  \
  template void launch_mv_forward_up<T>(const SideView<T>&, const int32_t*, int, int, C2<T>*,              \
                                        const int64_t*, cudaStream_t);                                     \
  template void launch_mv_coupling<T>(const MvArgs<T>&, int, int, cudaStream_t);                           \
  template void launch_mv_backward_down<T>(const MvArgs<T>&, const int32_t*, int, int, cudaStream_t);      \
  template void launch_mv_backward_leaf<T>(const MvArgs<T>&, const int32_t*, int, int, C2<T>*, int64_t,    \
                                           cudaStream_t);                                                  \
  template void launch_mv_near<T>(const MvArgs<T>&, const int32_t*, int, int, const C2<T>*, C2<T>*,        \
                                  int64_t, cudaStream_t);                                                  \
  template void launch_error<T, float>(const ErrArgs<T>&, const C2<float>*, int64_t, int, double*,        \
                                       cudaStream_t);                                                      \
  template void launch_error<T, double>(const ErrArgs<T>&, const C2<double>*, int64_t, int, double*,      \
                                        cudaStream_t);                                                      \
  template void launch_mv_coupling_adj<T>(const MvArgs<T>&, int, int, cudaStream_t);                       \
  template void launch_mv_near_adj<T>(const MvArgs<T>&, const int32_t*, int, int, const C2<T>*, C2<T>*,    \
                                      int64_t, cudaStream_t);                                              \
  template void launch_closed_form<T>(const ErrArgs<T>&, const double*, int, double*, cudaStream_t);            \
  template void launch_to_type<T>(const C2<double>*, C2<T>*, int64_t, cudaStream_t);                       \
  template void launch_norms_adm<T>(const NormsArgs<T>*, const uint64_t*, int64_t, const uint32_t*, const int64_t*, \
                                    int64_t, double*, cudaStream_t);                                           \
  template void launch_sub<T>(C2<double>*, const C2<T>*, int64_t, cudaStream_t);

DH2_INST(float)
DH2_INST(double)

}  // namespace dh2
