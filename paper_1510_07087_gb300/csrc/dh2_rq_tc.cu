// R_tc = Q_tc^* A for the leaf pairs of the mixed mode on the tensor cores
// (tcgen05, sm_103a): the R recursion of Section 6 at the leaves, R_tc =
// V_tc^* G^omega_tc, with V_tc = Q from the leaf factor.  For the row basis
// A = G|_{t x F_tc} and R = w conj(Q)^T A (w the column's block weight
// 1/omega_b); for the column basis A = conj(G^T) on the pair's rows and
// columns, so that both sides read R = w conj(Q)^T A.
//
// The product is an ordinary contraction that only has to be as accurate as
// FP32: both operands are split into three bf16 slices in floating point
// (x = h + m + l, each the bf16 nearest to what is left, 24 significant bits
// in all), and the six slice products of weight >= 2^-16 (hh, hm, mh, hl,
// mm, lh) accumulate in one FP32 accumulator in tensor memory; the dropped
// products are below 2^-24 of the result.
//
// Complex as real: a tile is 128 columns j of A (the MMA's M = 128 rows, one
// TMEM lane per column) and K = 2 mp (mp = m rounded up to 8): row j of the
// A operand is [Re A(:, j); Im A(:, j)].  The B operand has N = 2k rows (k =
// the pair's rank, N rounded up to 16): row q is [Re Q(:, q); Im Q(:, q)] and
// row k + q is [-Im Q(:, q); Re Q(:, q)], so that column q of the accumulator
// holds Re R(q, j) and column k + q holds Im R(q, j).
//
// One CTA per SM over a contiguous range of the launch's tile list (tiles of
// 32 columns; a 128-column tile starts at every list entry whose first column
// is a multiple of 128), in three roles that walk the same schedule:
//   warps 0-7   producers: slice the tile's entries of A (loaded into
//               registers while the tensor cores work on the tile before)
//               into the A stage and, when the pair changes, Q into the B
//               operand; arrive on full;
//   warp 8      one thread issues the tile's MMAs into one of two
//               accumulator sets, commits to empty (the stage may be
//               rewritten) and to accfull[set];
//   warps 9-12  epilogue: read the accumulator (lane = column), scale by the
//               column's weight and write R, arrive on accempty[set].
// Every wait is bounded; a wait that runs out sets the CTA's abort flag, and
// every role leaves the schedule at its next wait.
#include <algorithm>
#include <cstdint>
#include <cstdio>

#include "dh2_internal.h"
#include "dh2_kernels.cuh"
#include "dh2_sm100.cuh"

#include <cuda_bf16.h>

namespace dh2 {

namespace {

using namespace sm100;

constexpr int kTcCols = 128;                   // columns of A per tile (the MMA's M)
constexpr int kTcProd = 256;                   // producer threads (warps 0-7)
constexpr int kTcMmaWarp = 8;
constexpr int kTcEpi0 = 9;                     // first epilogue warp
constexpr int kTcThreads = 13 * 32;
constexpr uint32_t kTcAtom = kTcCols * 128u;   // one K atom (64 bf16 of K) of 128 operand rows
constexpr uint32_t kTcASlice = 2 * kTcAtom;    // K = 2 mp <= 128: two atoms per slice
constexpr uint32_t kTcAStage = 3 * kTcASlice;  // three slices
constexpr int kTcNMax = 128;                   // B rows: N = 2k <= 128 (ranks up to 64)
constexpr uint32_t kTcBSlice = 2 * kTcNMax * 128u;
constexpr uint32_t kTcSmem = 1024 + kTcAStage + 3 * kTcBSlice;
constexpr uint32_t kTcSetCols = kTcNMax;       // columns of one accumulator set
constexpr uint32_t kTcBarProd = 1, kTcBarEpi = 2;
constexpr uint32_t kTcWaitPolls = 1u << 23;    // default bound of a wait: about a second of polls
static_assert(kTcSmem <= 227 * 1024, "one CTA per SM");

// byte offset of 16-byte chunk g of operand row R in a 128-byte-swizzled atom
__device__ __forceinline__ uint32_t tc_swz(int R, int g) {
  return (uint32_t)R * 128u + ((uint32_t)(g ^ (R & 7)) << 4);
}

// the float value of x rounded to the nearest bf16
__device__ __forceinline__ float bf16_near(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// x = h + m + l with h, m, l each the bf16 nearest to what is left (every
// difference is exact in FP32)
__device__ __forceinline__ void split3(float x, float& h, float& m, float& l) {
  h = bf16_near(x);
  const float r = __fsub_rn(x, h);
  m = bf16_near(r);
  l = bf16_near(__fsub_rn(r, m));
}

// two floats that bf16 represents exactly, as two bf16 in one word (first in the low half)
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

// 8 consecutive K values of one operand row, sliced, as three 16-byte chunks
struct Chunk3 {
  uint4 s[3];
};
__device__ __forceinline__ Chunk3 slice8(const float (&v)[8]) {
  Chunk3 c;
  uint32_t w[3][4];
#pragma unroll
  for (int e = 0; e < 8; e += 2) {
    float h0, m0, l0, h1, m1, l1;
    split3(v[e], h0, m0, l0);
    split3(v[e + 1], h1, m1, l1);
    w[0][e >> 1] = pack2(h0, h1);
    w[1][e >> 1] = pack2(m0, m1);
    w[2][e >> 1] = pack2(l0, l1);
  }
#pragma unroll
  for (int s = 0; s < 3; ++s) c.s[s] = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
  return c;
}

// the schedule's per-tile facts, the same in every role
struct TcTile {
  const PairArgs<float>* a;
  uint32_t code;
  int side, pid, m, mp, k, n16, j0, cw;
  bool run;  // false: not a tile start, or nothing to multiply
};
__device__ __forceinline__ TcTile tc_tile(const PairArgs<float>* __restrict__ args, uint64_t t) {
  TcTile x;
  x.code = (uint32_t)(t >> 32);
  x.j0 = (int)(uint32_t)t;
  x.a = args + (x.code >> kCodeProbShift);
  x.side = (int)((x.code >> kCodeSideShift) & 1u);
  x.pid = (int)(x.code & kCodePairMask);
  x.run = false;
  x.m = x.mp = x.k = x.n16 = x.cw = 0;
  if (x.j0 % kTcCols != 0) return x;
  const PairArgs<float>& a = *x.a;
  const int N = a.ncols[x.side][x.pid];
  x.m = a.m[x.side][x.pid];
  x.k = a.rank[x.side][x.pid];
  x.mp = (x.m + 7) & ~7;
  x.n16 = 2 * ((x.k + 7) & ~7);  // B rows: real parts at [0, k), imaginary parts at [kk, kk + k)
  x.cw = min(kTcCols, N - x.j0);
  x.run = x.k > 0 && x.k <= kTcNMax / 2 && x.m > 0 && x.m <= 64 && x.cw > 0;
  return x;
}

__global__ void __launch_bounds__(kTcThreads, 1)
    rq_tc_kernel(const PairArgs<float>* __restrict__ args, const uint64_t* __restrict__ tiles, int64_t ntiles,
                 uint32_t spin_limit) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* As = smem;               // slice s, K atom a at As + s * kTcASlice + a * kTcAtom
  unsigned char* Bs = smem + kTcAStage;   // slice s, K atom a at Bs + s * kTcBSlice + a * kTcNMax * 128
  __shared__ int gcT[kTcCols];            // the tile's column table: G index
  __shared__ __align__(8) uint64_t full, empty, accfull[2], accempty[2], drain;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t lo = ntiles * blockIdx.x / gridDim.x, hi = ntiles * (blockIdx.x + 1) / gridDim.x;
  if (warp == 0) {
    tmem_alloc(&tmem_base, 2 * kTcSetCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&full, kTcProd);
    mbar_init(&empty, 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(&accfull[i], 1);
      mbar_init(&accempty[i], 128);
    }
    mbar_init(&drain, 1);
    mbar_init_fence();
    abort_flag = 0;
  }
  {
    uint4* z = reinterpret_cast<uint4*>(smem);
    for (uint32_t i = tid; i < (kTcAStage + 3 * kTcBSlice) / 16; i += kTcThreads) z[i] = make_uint4(0, 0, 0, 0);
  }
  fence_async_smem();
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tbase = tmem_base;
  const uint32_t polls = spin_limit > 0 ? spin_limit : kTcWaitPolls;
  auto wait = [&](uint64_t* bar, uint32_t parity) -> bool {
    if (*(volatile int*)&abort_flag) return false;
    if (mbar_wait(bar, parity, polls)) return true;
    atomicExch(&abort_flag, 1);
    return false;
  };
  if (warp < kTcProd / 32) {
    // ================================================================ producers
    // item (column jj, group g of 8 rows); up to 4 items per thread (mp <= 64)
    float vr[4][8], vi[4][8];
    TcTile cur;
    // the column table and the entries of tile x into vr / vi (zero outside the pair)
    auto load = [&](const TcTile& x) {
      const PairArgs<float>& a = *x.a;
      const int64_t cmo = a.cmoff[x.side][x.pid];
      named_bar_sync(kTcBarProd, kTcProd);  // no producer still reads the previous table
      if (tid < kTcCols) gcT[tid] = tid < x.cw ? a.gcol[x.side][cmo + x.j0 + tid] : 0;
      named_bar_sync(kTcBarProd, kTcProd);
      const int ng = x.mp >> 3, r0 = a.start[x.side][x.pid];
      const C2<float>* G = a.G;
      const int64_t ld = a.ld;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int it = tid + kTcProd * u;
        const int jj = x.side == 0 ? it / ng : it % kTcCols;
        const int g = x.side == 0 ? it % ng : it / kTcCols;
        const bool live = it < kTcCols * ng && jj < x.cw;
        const int64_t gc = live ? gcT[jj] : 0;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int r = 8 * g + e;
          C2<float> v{0.f, 0.f};
          if (live && r < x.m) v = x.side == 0 ? G[gc * ld + r0 + r] : G[(int64_t)(r0 + r) * ld + gc];
          vr[u][e] = v.re;
          vi[u][e] = x.side == 0 ? v.im : -v.im;  // column basis: A = conj(G^T)
        }
      }
    };
    // the B operand of tile x's pair from its Q (m x k, ld rowcap): row q =
    // [Re Q(:, q); Im Q(:, q)], row kk + q = [-Im Q(:, q); Re Q(:, q)], kk = k
    // rounded up to 8
    auto write_b = [&](const TcTile& x) {
      const PairArgs<float>& a = *x.a;
      const C2<float>* Q = a.Q[x.side] + a.Qoff[x.side][x.pid];
      const int ldq = a.rowcap[x.side][x.pid];
      const int ng = x.mp >> 3, kk = (x.k + 7) & ~7;
      for (int it = tid; it < x.k * ng; it += kTcProd) {
        const int q = it / ng, g = it % ng;
        float qr[8], qi[8], nq[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int r = 8 * g + e;
          const C2<float> v = r < x.m ? Q[r + (int64_t)q * ldq] : C2<float>{0.f, 0.f};
          qr[e] = v.re;
          qi[e] = v.im;
          nq[e] = -v.im;
        }
        const Chunk3 cr = slice8(qr), ci = slice8(qi), cn = slice8(nq);
        const int cre = g, cim = ng + g;  // K chunks of the real and imaginary parts
#pragma unroll
        for (int s = 0; s < 3; ++s) {
          unsigned char* b = Bs + s * kTcBSlice;
          *reinterpret_cast<uint4*>(b + (cre >> 3) * (kTcNMax * 128) + tc_swz(q, cre & 7)) = cr.s[s];
          *reinterpret_cast<uint4*>(b + (cim >> 3) * (kTcNMax * 128) + tc_swz(q, cim & 7)) = ci.s[s];
          *reinterpret_cast<uint4*>(b + (cre >> 3) * (kTcNMax * 128) + tc_swz(kk + q, cre & 7)) = cn.s[s];
          *reinterpret_cast<uint4*>(b + (cim >> 3) * (kTcNMax * 128) + tc_swz(kk + q, cim & 7)) = cr.s[s];
        }
      }
    };
    uint32_t tcnt = 0, prev = 0xffffffffu;
    bool ok = true;  // the same in every producer (decided by thread 0, spread by a barrier)
    int64_t i = lo;
    for (; i < hi; ++i) {
      cur = tc_tile(args, tiles[i]);
      if (cur.run) break;
    }
    if (i < hi) load(cur);
    while (i < hi && ok) {
      // the stage is free once the MMAs of the tile before have completed
      ok = named_bar_and(kTcBarProd, kTcProd, tid == 0 ? wait(&empty, (tcnt & 1u) ^ 1u) : true);
      if (!ok) break;
      if (cur.code != prev) {
        write_b(cur);
        prev = cur.code;
      }
      const int ng = cur.mp >> 3;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int it = tid + kTcProd * u;
        if (it < kTcCols * ng) {
          const int jj = cur.side == 0 ? it / ng : it % kTcCols;
          const int g = cur.side == 0 ? it % ng : it / kTcCols;
          const Chunk3 cr = slice8(vr[u]), ci = slice8(vi[u]);
          const int cre = g, cim = ng + g;
#pragma unroll
          for (int s = 0; s < 3; ++s) {
            unsigned char* a = As + s * kTcASlice;
            *reinterpret_cast<uint4*>(a + (cre >> 3) * kTcAtom + tc_swz(jj, cre & 7)) = cr.s[s];
            *reinterpret_cast<uint4*>(a + (cim >> 3) * kTcAtom + tc_swz(jj, cim & 7)) = ci.s[s];
          }
        }
      }
      fence_async_smem();
      mbar_arrive(&full);
      ++tcnt;
      for (++i; i < hi; ++i) {
        cur = tc_tile(args, tiles[i]);
        if (cur.run) break;
      }
      if (i < hi) load(cur);  // in flight while the tensor cores work on this tile
    }
  }
  else if (warp == kTcMmaWarp) {
    // ================================================================ MMA issue
    if (lane == 0) {
      const uint32_t as = smem_addr(As), bs = smem_addr(Bs);
      uint32_t tcnt = 0;
      bool ok = true;
      // slice products of weight >= 2^-16: (h,h), (h,m), (m,h), (h,l), (m,m), (l,h)
      const int pa[6] = {0, 0, 1, 0, 1, 2};
      const int pb[6] = {0, 1, 0, 2, 1, 0};
      for (int64_t i = lo; i < hi && ok; ++i) {
        const TcTile x = tc_tile(args, tiles[i]);
        if (!x.run) continue;
        const uint32_t set = tcnt & 1u;
        ok = wait(&accempty[set], ((tcnt >> 1) & 1u) ^ 1u);  // the epilogue has read this set's last tile
        if (!ok) break;
        tc_fence_after_sync();
        ok = wait(&full, tcnt & 1u);
        if (!ok) break;
        tc_fence_after_sync();
        const uint32_t idesc = idesc_bf16_f32(128, x.n16);
        const uint32_t dt = tbase + set * kTcSetCols;
        const int nks = x.mp >> 3;  // K = 2 mp in steps of 16
        for (int ks = 0; ks < nks; ++ks) {
          const uint32_t at = (uint32_t)(ks >> 2);
          const uint64_t ko = (uint64_t)(2 * (ks & 3));
#pragma unroll
          for (int p = 0; p < 6; ++p) {
            const uint64_t ad = desc_kmajor_sw128(as + pa[p] * kTcASlice + at * kTcAtom) + ko;
            const uint64_t bd = desc_kmajor_sw128(bs + pb[p] * kTcBSlice + at * (kTcNMax * 128u)) + ko;
            mma_bf16(dt, ad, bd, idesc, ks > 0 || p > 0);
          }
        }
        mma_commit(&empty);
        mma_commit(&accfull[set]);
        ++tcnt;
      }
      // every MMA issued has completed before the tensor memory is released
      mma_commit(&drain);
      mbar_wait(&drain, 0, polls);
    }
  } else {
    // ================================================================ epilogue
    const int q4 = warp & 3;
    const int jj = q4 * 32 + lane;  // TMEM lane = column of the tile
    const int et = tid - kTcEpi0 * 32;
    const uint32_t lane_base = (uint32_t)(q4 * 32) << 16;
    uint32_t tcnt = 0;
    bool ok = true;
    for (int64_t i = lo; i < hi && ok; ++i) {
      const TcTile x = tc_tile(args, tiles[i]);
      if (!x.run) continue;
      const uint32_t set = tcnt & 1u;
      ok = named_bar_and(kTcBarEpi, 128, et == 0 ? wait(&accfull[set], (tcnt >> 1) & 1u) : true);
      if (!ok) break;
      tc_fence_after_sync();
      const PairArgs<float>& a = *x.a;
      const bool live = jj < x.cw;
      const int64_t col = (int64_t)x.j0 + jj;
      const float w = live ? a.colw[x.side][a.cmoff[x.side][x.pid] + col] : 0.f;
      C2<float>* Rc = a.R[x.side] + a.Roff[x.side][x.pid] + col * a.kcap[x.side][x.pid];
      const int kk = (x.k + 7) & ~7;
      const uint32_t tc = tbase + lane_base + set * kTcSetCols;
      for (int q0 = 0; q0 < x.k; q0 += 8) {
        float re[8], im[8];
        tmem_ld8(tc + q0, re);
        tmem_ld8(tc + kk + q0, im);
        tmem_ld_wait();
        if (live) {
#pragma unroll
          for (int e = 0; e < 8; ++e)
            if (q0 + e < x.k) Rc[q0 + e] = C2<float>{re[e] * w, im[e] * w};
        }
      }
      tc_fence_before_sync();
      mbar_arrive(&accempty[set]);
      ++tcnt;
    }
  }
  tc_fence_before_sync();
  __syncthreads();
  if (abort_flag && tid == 0) atomicOr(args[0].status, kStatusTimeout);
  if (warp == 0) tmem_dealloc(tbase, 2 * kTcSetCols);
}

}  // namespace

bool launch_rq_tc(const PairArgs<float>* args, const uint64_t* tiles, int64_t ntiles, uint32_t spin_limit,
                  cudaStream_t st) {
  if (ntiles <= 0) return true;
  int dev = 0, maxopt = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || kTcSmem > (uint32_t)maxopt ||
      cudaFuncSetAttribute(rq_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const int grid = (int)std::min<int64_t>(nsm, (ntiles + 3) / 4);
  rq_tc_kernel<<<grid, kTcThreads, kTcSmem, st>>>(args, tiles, ntiles, spin_limit);
  return true;
}

}  // namespace dh2
