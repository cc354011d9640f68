// Leaf Gram matrices on the tensor cores (tcgen05, sm_103a) for the mixed
// modes: for every leaf pair (t, c) of a launch list, H = A A^* with
// A = G^omega_tc (the leaf step of Section 6: the rows of t, the columns of
// F_tc, each block's columns scaled by 1/omega_b; for the column basis the same
// on G^*).  The left singular vectors of A and its singular values are those of
// H; the factor kernel takes H from here (pivoted Cholesky, then Jacobi on the
// pivoted factor), so the m x #F_tc matrix is reduced on the tensor cores and
// only m x m data reaches the CUDA cores.
//
// A Gram matrix squares the singular values, so H must be accurate to far more
// than FP32 (the rank decision resolves sigma^2 ~ eps_l^2 ~ 1e-11 sigma_1^2
// at eps = 1e-4).  Each row of A is therefore written in fixed point relative
// to a power of two above its largest entry, as three 8-bit slices
// (a = 2^(e-6) (s1 + 2^-8 s2 + 2^-16 s3), |s1| <= 64, |s2|, |s3| <= 128, all
// integers and exact in bf16), and the slice products accumulate in FP32
// tensor memory where every partial sum is an integer below 2^24, i.e.
// exactly.  Per complex column a product adds at most 2 * 2^14 (s2 s2), so a
// window of 448 columns stays exact; longer rows are summed window by window
// in int64.  The result is H of the sliced matrix A' to ~48 bits, where A'
// differs from A by at most 2^-23 of each row's largest entry (a backward
// error of the order of the complex64 input's own rounding).
//
// Complex products as real ones: with X = Re A_p, Y = Im A_p (slice p) and
// likewise X', Y' for slice q, A_p A_q^* = (X X'^T + Y Y'^T) + i (Y X'^T - X Y'^T).
// A slice is stored as the K-major bf16 operand rows [X; Y; -X] (each block
// padded to mp = roundup(m, 8) rows), so that one M = 128 MMA on rows [0, 128)
// against B rows [0, N) (= X') and one on rows [mp, mp + 128) against B rows
// [mp, mp + N) (= Y') give the real part in TMEM lanes [0, mp) and the
// imaginary part in lanes [mp, 2 mp) of the same accumulator.  Products of
// slice pairs (1,1), (1,2), (1,3), (2,2) each have an exact accumulator; the
// (2,3) and (3,3) products (weight 2^-40 and below) share an FP32 accumulator
// whose rounding is far below the precision kept.  Since A_q A_p^* =
// (A_p A_q^*)^*, only p <= q is formed and H is symmetrised at the end.
#include <algorithm>
#include <cfloat>
#include <cstdint>
#include <cstdio>

#include "dh2_internal.h"
#include "dh2_kernels.cuh"
#include "dh2_sm100.cuh"

#include <cuda_bf16.h>

namespace dh2 {

namespace {

using namespace sm100;

#ifdef DH2_PROFILE
// summed over CTAs, seen by thread 0: pairs, chunks, then cycles in row
// scales, table loads, issuing chunk loads, waits for MMA batches, slicing,
// issuing MMAs, window flushes, H output
__device__ unsigned long long g_gprof[10];
// the pipelined form: pairs, chunks; producer thread 0: cycles waiting for a
// free stage (with the barrier), slicing, issuing loads (with table
// segments); MMA thread: waiting for a full stage, for a free accumulator set,
// issuing; epilogue thread 0: waiting for a window, flushing it, forming H
__device__ unsigned long long g_pprof[12];
#define GP_T(v) v = clock64()
#define GP_ON 1
#else
#define GP_T(v)
#define GP_ON 0
#endif

constexpr int kGramThreads = 256;
constexpr int kGramChunk = 64;        // complex columns per chunk (one 128-byte K row of bf16)
constexpr int kTableCols = 1024;      // columns of the pair's column table held in shared memory at once
static_assert(kGramWindow % kGramChunk == 0 && kTableCols % kGramChunk == 0, "chunk-aligned windows and tables");
constexpr uint32_t kWaitPolls = 1u << 23;  // default bound of a wait: about a second of polls

// Two floats that bf16 represents exactly (integers of at most 8 significant
// bits, times powers of two) as two bf16 in one word, the first in the low
// half: their upper 16 bits, since the lower 16 are zero.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

// x (|x| < 64, an FP32 value) = s1 + 2^-8 s2 + 2^-16 s3 + rest with s1, s2, s3
// the nearest integers in turn (|s1| <= 64, |s2|, |s3| <= 128): adding and
// subtracting 1.5 * 2^23 rounds to the nearest integer (ties to even) for
// |x| < 2^22, and x - s, (x - s) * 256 are exact.  Written with _rn
// intrinsics so that no step is contracted into a fused multiply-add.
__device__ __forceinline__ void slice3(float x, float& s1, float& s2, float& s3) {
  constexpr float M = 12582912.f;  // 1.5 * 2^23
  s1 = __fsub_rn(__fadd_rn(x, M), M);
  const float t1 = __fmul_rn(__fsub_rn(x, s1), 256.f);
  s2 = __fsub_rn(__fadd_rn(t1, M), M);
  const float t2 = __fmul_rn(__fsub_rn(t1, s2), 256.f);
  s3 = __fsub_rn(__fadd_rn(t2, M), M);
}

// byte offset of the 16-byte chunk g of operand row R in a 128-byte-swizzled buffer
__device__ __forceinline__ uint32_t swz(int R, int g) { return (uint32_t)R * 128u + ((uint32_t)(g ^ (R & 7)) << 4); }

// 2^ex as a float (exponent field for the normal range)
__device__ __forceinline__ float pow2f(int ex) {
  return (ex >= -126 && ex <= 127) ? __int_as_float((ex + 127) << 23) : ldexpf(1.f, ex);
}

// double-float value hi + lo of an integer |X| < 2^59, times 2^ex, from
// 32-bit conversions only: hi holds the top 24 bits of X >> 31, lo the rest
// (to within 2^11, far below 2^-40 of the largest entries of a Gram matrix)
__device__ __forceinline__ float2 ll_to_df(long long X, int ex) {
  const int xh = (int)(X >> 31);                               // |xh| < 2^28
  const float fh = __int2float_rn(xh);
  const long long rest = X - (long long)__float2int_rn(fh) * (1LL << 31);  // |rest| < 2^35
  const float fl = __int2float_rn((int)(rest >> 4)) * 16.f;
  const float h0 = fh * 2147483648.f;
  const float hs = h0 + fl;                                     // |h0| >= |fl| unless h0 == 0
  const float ls = fl - (hs - h0);
  const float sc = pow2f(ex);
  return make_float2(hs * sc, ls * sc);
}

template <int NP>
struct GramShape {
  static constexpr int MPMAX = NP;                  // mp <= NP
  static constexpr int SLROWS = MPMAX + 128;        // A reads rows [mp, mp + 128)
  static constexpr int BROWS = 2 * MPMAX + 16;      // B reads rows [mp, mp + NP)
  static constexpr uint32_t SLBYTES = SLROWS * 128u;
  static constexpr uint32_t BBYTES = BROWS * 128u;
  static constexpr int NACC = 5;
  static constexpr uint32_t TCOLS = NACC * NP <= 256 ? 256u : 512u;
  static constexpr uint32_t VSBYTES = 2 * MPMAX * (MPMAX + 1) * 8;  // the pair's window sums, 2 mp rows of mp + 1
  static constexpr uint32_t SMEM = 1024 + 3 * SLBYTES + BBYTES + VSBYTES;
};

constexpr int kBadRow = 0x7fffffff;  // row-scale marker of a non-finite entry

// Row scales of the leaf pairs of a launch list, one warp per pair: for row i
// of A = G^omega_tc the exponent e_i >= -120 with every |re|, |im| of the row
// below 2^e_i, from the block norms pass's per-block row (column basis:
// column) maxima times the block's FP32 weight -- the same value as the
// maximum over the weighted entries, since rounding a product with a positive
// factor is monotonic.  Written as int bits over the first m entries of the
// pair's Gram slot, where the Gram kernel reads them before it writes H.
__global__ void __launch_bounds__(256) gram_scales_kernel(const GramArgs* __restrict__ args,
                                                          const uint32_t* __restrict__ codes, int ncodes) {
  const int w = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (w >= ncodes) return;
  const uint32_t code = codes[w];
  const GramArgs& a = args[code >> kCodeProbShift];
  const int side = (int)((code >> kCodeSideShift) & 1u);
  const int pid = (int)(code & kCodePairMask);
  const int m = a.m[side][pid];
  if (m > 64 || m <= 0) return;  // the Gram kernel reports rows beyond its class
  const int r0 = a.start[side][pid];
  float4* Hout = a.H + a.hoff[side][pid];
  const int64_t sg0 = a.seg_begin[side][pid], sg1 = a.seg_begin[side][pid + 1];
  float mx0 = 0.f, mx1 = 0.f;  // rows lane and lane + 32
  bool bad = false;
  for (int64_t sb = sg0; sb < sg1; sb += 32) {
    const int nb = (int)(sg1 - sb < 32 ? sg1 - sb : 32);
    long long off = 0;
    float wt = 0.f;
    if (lane < nb) {
      const int b = a.seg_blk[side][sb + lane];
      const int cl = side == 0 ? a.bt[b] : a.bs[b];  // the block's cluster on this side
      // the block's maxima: rows of t+ first (row basis), then columns of s+ (column basis)
      off = a.bmax_off[b] + (side == 0 ? 0 : a.csize[a.bt[b]]) + (r0 - a.cstart[cl]);
      wt = (float)a.invw[b];
    }
    for (int k = 0; k < nb; ++k) {
      const long long o = __shfl_sync(0xffffffffu, off, k);
      const float ww = __shfl_sync(0xffffffffu, wt, k);
      if (lane < m) {
        const float x = a.bmax[o + lane] * ww;
        bad = bad || !(x <= FLT_MAX);
        mx0 = fmaxf(mx0, x);
      }
      if (lane + 32 < m) {
        const float x = a.bmax[o + lane + 32] * ww;
        bad = bad || !(x <= FLT_MAX);
        mx1 = fmaxf(mx1, x);
      }
    }
  }
  auto expo = [](float mx) {
    int e = 0;
    if (mx > 0.f) frexpf(mx, &e);  // mx < 2^e
    return e < -120 ? -120 : e;    // keeps 2^(6 - e) finite; smaller entries slice to zero
  };
  if (lane < m) Hout[lane].x = __int_as_float(bad ? kBadRow : expo(mx0));
  if (lane + 32 < m) Hout[lane + 32].x = __int_as_float(bad ? kBadRow : expo(mx1));
}

// Persistent over the launch list: CTA b takes codes b, b + grid, ...
// Eight warps: all of them load and slice (two (row, 8-column) items per
// thread and chunk); thread 0 issues the MMAs; the window sums are read from
// tensor memory by all eight (warp w: lanes 32 (w % 4) .., every other group
// of 8 columns).  The loads of chunk c + 1 are issued as soon as chunk c is
// sliced, so that they are in flight while the tensor cores work on chunk c.
template <int NP>
__global__ void __launch_bounds__(kGramThreads, GramShape<NP>::TCOLS == 512 ? 1 : 2)
    gram_kernel(const GramArgs* __restrict__ args, const uint32_t* __restrict__ codes, int ncodes) {
  using Sh = GramShape<NP>;
  constexpr int U = (64 * 8 + kGramThreads - 1) / kGramThreads;  // items per thread and chunk (m <= 64)
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sl0 = smem;
  unsigned char* bsl = smem + 3 * Sh::SLBYTES;  // slice 3 times 2^-9, rows [X; Y] (B operand of (3,3))
  long long* Vs = reinterpret_cast<long long*>(smem + 3 * Sh::SLBYTES + Sh::BBYTES);  // V, 2 mp x mp, row stride mp + 1
  __shared__ int cgcT[kTableCols];  // column table of the pair: G index of each column
  __shared__ float cwtT[kTableCols]; // and its weight 1/omega_b
  __shared__ float rsc[64];
  __shared__ int rexp[64];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    tmem_alloc(&tmem_base, Sh::TCOLS);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  {
    uint4* z = reinterpret_cast<uint4*>(smem);
    for (uint32_t i = tid; i < (3 * Sh::SLBYTES + Sh::BBYTES) / 16; i += kGramThreads) z[i] = make_uint4(0, 0, 0, 0);
  }
  fence_async_smem();
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tbase = tmem_base;
  const uint32_t sbase = smem_addr(smem);
  constexpr uint32_t idesc = idesc_bf16_f32(128, NP);
  uint32_t phase = 0;
  bool timed_out = false;
  uint32_t* st_ptr = args[0].status;
  const uint32_t polls = args[0].spin_limit > 0 ? args[0].spin_limit : kWaitPolls;
#if GP_ON
  long long gp[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  long long ga = 0, gb = 0;
#endif

  for (int ci = blockIdx.x; ci < ncodes && !timed_out; ci += gridDim.x) {
    const uint32_t code = codes[ci];
    const GramArgs& a = args[code >> kCodeProbShift];
    const int side = (int)((code >> kCodeSideShift) & 1u);
    const int pid = (int)(code & kCodePairMask);
    const int m = a.m[side][pid];
    const int N = a.ncols[side][pid];
    const int r0 = a.start[side][pid];
    const int64_t cmo = a.cmoff[side][pid];
    const int32_t* gcol = a.gcol[side] + cmo;
    const float* colw = a.colw[side] + cmo;
    const C2<float>* G = a.G;
    const int64_t ld = a.ld;
    const int mp = (m + 7) & ~7;
    float4* Hout = a.H + a.hoff[side][pid];
    st_ptr = a.status;
    if (m > NP) {  // not for this launch: reported, nothing written
      if (tid == 0) atomicOr(a.status, kStatusTooLarge);
      continue;
    }
    if (N == 0 || m == 0) {
      for (int i = tid; i < mp * mp; i += kGramThreads) Hout[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    const int nitem = m * 8;  // (row, group of 8 columns) items of a chunk
#if GP_ON
    gp[0] += 1;
    GP_T(ga);
#endif
    // column table of the pair (segments of kTableCols columns)
    auto load_table = [&](int tb) {
#if GP_ON
      long long t0 = clock64();
#endif
      __syncthreads();  // no thread still reads the previous segment
      for (int jj = tid; jj < kTableCols && tb + jj < N; jj += kGramThreads) {
        cgcT[jj] = gcol[tb + jj];
        cwtT[jj] = colw[tb + jj];
      }
      __syncthreads();
#if GP_ON
      gp[3] += clock64() - t0;
#endif
    };
    // entries of this thread's items of the chunk at j0 (zero past the chunk)
    auto load_chunk = [&](int j0, int cw, int tb, C2<float> (&v)[U][8]) {
#if GP_ON
      long long t0 = clock64();
#endif
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int q = tid + kGramThreads * u;
        const int r = q % m, g = q / m;
        // column basis: the item's 8 entries lie in one row of G; where their
        // columns are consecutive and the first is 16-byte aligned they arrive
        // as four 16-byte loads
        bool vec = false;
        int64_t e0 = 0;
        if (side == 1 && q < nitem && 8 * g + 7 < cw) {
          const int* cg = cgcT + (j0 - tb + 8 * g);
          const int gc0 = cg[0];
          e0 = (int64_t)(r0 + r) * ld + gc0;
          vec = (e0 & 1) == 0;
#pragma unroll
          for (int k = 1; k < 8; ++k) vec = vec && cg[k] == gc0 + k;
        }
        if (vec) {
          const float4* src = reinterpret_cast<const float4*>(G + e0);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float4 x = src[k];
            v[u][2 * k] = C2<float>{x.x, x.y};
            v[u][2 * k + 1] = C2<float>{x.z, x.w};
          }
        } else {
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int jj = 8 * g + k;
            v[u][k] = C2<float>{0.f, 0.f};
            if (q < nitem && jj < cw) {
              const int gc = cgcT[j0 - tb + jj];
              const int64_t e = side == 0 ? (int64_t)gc * ld + r0 + r : (int64_t)(r0 + r) * ld + gc;
              v[u][k] = G[e];
            }
          }
        }
      }
#if GP_ON
      gp[4] += clock64() - t0;
#endif
    };
    // the table and the first chunk's loads go out before the row scales, so
    // that their latencies overlap
    int tb = 0;
    load_table(0);
    C2<float> v[U][8];
    load_chunk(0, min(kGramChunk, N), 0, v);

    // ---------------------------------------------------------------- row scales
    // e_i with every |re|, |im| of row i of A below 2^e_i, from
    // gram_scales_kernel (over the first m entries of this pair's H slot;
    // kBadRow marks non-finite entries)
    {
      int bad = 0;
      if (tid < m) {
        const int e = __float_as_int(Hout[tid].x);
        bad = e == kBadRow;
        rexp[tid] = e;
        rsc[tid] = ldexpf(1.f, 6 - e);  // |a| * rsc < 64
      }
      if (__syncthreads_or(bad)) {  // non-finite entries: reported, H of this pair left as zero
        if (tid == 0) atomicOr(a.status, kStatusNaN);
        for (int k = tid; k < mp * mp; k += kGramThreads) Hout[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        continue;
      }
    }
#if GP_ON
    GP_T(gb);
    gp[2] += gb - ga;
#endif

    // ---------------------------------------------------------------- sliced products
    bool pending = false;  // an MMA batch was committed and not yet waited for
    auto wait_mma = [&]() -> bool {
#if GP_ON
      long long t0 = clock64();
#endif
      const bool ok = mbar_wait(&bar, phase, polls);
      phase ^= 1u;
      pending = false;
      const bool r = __syncthreads_or(!ok) == 0;
#if GP_ON
      gp[5] += clock64() - t0;
#endif
      return r;
    };
    // operand descriptors of this pair: slices 1-3 (rows 0 and mp) and the
    // scaled copy of slice 3
    uint64_t dA0[3], dA1[3], dB0[4], dB1[4];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const uint32_t base = sbase + (uint32_t)x * Sh::SLBYTES;  // x = 3: the scaled copy follows slice 3
      dB0[x] = desc_kmajor_sw128(base);
      dB1[x] = desc_kmajor_sw128(base + (uint32_t)mp * 128u);
      if (x < 3) {
        dA0[x] = dB0[x];
        dA1[x] = dB1[x];
      }
    }
    for (int w0 = 0; w0 < N && !timed_out; w0 += kGramWindow) {
      const int wend = min(N, w0 + kGramWindow);
      for (int j0 = w0; j0 < wend; j0 += kGramChunk) {
        const int cw = min(kGramChunk, wend - j0);
        if (pending && !wait_mma()) {  // the previous chunk's MMAs still read the slices
          timed_out = true;
          break;
        }
        // slices of this thread's items -> operand rows X (r), Y (mp + r), -X (2 mp + r)
#if GP_ON
        gp[1] += 1;
        GP_T(ga);
#endif
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int q = tid + kGramThreads * u;
          if (q >= nitem) continue;
          const int r = q % m, g = q / m;
          const float sc = rsc[r];
          uint32_t px[3][4], py[3][4], pn[3][4], pb[2][4];
#pragma unroll
          for (int k = 0; k < 8; k += 2) {
            float sx[3][2], sy[3][2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int jj = 8 * g + k + h;
              const float w = __fmul_rn(jj < cw ? cwtT[j0 - tb + jj] : 0.f, sc);  // exact: sc is a power of two
              const float xr = __fmul_rn(v[u][k + h].re, w);
              const float xi = __fmul_rn(side == 0 ? v[u][k + h].im : -v[u][k + h].im, w);
              // three 8-bit slices of each part, every step exact in FP32
              slice3(xr, sx[0][h], sx[1][h], sx[2][h]);
              slice3(xi, sy[0][h], sy[1][h], sy[2][h]);
            }
#pragma unroll
            for (int s = 0; s < 3; ++s) {
              px[s][k >> 1] = pack_bf16(sx[s][0], sx[s][1]);
              py[s][k >> 1] = pack_bf16(sy[s][0], sy[s][1]);
              pn[s][k >> 1] = px[s][k >> 1] ^ 0x80008000u;  // -X: sign bits flipped
            }
            // slice 3 times 2^-9 (a power of two: still exact in bf16)
            pb[0][k >> 1] = pack_bf16(__fmul_rn(sx[2][0], 0.001953125f), __fmul_rn(sx[2][1], 0.001953125f));
            pb[1][k >> 1] = pack_bf16(__fmul_rn(sy[2][0], 0.001953125f), __fmul_rn(sy[2][1], 0.001953125f));
          }
#pragma unroll
          for (int s = 0; s < 3; ++s) {
            unsigned char* buf = sl0 + s * Sh::SLBYTES;
            *reinterpret_cast<uint4*>(buf + swz(r, g)) = make_uint4(px[s][0], px[s][1], px[s][2], px[s][3]);
            *reinterpret_cast<uint4*>(buf + swz(mp + r, g)) = make_uint4(py[s][0], py[s][1], py[s][2], py[s][3]);
            *reinterpret_cast<uint4*>(buf + swz(2 * mp + r, g)) = make_uint4(pn[s][0], pn[s][1], pn[s][2], pn[s][3]);
          }
          *reinterpret_cast<uint4*>(bsl + swz(r, g)) = make_uint4(pb[0][0], pb[0][1], pb[0][2], pb[0][3]);
          *reinterpret_cast<uint4*>(bsl + swz(mp + r, g)) = make_uint4(pb[1][0], pb[1][1], pb[1][2], pb[1][3]);
        }
#if GP_ON
        GP_T(gb);
        gp[6] += gb - ga;
#endif
        // the next chunk's loads go out now: in flight while the tensor cores
        // work on this chunk (a new table segment waits until every thread has
        // sliced, inside load_table)
        const int jn = j0 + kGramChunk;
        if (jn < N) {
          if (jn >= tb + kTableCols) {
            tb = jn;
            load_table(tb);
          }
          load_chunk(jn, min(kGramChunk, min(N, jn < wend ? wend : jn + kGramWindow) - jn), tb, v);
        }
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
#if GP_ON
          GP_T(gb);
#endif
          tc_fence_after_sync();
          const bool first = j0 == w0;
          // products (A slice, B slice or the scaled copy, accumulator); the
          // descriptors of the pair's operand tiles are formed once, a K step
          // adds 32 bytes (2 units of 16) to their start address
          const int pa[6] = {0, 0, 0, 1, 1, 2};
          const int pb_[6] = {0, 1, 2, 1, 2, 3};  // 3 = slice 3 times 2^-9
          const int pacc[6] = {0, 1, 2, 3, 4, 4};
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
#pragma unroll
            for (int x = 0; x < 6; ++x) {
              const uint64_t ko = (uint64_t)(2 * ks);
              const uint32_t dt = tbase + (uint32_t)(pacc[x] * NP);
              const bool acc0 = !(first && ks == 0 && x != 5);
              mma_bf16(dt, dA0[pa[x]] + ko, dB0[pb_[x]] + ko, idesc, acc0);
              mma_bf16(dt, dA1[pa[x]] + ko, dB1[pb_[x]] + ko, idesc, true);
            }
          }
          mma_commit(&bar);
#if GP_ON
          gp[7] += clock64() - gb;
#endif
        }
        pending = true;
      }
      if (timed_out || (pending && !wait_mma())) {
        timed_out = true;
        break;
      }
      // window done: V += P11 2^31 + P12 2^24 + P13 2^16 + P22 2^15 + low 2^8 per lane (row of [Re; Im]);
      // every P is an integer below 2^24 held exactly in FP32.  The sums of
      // the pair's windows stay in shared memory (each entry owned by one thread).
#if GP_ON
      GP_T(ga);
#endif
      tc_fence_after_sync();
      const int L = (warp & 3) * 32 + lane;  // TMEM lane of this thread
      const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
#pragma unroll 1
      for (int cb = (warp >> 2) * 8; cb < NP; cb += 16) {
        float p11[8], p12[8], p13[8], p22[8], plo[8];
        tmem_ld8(tbase + lane_base + 0 * NP + cb, p11);
        tmem_ld8(tbase + lane_base + 1 * NP + cb, p12);
        tmem_ld8(tbase + lane_base + 2 * NP + cb, p13);
        tmem_ld8(tbase + lane_base + 3 * NP + cb, p22);
        tmem_ld8(tbase + lane_base + 4 * NP + cb, plo);
        tmem_ld_wait();
        if (L < 2 * mp) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int j = cb + i;
            if (j >= mp) break;
            long long x = (long long)__float2int_rn(p11[i]) * (1LL << 31) +
                          (long long)__float2int_rn(p12[i]) * (1LL << 24) +
                          (long long)__float2int_rn(p13[i]) * (1LL << 16) +
                          (long long)__float2int_rn(p22[i]) * (1LL << 15) + (long long)__float2int_rn(plo[i] * 256.f);
            long long* vp = Vs + (int64_t)L * (mp + 1) + j;  // padded rows: no shared-memory bank conflicts
            *vp = w0 > 0 ? *vp + x : x;
          }
        }
      }
      tc_fence_before_sync();
      __syncthreads();
#if GP_ON
      gp[8] += clock64() - ga;
#endif
    }
    if (timed_out) break;
#if GP_ON
    GP_T(ga);
#endif
    // ---------------------------------------------------------------- H = V + V^*, scaled, double-float
    for (int idx = tid; idx < m * m; idx += kGramThreads) {
      const int i = idx % m, j = idx / m;
      const int64_t ls = mp + 1;
      const long long re = Vs[(int64_t)i * ls + j] + Vs[(int64_t)j * ls + i];
      const long long im = Vs[(int64_t)(mp + i) * ls + j] - Vs[(int64_t)(mp + j) * ls + i];
      const int ex = rexp[i] + rexp[j] - 12 - 32;
      const float2 hr = ll_to_df(re, ex), hi = ll_to_df(im, ex);
      Hout[i + (int64_t)j * mp] = make_float4(hr.x, hr.y, hi.x, hi.y);
    }
    __syncthreads();  // Vs read before the next pair's first window
#if GP_ON
    gp[9] += clock64() - ga;
#endif
  }
#if GP_ON
  if (tid == 0)
    for (int i = 0; i < 10; ++i) atomicAdd(&g_gprof[i], (unsigned long long)gp[i]);
#endif
  if (timed_out && tid == 0) atomicOr(st_ptr, kStatusTimeout);
  // a timed-out batch may still be running: one more bounded wait before the
  // tensor memory is released
  if (timed_out) mbar_wait(&bar, phase, kWaitPolls);
  tc_fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, Sh::TCOLS);
}

// ---------------------------------------------------------------- pipelined form (leaves of <= 48 rows)
// One CTA per SM, 17 warps in three roles that walk the same schedule (the
// launch list's pairs, their windows of kGramWindow columns, their chunks of
// kGramChunk columns), so that no work description passes between them:
//   warps 0-11  producers: load a chunk of A, slice it into one of two
//               shared-memory stages, arrive on full[s];
//   warp 12     one thread issues the chunk's 48 MMAs into one of two
//               accumulator sets of tensor memory (one set per window,
//               alternating), then commits to empty[s] (the stage may be
//               refilled) and, after a window's last chunk, to accfull[a];
//   warps 13-16 epilogue: reads a finished window's accumulators (warp w the
//               TMEM lanes 32 (w % 4) ..), adds it to the pair's window sums
//               in shared memory, arrives on accempty[a], and after a pair's
//               last window forms H = V + V^* in double-float.
// Chunks c + 1 and c + 2 are being loaded while chunk c is sliced, slicing
// runs while the tensor cores work on the chunk before, and a pair's window
// sums and H while the next pair's chunks are sliced and multiplied.  Every
// wait is bounded: a wait that runs out sets the CTA's abort flag and every
// role leaves its schedule at its next wait.
constexpr int kPipeProd = 384;                // producer threads (warps 0-11): one item each, m <= 48
constexpr int kPipeMmaWarp = 12;
constexpr int kPipeEpi0 = 13;                 // first epilogue warp
constexpr int kPipeThreads = 17 * 32;
constexpr uint32_t kBarProd = 1, kBarEpi = 2;  // named barriers of the producers, of the epilogue

template <int NP>
struct PipeShape {
  static constexpr uint32_t SLBYTES = (NP + 128) * 128u;  // one slice: rows [X; Y; -X], MMA reads [0,128), [mp, mp+128)
  static constexpr uint32_t BBYTES = (2 * NP + 16) * 128u;  // slice 3 times 2^-9, rows [X; Y]
  static constexpr uint32_t STAGE = 3 * SLBYTES + BBYTES;
  static constexpr uint32_t VSBYTES = 2 * NP * (NP + 1) * 8;  // the pair's window sums, 2 mp rows of mp + 1
  static constexpr uint32_t SMEM = 1024 + 2 * STAGE + VSBYTES;
  static constexpr uint32_t SETCOLS = 5 * NP;  // accumulators of one set
  static_assert(STAGE % 1024 == 0 && 2 * SETCOLS <= 512, "stages on 1 KiB, two sets in 512 columns");
};

// the schedule's per-pair facts, the same in every role
struct PipePair {
  int side, pid, m, N, r0, mp;
  bool run;  // false: nothing to multiply (empty, or beyond the launch's size)
};
__device__ __forceinline__ PipePair pipe_pair(const GramArgs& a, uint32_t code, int np) {
  PipePair q;
  q.side = (int)((code >> kCodeSideShift) & 1u);
  q.pid = (int)(code & kCodePairMask);
  q.m = a.m[q.side][q.pid];
  q.N = a.ncols[q.side][q.pid];
  q.r0 = a.start[q.side][q.pid];
  q.mp = (q.m + 7) & ~7;
  q.run = q.m <= np && q.m > 0 && q.N > 0;
  return q;
}

template <int NP>
__global__ void __launch_bounds__(kPipeThreads, 1)
    gram_pipe_kernel(const GramArgs* __restrict__ args, const uint32_t* __restrict__ codes, int ncodes) {
  using Sh = PipeShape<NP>;
  static_assert(NP * 8 <= kPipeProd, "one item per producer thread");
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  long long* Vs = reinterpret_cast<long long*>(smem + 2 * Sh::STAGE);
  __shared__ int cgcT[2 * kTableCols];   // two segments of the pair's column table: G index
  __shared__ float cwtT[2 * kTableCols];  // and weight 1/omega_b of each column
  __shared__ float rsc[64];
  __shared__ int erexp[64];
  __shared__ __align__(8) uint64_t full[2], empty[2], accfull[2], accempty[2], drain;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    tmem_alloc(&tmem_base, 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&full[i], kPipeProd);
      mbar_init(&empty[i], 1);
      mbar_init(&accfull[i], 1);
      mbar_init(&accempty[i], 128);
    }
    mbar_init(&drain, 1);
    mbar_init_fence();
    abort_flag = 0;
  }
  {
    uint4* z = reinterpret_cast<uint4*>(smem);
    for (uint32_t i = tid; i < 2 * Sh::STAGE / 16; i += kPipeThreads) z[i] = make_uint4(0, 0, 0, 0);
  }
  fence_async_smem();
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tbase = tmem_base;
  const uint32_t sbase = smem_addr(smem);
  const uint32_t polls = args[0].spin_limit > 0 ? args[0].spin_limit : kWaitPolls;
  // a bounded wait; false (and the abort flag set) when it runs out
  auto wait = [&](uint64_t* bar, uint32_t parity) -> bool {
    if (*(volatile int*)&abort_flag) return false;
    if (mbar_wait(bar, parity, polls)) return true;
    atomicExch(&abort_flag, 1);
    return false;
  };

  if (warp < kPipeProd / 32) {
    // ================================================================ producers
    // one (row, 8-column group) item per thread and chunk; the entries of
    // chunks c + 1 and c + 2 are in flight while chunk c is sliced.  The
    // column table is held in two segment buffers of kTableCols columns
    // (segment k in buffer k % 2), so that a chunk's weights are still there
    // when it is sliced after the next segment has been loaded.
    uint32_t cc = 0;  // chunks produced
    bool ok = true;   // the same in every producer thread (decided by thread 0, spread by a barrier)
#if GP_ON
    long long pw = 0, psl = 0, pld = 0, npair = 0;
#endif
    for (int ci = blockIdx.x; ci < ncodes && ok; ci += gridDim.x) {
      const uint32_t code = codes[ci];
      const GramArgs& a = args[code >> kCodeProbShift];
      const PipePair q = pipe_pair(a, code, NP);
      if (!q.run) continue;
#if GP_ON
      ++npair;
#endif
      const int m = q.m, N = q.N, mp = q.mp, side = q.side, r0 = q.r0;
      const int64_t cmo = a.cmoff[side][q.pid];
      const int32_t* gcol = a.gcol[side] + cmo;
      const float* colw = a.colw[side] + cmo;
      const C2<float>* G = a.G;
      const int64_t ld = a.ld;
      const float4* Hin = a.H + a.hoff[side][q.pid];
      const int nitem = m * 8;
      const int r = tid % m, g = tid / m;  // this thread's item
      const bool live = tid < nitem;
      const int nch = (N + kGramChunk - 1) / kGramChunk;
      int seg_loaded = 0;  // segments 0 .. seg_loaded - 1 have been loaded (the last two are held)
      auto load_table = [&](int sg) {
        named_bar_sync(kBarProd, kPipeProd);  // no producer still reads segment sg - 2 (its buffer)
        const int t0 = sg * kTableCols, b = (sg & 1) * kTableCols;
        for (int jj = tid; jj < kTableCols && t0 + jj < N; jj += kPipeProd) {
          cgcT[b + jj] = gcol[t0 + jj];
          cwtT[b + jj] = colw[t0 + jj];
        }
        named_bar_sync(kBarProd, kPipeProd);
      };
      // entries of this thread's item of chunk jc (zero past the pair)
      auto load_chunk = [&](int jc, C2<float> (&v)[8]) {
        const int j0 = jc * kGramChunk;
        if (j0 >= N) return;
#if GP_ON
        const long long t0 = clock64();
#endif
        const int sg = j0 / kTableCols;
        if (sg >= seg_loaded) {  // chunks run in order: the next segment
          load_table(sg);
          seg_loaded = sg + 1;
        }
        const int cw = min(kGramChunk, N - j0);
        const int* cg = cgcT + ((sg & 1) * kTableCols + j0 - sg * kTableCols + 8 * g);
        bool vec = false;
        int64_t e0 = 0;
        if (side == 1 && live && 8 * g + 7 < cw) {
          const int gc0 = cg[0];
          e0 = (int64_t)(r0 + r) * ld + gc0;
          vec = (e0 & 1) == 0;
#pragma unroll
          for (int k = 1; k < 8; ++k) vec = vec && cg[k] == gc0 + k;
        }
        if (vec) {
          const float4* src = reinterpret_cast<const float4*>(G + e0);
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float4 x = src[k];
            v[2 * k] = C2<float>{x.x, x.y};
            v[2 * k + 1] = C2<float>{x.z, x.w};
          }
        } else {
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int jj = 8 * g + k;
            v[k] = C2<float>{0.f, 0.f};
            if (live && jj < cw) {
              const int gc = cg[k];
              const int64_t e = side == 0 ? (int64_t)gc * ld + r0 + r : (int64_t)(r0 + r) * ld + gc;
              v[k] = G[e];
            }
          }
        }
#if GP_ON
        pld += clock64() - t0;
#endif
      };
      C2<float> vA[8], vB[8];
      load_chunk(0, vA);
      load_chunk(1, vB);
      if (tid < m) {
        const int e = __float_as_int(Hin[tid].x);  // row scale from gram_scales_kernel (kBadRow: see the epilogue)
        rsc[tid] = ldexpf(1.f, 6 - (e == kBadRow ? 0 : e));
      }
      named_bar_sync(kBarProd, kPipeProd);
      const float sc = live ? rsc[r] : 0.f;
      // slice chunk jc from v into its stage, then refill v with chunk jc + 2
      auto produce = [&](int jc, C2<float> (&v)[8]) -> bool {
        const uint32_t s = cc & 1u;
#if GP_ON
        const long long t0 = clock64();
#endif
        // stage s is free once the MMAs of the chunk it held have completed
        if (!named_bar_and(kBarProd, kPipeProd, tid == 0 ? wait(&empty[s], ((cc >> 1) & 1u) ^ 1u) : true))
          return false;
#if GP_ON
        const long long t1 = clock64();
        pw += t1 - t0;
#endif
        unsigned char* sl0 = smem + s * Sh::STAGE;
        unsigned char* bsl = sl0 + 3 * Sh::SLBYTES;
        const int j0 = jc * kGramChunk, cw = min(kGramChunk, N - j0), sg = j0 / kTableCols;
        const float* cwp = cwtT + ((sg & 1) * kTableCols + j0 - sg * kTableCols + 8 * g);
        if (live) {
          uint32_t px[3][4], py[3][4], pn[3][4], pb[2][4];
#pragma unroll
          for (int k = 0; k < 8; k += 2) {
            float sx[3][2], sy[3][2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const float wt = __fmul_rn(8 * g + k + h < cw ? cwp[k + h] : 0.f, sc);  // exact: sc is a power of two
              const float xr = __fmul_rn(v[k + h].re, wt);
              const float xi = __fmul_rn(side == 0 ? v[k + h].im : -v[k + h].im, wt);
              slice3(xr, sx[0][h], sx[1][h], sx[2][h]);
              slice3(xi, sy[0][h], sy[1][h], sy[2][h]);
            }
#pragma unroll
            for (int t = 0; t < 3; ++t) {
              px[t][k >> 1] = pack_bf16(sx[t][0], sx[t][1]);
              py[t][k >> 1] = pack_bf16(sy[t][0], sy[t][1]);
              pn[t][k >> 1] = px[t][k >> 1] ^ 0x80008000u;
            }
            pb[0][k >> 1] = pack_bf16(__fmul_rn(sx[2][0], 0.001953125f), __fmul_rn(sx[2][1], 0.001953125f));
            pb[1][k >> 1] = pack_bf16(__fmul_rn(sy[2][0], 0.001953125f), __fmul_rn(sy[2][1], 0.001953125f));
          }
#pragma unroll
          for (int t = 0; t < 3; ++t) {
            unsigned char* buf = sl0 + t * Sh::SLBYTES;
            *reinterpret_cast<uint4*>(buf + swz(r, g)) = make_uint4(px[t][0], px[t][1], px[t][2], px[t][3]);
            *reinterpret_cast<uint4*>(buf + swz(mp + r, g)) = make_uint4(py[t][0], py[t][1], py[t][2], py[t][3]);
            *reinterpret_cast<uint4*>(buf + swz(2 * mp + r, g)) = make_uint4(pn[t][0], pn[t][1], pn[t][2], pn[t][3]);
          }
          *reinterpret_cast<uint4*>(bsl + swz(r, g)) = make_uint4(pb[0][0], pb[0][1], pb[0][2], pb[0][3]);
          *reinterpret_cast<uint4*>(bsl + swz(mp + r, g)) = make_uint4(pb[1][0], pb[1][1], pb[1][2], pb[1][3]);
        }
        fence_async_smem();
        mbar_arrive(&full[s]);
#if GP_ON
        psl += clock64() - t1;
#endif
        ++cc;
        load_chunk(jc + 2, v);
        return true;
      };
      for (int jc = 0; jc < nch && ok; jc += 2) {
        ok = produce(jc, vA);
        if (ok && jc + 1 < nch) ok = produce(jc + 1, vB);
      }
      if (ok) named_bar_sync(kBarProd, kPipeProd);  // rsc and the table are read before the next pair rewrites them
    }
#if GP_ON
    if (tid == 0) {
      atomicAdd(&g_pprof[0], (unsigned long long)npair);
      atomicAdd(&g_pprof[1], (unsigned long long)cc);
      atomicAdd(&g_pprof[2], (unsigned long long)pw);
      atomicAdd(&g_pprof[3], (unsigned long long)psl);
      atomicAdd(&g_pprof[4], (unsigned long long)pld);
    }
#endif
  } else if (warp == kPipeMmaWarp) {
    // ================================================================ MMA issue
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16_f32(128, NP);
      uint32_t cc = 0, wc = 0;  // chunks and windows consumed
      bool ok = true;
#if GP_ON
      long long mwf = 0, mwa = 0, mis = 0;
#endif
      for (int ci = blockIdx.x; ci < ncodes && ok; ci += gridDim.x) {
        const uint32_t code = codes[ci];
        const PipePair q = pipe_pair(args[code >> kCodeProbShift], code, NP);
        if (!q.run) continue;
        for (int w0 = 0; w0 < q.N && ok; w0 += kGramWindow, ++wc) {
          const int wend = min(q.N, w0 + kGramWindow);
          const uint32_t aset = wc & 1u;
#if GP_ON
          long long t0 = clock64();
#endif
          ok = wait(&accempty[aset], ((wc >> 1) & 1u) ^ 1u);  // the epilogue has read this set's last window
#if GP_ON
          mwa += clock64() - t0;
#endif
          tc_fence_after_sync();
          for (int j0 = w0; j0 < wend && ok; j0 += kGramChunk, ++cc) {
            const uint32_t s = cc & 1u;
#if GP_ON
            long long t1 = clock64();
#endif
            ok = wait(&full[s], (cc >> 1) & 1u);
            if (!ok) break;
#if GP_ON
            long long t2 = clock64();
            mwf += t2 - t1;
#endif
            tc_fence_after_sync();
            const uint32_t base = sbase + s * Sh::STAGE;
            const bool first = j0 == w0;
            // the stage's operand descriptors, formed once per chunk: slices 1-3
            // and the scaled copy of slice 3, at rows 0 and mp; a K step adds 32
            // bytes (2 units of 16) to the start address field
            uint64_t d0[4], d1[4];
#pragma unroll
            for (int x = 0; x < 4; ++x) {
              d0[x] = desc_kmajor_sw128(base + (uint32_t)x * Sh::SLBYTES);
              d1[x] = desc_kmajor_sw128(base + (uint32_t)x * Sh::SLBYTES + (uint32_t)q.mp * 128u);
            }
            const uint32_t dt0 = tbase + aset * Sh::SETCOLS;
            // products in an order where no two consecutive MMAs write the same
            // accumulator: (1,1), (2,2), (1,2), (2,3), (1,3), (3,3)/512, first on
            // rows 0 (X' columns) then on rows mp (Y' columns)
            const int pa[6] = {0, 1, 0, 1, 0, 2};
            const int pbx[6] = {0, 1, 1, 2, 2, 3};  // 3 = slice 3 times 2^-9
            const int pacc[6] = {0, 3, 1, 4, 2, 4};
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
              const uint64_t ko = (uint64_t)(2 * ks);
#pragma unroll
              for (int x = 0; x < 6; ++x) {
                // the window's first MMA into an accumulator overwrites it ((3,3)
                // follows (2,3) into the same one)
                const bool acc0 = !(first && ks == 0 && x != 5);
                mma_bf16(dt0 + (uint32_t)(pacc[x] * NP), d0[pa[x]] + ko, d0[pbx[x]] + ko, idesc, acc0);
              }
#pragma unroll
              for (int x = 0; x < 6; ++x)
                mma_bf16(dt0 + (uint32_t)(pacc[x] * NP), d1[pa[x]] + ko, d1[pbx[x]] + ko, idesc, true);
            }
            mma_commit(&empty[s]);
            if (j0 + kGramChunk >= wend) mma_commit(&accfull[aset]);
#if GP_ON
            mis += clock64() - t2;
#endif
          }
        }
      }
#if GP_ON
      atomicAdd(&g_pprof[5], (unsigned long long)mwf);
      atomicAdd(&g_pprof[6], (unsigned long long)mwa);
      atomicAdd(&g_pprof[7], (unsigned long long)mis);
#endif
      // every MMA issued has completed before the tensor memory is released
      mma_commit(&drain);
      mbar_wait(&drain, 0, kWaitPolls);
    }
  } else {
    // ================================================================ epilogue
    const int q4 = warp & 3;
    const int L = q4 * 32 + lane;  // TMEM lane of this thread
    const int et = tid - kPipeEpi0 * 32;  // 0..127
    const uint32_t lane_base = (uint32_t)(q4 * 32) << 16;
    uint32_t wc = 0;
    bool ok = true;
#if GP_ON
    long long ew = 0, efl = 0, eh = 0;
#endif
    for (int ci = blockIdx.x; ci < ncodes && ok; ci += gridDim.x) {
      const uint32_t code = codes[ci];
      const GramArgs& a = args[code >> kCodeProbShift];
      const PipePair q = pipe_pair(a, code, NP);
      float4* Hout = a.H + a.hoff[q.side][q.pid];
      const int m = q.m, mp = q.mp;
      if (!q.run) {
        if (m > NP) {
          if (et == 0) atomicOr(a.status, kStatusTooLarge);
        } else {
          for (int i = et; i < mp * mp; i += 128) Hout[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        continue;
      }
      if (et < m) erexp[et] = __float_as_int(Hout[et].x);
      named_bar_sync(kBarEpi, 128);
      for (int w0 = 0; w0 < q.N && ok; w0 += kGramWindow, ++wc) {
        const uint32_t aset = wc & 1u;
#if GP_ON
        long long t0 = clock64();
#endif
        ok = named_bar_and(kBarEpi, 128, et == 0 ? wait(&accfull[aset], (wc >> 1) & 1u) : true);
        if (!ok) break;
#if GP_ON
        long long t1 = clock64();
        ew += t1 - t0;
#endif
        tc_fence_after_sync();
#pragma unroll 1
        for (int cb = 0; cb < mp; cb += 8) {
          float p11[8], p12[8], p13[8], p22[8], plo[8];
          const uint32_t tc = tbase + lane_base + aset * Sh::SETCOLS + cb;
          tmem_ld8(tc + 0 * NP, p11);
          tmem_ld8(tc + 1 * NP, p12);
          tmem_ld8(tc + 2 * NP, p13);
          tmem_ld8(tc + 3 * NP, p22);
          tmem_ld8(tc + 4 * NP, plo);
          tmem_ld_wait();
          if (L < 2 * mp) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int j = cb + i;
              if (j >= mp) break;
              long long x = (long long)__float2int_rn(p11[i]) * (1LL << 31) +
                            (long long)__float2int_rn(p12[i]) * (1LL << 24) +
                            (long long)__float2int_rn(p13[i]) * (1LL << 16) +
                            (long long)__float2int_rn(p22[i]) * (1LL << 15) + (long long)__float2int_rn(plo[i] * 256.f);
              long long* vp = Vs + (int64_t)L * (mp + 1) + j;  // the pair's sums, owned by this thread
              *vp = w0 > 0 ? *vp + x : x;
            }
          }
        }
        tc_fence_before_sync();
        mbar_arrive(&accempty[aset]);
#if GP_ON
        efl += clock64() - t1;
#endif
      }
      if (!ok) break;
#if GP_ON
      long long t2 = clock64();
#endif
      named_bar_sync(kBarEpi, 128);  // the pair's sums are in Vs
      bool bad = false;
      for (int i = 0; i < m; ++i) bad = bad || erexp[i] == kBadRow;
      if (bad) {  // non-finite entries: reported, H of this pair left as zero
        if (et == 0) atomicOr(a.status, kStatusNaN);
        for (int i = et; i < mp * mp; i += 128) Hout[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      } else {
        for (int idx = et; idx < m * m; idx += 128) {
          const int i = idx % m, j = idx / m;
          const int64_t ls = mp + 1;
          const long long re = Vs[(int64_t)i * ls + j] + Vs[(int64_t)j * ls + i];
          const long long im = Vs[(int64_t)(mp + i) * ls + j] - Vs[(int64_t)(mp + j) * ls + i];
          const int ex = erexp[i] + erexp[j] - 12 - 32;
          const float2 hr = ll_to_df(re, ex), hi = ll_to_df(im, ex);
          Hout[i + (int64_t)j * mp] = make_float4(hr.x, hr.y, hi.x, hi.y);
        }
      }
      named_bar_sync(kBarEpi, 128);  // Vs and erexp read before the next pair's first window
#if GP_ON
      eh += clock64() - t2;
#endif
    }
#if GP_ON
    if (et == 0) {
      atomicAdd(&g_pprof[8], (unsigned long long)ew);
      atomicAdd(&g_pprof[9], (unsigned long long)efl);
      atomicAdd(&g_pprof[10], (unsigned long long)eh);
    }
#endif
  }
  tc_fence_before_sync();
  __syncthreads();
  if (abort_flag && tid == 0) atomicOr(args[0].status, kStatusTimeout);
  if (warp == 0) tmem_dealloc(tbase, 512);
}

template <int NP>
bool launch_np(const GramArgs* args, const uint32_t* codes, int n, cudaStream_t st) {
  using Sh = GramShape<NP>;
  // shared memory per CTA is padded so that the CTAs an SM can hold never ask
  // for more tensor memory than its 512 columns (2 CTAs of 256, or 1 of 512)
  const size_t smem = std::max<size_t>(Sh::SMEM, Sh::TCOLS == 512 ? 120 * 1024 : 80 * 1024);
  auto kern = gram_kernel<NP>;
  int dev = 0, maxopt = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || smem > (size_t)maxopt ||
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  // the whole shared-memory carveout: two CTAs of the 256-column classes per SM
  cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  cudaGetLastError();
  // CTAs per SM from the SM's registers and shared memory (the occupancy
  // query reports one CTA for these kernels where two run side by side),
  // capped by tensor memory: 512 columns per SM
  cudaFuncAttributes fa{};
  int smem_sm = 0, regs_sm = 0;
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const int regs_cta = ((fa.numRegs * 32 + 255) / 256 * 256) * (kGramThreads / 32);  // per-warp granules of 256
  const int by_regs = regs_cta > 0 ? regs_sm / regs_cta : 1;
  const int by_smem = smem_sm / (int)(smem + fa.sharedSizeBytes + 1024);  // 1 KiB reserved per CTA
  const int per_sm = std::max(1, std::min(std::min(by_regs, by_smem), (int)(512 / Sh::TCOLS)));
#ifdef DH2_PROFILE
  {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kGramThreads, smem);
    std::fprintf(stderr, "dh2 gram<%d>: %d pairs, %d CTAs per SM (occupancy query: %d), %zu + %zu B shared, %d registers\n",
                 NP, n, per_sm, occ, smem, fa.sharedSizeBytes, fa.numRegs);
  }
#endif
  const int grid = std::min(n, nsm * per_sm);
  gram_scales_kernel<<<(n + 7) / 8, 256, 0, st>>>(args, codes, n);
  kern<<<grid, kGramThreads, smem, st>>>(args, codes, n);
  return true;
}

}  // namespace

void prof_reset_gram() {
#ifdef DH2_PROFILE
  unsigned long long z[12] = {};
  cudaMemcpyToSymbol(g_gprof, z, 10 * sizeof(unsigned long long));
  cudaMemcpyToSymbol(g_pprof, z, sizeof(z));
#endif
}

bool prof_read_gram(unsigned long long* out22) {
#ifdef DH2_PROFILE
  cudaMemcpyFromSymbol(out22, g_gprof, 10 * sizeof(unsigned long long));
  cudaMemcpyFromSymbol(out22 + 10, g_pprof, 12 * sizeof(unsigned long long));
  return true;
#else
  (void)out22;
  return false;
#endif
}

// the pipelined kernel: one CTA per SM
template <int NP>
bool launch_pipe(const GramArgs* args, const uint32_t* codes, int n, cudaStream_t st) {
  using Sh = PipeShape<NP>;
  auto kern = gram_pipe_kernel<NP>;
  int dev = 0, maxopt = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      Sh::SMEM > (uint32_t)maxopt ||
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const int grid = std::min(n, nsm);
#ifdef DH2_PROFILE
  std::fprintf(stderr, "dh2 gram_pipe<%d>: %d pairs, grid %d, %u B shared\n", NP, n, grid, Sh::SMEM);
#endif
  gram_scales_kernel<<<(n + 7) / 8, 256, 0, st>>>(args, codes, n);
  kern<<<grid, kPipeThreads, Sh::SMEM, st>>>(args, codes, n);
  return true;
}

bool launch_gram(const GramArgs* args_dev, const uint32_t* codes, int n, int maxm, cudaStream_t st) {
  if (n <= 0) return true;
  if (maxm <= 32) return launch_pipe<32>(args_dev, codes, n, st);
  if (maxm <= 48) return launch_pipe<48>(args_dev, codes, n, st);
  if (maxm <= 64) return launch_np<64>(args_dev, codes, n, st);
  return false;
}

}  // namespace dh2
