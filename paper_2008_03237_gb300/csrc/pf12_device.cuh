// Device building blocks of the pair-F12 kernels: a CTA-wide GEMM tile, the
// FP64 right-looking Cholesky of an augmented matrix (factor + forward solve in
// one sweep), the FP64 backward solve, and a fixed-order block reduction.
//
// Every routine is executed by all kThreads threads of one CTA and works on a
// single pair's workspace; none waits on another CTA.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pf12_internal.h"

namespace pf12 {

// Shared tiles of the CTA GEMM.  FP64 products: A and B as double[kBK][kTile
// + 1].  FP32 products: A and B as float[kBK][kTileF] (rows 16-byte aligned
// for vector loads), followed by the raw FP64 stage of the next K chunk
// (16 values per thread, copied with cp.async while the current chunk is
// computed).
constexpr int kTileF = kTile + 4;
constexpr int kTilesF64 = 2 * kBK * (kTile + 1);          // doubles
constexpr int kRawOff = kBK * kTileF;                     // doubles (= 2 kBK kTileF floats)
constexpr int kRawLen = 16 * kThreads;                    // doubles
struct __align__(128) GemmSmem {
  double buf[kTilesF64 > kRawOff + kRawLen ? kTilesF64 : kRawOff + kRawLen];
};

struct __align__(16) CholSmem {
  double d[kNB][kNB + 1];  // diagonal block of L
  double inv[kNB];         // 1 / L_tt
  int ok;
};

// ---------------------------------------------------------------------------
// CTA GEMM tile:  C[r, c] = (acc ? C[r, c] : 0) + alpha * sum_{t<K} A(r, t) B(t, c)
// for r0 <= r < min(r0 + 64, M), c0 <= c < min(c0 + 64, N), where
//   A(r, t) = TA ? A[t * lda + r] : A[r * lda + t]
//   B(t, c) = TB ? B[c * ldb + t] : B[t * ldb + c].
// FP64 <-> FP32 conversions in integer arithmetic.  On this part the FP64 pipe
// is the bottleneck and executes the hardware conversions too; these run on
// the integer pipes instead, for every input (no hardware fallback, so that a
// warp in an FP32 phase never queues behind the co-resident CTAs' DFMAs).
// Binary64 -> binary32 rounds to nearest, ties to even: keep 23 of the 52
// fraction bits, rebias the exponent (1023 -> 127) and add one unit when the
// 29 dropped bits exceed half a unit, or equal it with an odd kept fraction (a
// carry into the exponent is the correct result, including the step to
// infinity).  Results below the binary32 normal range are rounded the same way
// at the subnormal spacing 2^-149; exponents above it overflow to infinity;
// NaN stays NaN.
__device__ __forceinline__ float f64_to_f32_rne(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned int hi = static_cast<unsigned int>(b >> 32), lo = static_cast<unsigned int>(b);
  const unsigned int sign = hi & 0x80000000u;
  const unsigned int e = (hi >> 20) & 0x7ffu;
  if (e - (1023u - 126u) <= 253u) {
    // (hi, lo) << 3 keeps the low 9 exponent bits, e - 512 for these e, on
    // top of the 23 kept fraction bits; rebias by 384 to e - 896
    unsigned int r = (__funnelshift_l(lo, hi, 3) - (384u << 23)) | sign;
    const unsigned int rest = lo & 0x1fffffffu;
    // +1 when rest > half, or rest == half with an odd kept fraction
    r += (rest + (r & 1u) + 0x0fffffffu) >> 29;
    return __uint_as_float(r);
  }
  if (e == 0x7ffu)   // infinity, or NaN (quiet, sign kept)
    return __uint_as_float(sign | ((b & 0xfffffffffffffull) ? 0x7fc00000u : 0x7f800000u));
  if (e > 1023u + 127u) return __uint_as_float(sign | 0x7f800000u);
  // binary32 subnormal or zero: significand * 2^(e - 1075) in units of 2^-149
  const unsigned int shift = 926u - e;          // > 29 here; e = 0 is below any result
  if (e == 0u || shift > 54u) return __uint_as_float(sign);
  const unsigned long long m53 = (b & 0xfffffffffffffull) | (1ull << 52);
  unsigned int q = static_cast<unsigned int>(m53 >> shift);
  const unsigned long long rem = m53 & ((1ull << shift) - 1ull), half = 1ull << (shift - 1u);
  q += (rem > half || (rem == half && (q & 1u))) ? 1u : 0u;
  return __uint_as_float(sign | q);
}

// Binary32 -> binary64, exact: rebias the exponent (127 -> 1023) and widen the
// fraction; subnormals are normalised, infinity and NaN keep their class.
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int e = (u >> 23) & 0xffu;
  const unsigned long long sign = static_cast<unsigned long long>(u & 0x80000000u) << 32;
  const unsigned long long frac = u & 0x7fffffu;
  unsigned long long b;
  if (e != 0u && e != 0xffu) {
    b = sign | (static_cast<unsigned long long>(e + 896u) << 52) | (frac << 29);
  } else if (e == 0xffu) {
    b = sign | (0x7ffull << 52) | (frac << 29);
  } else if (frac == 0u) {
    b = sign;
  } else {           // subnormal: frac * 2^-149 with its top bit at position n
    const unsigned int n = 31u - static_cast<unsigned int>(__clz(static_cast<int>(frac)));
    b = sign | (static_cast<unsigned long long>(n + 874u) << 52) |
        ((frac << (52u - n)) & 0xfffffffffffffull);
  }
  return __longlong_as_double(static_cast<long long>(b));
}

// FP32-product tile (TC = float): 256 threads as a 16 x 16 grid of 4 x 4
// output blocks, rows 4 (tid / 16) + i, columns 4 (tid % 16) + j, fed by one
// 16-byte shared load of A and one of B per K step (16 FFMAs).  FP64 operands
// are copied to the raw stage with cp.async one chunk ahead (zero-filled
// outside the matrices) and rounded to FP32 by the thread that copied them.
// Two-level FP32 summation: each 32-wide K chunk is summed on its own and
// then added to a running sum, so the rounding error grows as
// sqrt(32 + K / 32) units instead of sqrt(K); the sum is widened to FP64 once,
// in the epilogue, and no FP64 instruction runs before it (none at all for a
// plain store with alpha = +-1).  No triangular restriction (tri_rows).
template <bool TA, bool TB>
__device__ __forceinline__ void cta_gemm_tile_f32(int M, int N, int K, const double* A,
                                                  int64_t lda, const double* B, int64_t ldb,
                                                  double* C, int64_t ldc, int r0, int c0,
                                                  double alpha, bool accumulate, GemmSmem& sm) {
  float (*as)[kTileF] = reinterpret_cast<float (*)[kTileF]>(sm.buf);
  float (*bs)[kTileF] = reinterpret_cast<float (*)[kTileF]>(reinterpret_cast<float*>(sm.buf) + kBK * kTileF);
  double* raw = sm.buf + kRawOff;
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  const bool act = r0 + 4 * ty < M && c0 + 4 * tx < N;
  // operand (t, r) of A and (t, c) of B staged by this thread as its s-th value
  auto a_at = [&](int s, int& r, int& t) {
    if (!TA) { t = tid & 31; r = (tid >> 5) + 8 * s; }
    else     { r = tid & 63; t = (tid >> 6) + 4 * s; }
  };
  auto b_at = [&](int s, int& c, int& t) {
    if (TB) { t = tid & 31; c = (tid >> 5) + 8 * s; }
    else    { c = tid & 63; t = (tid >> 6) + 4 * s; }
  };
  auto issue_raw = [&](int k0) {
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      int r, t;
      a_at(s, r, t);
      const int gr = r0 + r, gt = k0 + t;
      const bool ok = gr < M && gt < K;
      const double* src = ok ? (TA ? A + (int64_t)gt * lda + gr : A + (int64_t)gr * lda + gt) : A;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(
                       static_cast<uint32_t>(__cvta_generic_to_shared(raw + s * kThreads + tid))),
                   "l"(src), "r"(ok ? 8 : 0)
                   : "memory");
    }
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      int c, t;
      b_at(s, c, t);
      const int gc = c0 + c, gt = k0 + t;
      const bool ok = gc < N && gt < K;
      const double* src = ok ? (TB ? B + (int64_t)gc * ldb + gt : B + (int64_t)gt * ldb + gc) : B;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(
                       static_cast<uint32_t>(__cvta_generic_to_shared(raw + (8 + s) * kThreads + tid))),
                   "l"(src), "r"(ok ? 8 : 0)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  float accf[4][4], accs[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { accf[i][j] = 0.0f; accs[i][j] = 0.0f; }

  if (K > 0) issue_raw(0);   // K = 0: no copy in flight; the epilogue stores +-0
  for (int k0 = 0; k0 < K; k0 += kBK) {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      int r, t;
      a_at(s, r, t);
      as[t][r] = f64_to_f32_rne(raw[s * kThreads + tid]);
    }
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      int c, t;
      b_at(s, c, t);
      bs[t][c] = f64_to_f32_rne(raw[(8 + s) * kThreads + tid]);
    }
    if (k0 + kBK < K) issue_raw(k0 + kBK);   // in flight during this chunk's products
    __syncthreads();
    if (act) {
      const int kn = min(kBK, K - k0);
#pragma unroll 4
      for (int kk = 0; kk < kn; ++kk) {
        const float4 a = *reinterpret_cast<const float4*>(&as[kk][4 * ty]);
        const float4 b = *reinterpret_cast<const float4*>(&bs[kk][4 * tx]);
        const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) accf[i][j] = fmaf(av[i], bv[j], accf[i][j]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          accs[i][j] = __fadd_rn(accs[i][j], accf[i][j]);
          accf[i][j] = 0.0f;
        }
    }
    __syncthreads();
  }
  if (!act) return;
  // Epilogue: a plain store of +-(sum) needs no FP64 instruction (the sign is
  // a bit flip; alpha is compared by its bits).
  const long long abits = __double_as_longlong(alpha);
  const bool plain = !accumulate && (abits == 0x3ff0000000000000ll ||
                                     abits == (long long)0xbff0000000000000ull);
  const unsigned long long flip = (abits < 0) ? 0x8000000000000000ull : 0ull;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + 4 * ty + i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + 4 * tx + j;
      if (c >= N) continue;
      double* pc = C + (int64_t)r * ldc + c;
      const double v = f32_to_f64(accs[i][j]);
      if (plain)
        *pc = __longlong_as_double(
            (long long)((unsigned long long)__double_as_longlong(v) ^ flip));
      else
        *pc = accumulate ? fma(alpha, v, *pc) : alpha * v;
    }
  }
}

// The 64 x 64 tile is split into 32 blocks of RB x (128 / RB): 8 x 16 by
// default, 4 x 32 for products with few rows (the triangular solves' 2k
// right-hand sides, where 8-row blocks would carry up to 6 rows of zeros).  A
// block is active when it meets [0, M) x [0, N) and, if tri_rows > 0, is not
// entirely above the diagonal within the first tri_rows rows.  Active blocks
// are dealt round-robin to the 8 warps (at most 4 each; lane: 2 x 2 outputs,
// rows lr + (RB / 2) i, columns lc + (64 / RB) j, conflict-free shared-memory
// reads), so ragged edges and the upper halves of diagonal tiles cost no
// arithmetic and the remaining work is spread evenly over the warps.
// TC is the product type: double (FP64 FMAs, this routine) or float (FP32
// FMAs, cta_gemm_tile_f32, which has no triangular restriction).  Operands may
// alias C's array as long as the tile's own C entries are not read as A/B.
// All threads must call; the C stores follow the last barrier and are read
// back only by the thread that wrote them.
template <typename TC, bool TA, bool TB, int RB = 8>
__device__ __forceinline__ void cta_gemm_tile(int M, int N, int K, const double* A, int64_t lda,
                                              const double* B, int64_t ldb, double* C,
                                              int64_t ldc, int r0, int c0, double alpha,
                                              bool accumulate, GemmSmem& sm, int tri_rows = 0) {
  static_assert(RB == 8 || RB == 4, "row block of 8 or 4");
  constexpr int CB = 128 / RB;       // block columns
  constexpr int LC = CB / 2;         // lanes along a block's columns
  constexpr int LR = 32 / LC;        // lanes along its rows (= RB / 2)
  constexpr int NCB = kTile / CB;    // blocks across the tile
  if constexpr (sizeof(TC) != sizeof(double)) {
    cta_gemm_tile_f32<TA, TB>(M, N, K, A, lda, B, ldb, C, ldc, r0, c0, alpha, accumulate, sm);
    return;
  } else {
  double (*as)[kTile + 1] = reinterpret_cast<double (*)[kTile + 1]>(sm.buf);
  double (*bs)[kTile + 1] = reinterpret_cast<double (*)[kTile + 1]>(sm.buf + kBK * (kTile + 1));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lr = lane / LC, lc = lane % LC;
  // this warp's blocks: tile-local origins (row, col); -1 = unused slot
  int orow[4] = {-1, -1, -1, -1}, ocol[4] = {0, 0, 0, 0};
  {
    int cnt = 0, slot = 0;
#pragma unroll
    for (int b = 0; b < 32; ++b) {
      const int br = r0 + RB * (b / NCB), bc = c0 + CB * (b % NCB);
      bool act = br < M && bc < N;
      if (tri_rows > 0 && br + RB - 1 < tri_rows && bc > br + RB - 1) act = false;
      if (act) {
        if ((cnt & 7) == warp && slot < 4) {
          orow[slot] = RB * (b / NCB);
          ocol[slot] = CB * (b % NCB);
          ++slot;
        }
        ++cnt;
      }
    }
  }
  const bool any = orow[0] >= 0;
  double accd[4][2][2];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) accd[q][i][j] = 0.0;

  for (int k0 = 0; k0 < K; k0 += kBK) {
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      int r, t;
      if (!TA) { t = tid & 31; r = (tid >> 5) + 8 * s; }
      else     { r = tid & 63; t = (tid >> 6) + 4 * s; }
      const int gr = r0 + r, gt = k0 + t;
      double v = 0.0;
      if (gr < M && gt < K) v = TA ? A[(int64_t)gt * lda + gr] : A[(int64_t)gr * lda + gt];
      as[t][r] = v;
    }
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      int c, t;
      if (TB) { t = tid & 31; c = (tid >> 5) + 8 * s; }
      else    { c = tid & 63; t = (tid >> 6) + 4 * s; }
      const int gc = c0 + c, gt = k0 + t;
      double v = 0.0;
      if (gc < N && gt < K) v = TB ? B[(int64_t)gc * ldb + gt] : B[(int64_t)gt * ldb + gc];
      bs[t][c] = v;
    }
    __syncthreads();
    if (any) {
      const int kn = min(kBK, K - k0);
#pragma unroll 4
      for (int kk = 0; kk < kn; ++kk) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (orow[q] < 0) continue;
          const double a0 = as[kk][orow[q] + lr], a1 = as[kk][orow[q] + lr + LR];
          const double b0 = bs[kk][ocol[q] + lc], b1 = bs[kk][ocol[q] + lc + LC];
          accd[q][0][0] = fma(a0, b0, accd[q][0][0]);
          accd[q][0][1] = fma(a0, b1, accd[q][0][1]);
          accd[q][1][0] = fma(a1, b0, accd[q][1][0]);
          accd[q][1][1] = fma(a1, b1, accd[q][1][1]);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (orow[q] < 0) continue;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int r = r0 + orow[q] + lr + LR * i;
      if (r >= M) continue;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int c = c0 + ocol[q] + lc + LC * j;
        if (c >= N) continue;
        double* pc = C + (int64_t)r * ldc + c;
        *pc = accumulate ? fma(alpha, accd[q][i][j], *pc) : alpha * accd[q][i][j];
      }
    }
  }
  }
}

// Whole-matrix product over all 64 x 64 output tiles of an M x N result.
template <typename TC, bool TA, bool TB, int RB = 8>
__device__ __forceinline__ void cta_gemm(int M, int N, int K, const double* A, int64_t lda,
                                         const double* B, int64_t ldb, double* C, int64_t ldc,
                                         double alpha, bool accumulate, GemmSmem& sm) {
  for (int r0 = 0; r0 < M; r0 += kTile)
    for (int c0 = 0; c0 < N; c0 += kTile)
      cta_gemm_tile<TC, TA, TB, RB>(M, N, K, A, lda, B, ldb, C, ldc, r0, c0, alpha, accumulate,
                                    sm);
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Blocked Cholesky of the leading m x m block of M (row-major, leading
// dimension ld, lower triangle used), FP64, extended to the extra rows
// [m, rows): on return M[0:m, 0:m] holds L (lower) and M[m:rows, 0:m] holds
// M[m:rows] L^{-T}, i.e. the forward solve rides along the factorisation as
// extra rows of every panel solve and update.  Entries above the diagonal are
// scratch.  Returns false on every thread when a pivot is not positive and
// finite (J_g not SPD).
//
// Panels are kNB = 32 wide and grouped LOOK at a time (8 by default; the
// autotuner also tries 16): inside a group each panel is first brought up to
// date by the group's earlier panels (a narrow left-looking update), then
// factored (warp-level diagonal block, in-register panel solve); the columns
// right of the group get one update of depth LOOK * 32.  The trailing matrix
// is thus read and written once per group instead of once per panel; the flop
// count is unchanged.
constexpr int kLook = 8;

template <int kLook = pf12::kLook>
__device__ __forceinline__ bool chol_augmented(double* M, int64_t ld, int m, int rows,
                                               CholSmem& cs, GemmSmem& gs) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int g0 = 0; g0 < m; g0 += kLook * kNB) {
    const int gend = min(m, g0 + kLook * kNB);
    for (int kb = g0; kb < gend; kb += kNB) {
      const int nb = min(kNB, m - kb);
      // bring panel [kb, kb + nb) up to date with the group's earlier panels
      if (kb > g0) {
        for (int R = kb; R < rows; R += kTile)
          cta_gemm_tile<double, false, true>(rows, kb + nb, kb - g0, M + g0, ld, M + g0, ld, M, ld,
                                             R, kb, -1.0, true, gs, m);
        __syncthreads();
      }
      for (int e = tid; e < nb * nb; e += kThreads) {
        const int r = e / nb, c = e - r * nb;
        cs.d[r][c] = (c <= r) ? M[(int64_t)(kb + r) * ld + kb + c] : 0.0;
      }
      __syncthreads();
      if (warp == 0) {
        int ok = 1;
        for (int j = 0; j < nb; ++j) {
          const double djj = cs.d[j][j];
          if (!(djj > 0.0) || !isfinite(djj)) ok = 0;
          const double l = sqrt(djj);
          const double inv = 1.0 / l;
          __syncwarp();
          if (lane == j) { cs.d[j][j] = l; cs.inv[j] = inv; }
          if (lane > j && lane < nb) cs.d[lane][j] *= inv;
          __syncwarp();
          if (lane > j && lane < nb) {
            const double lrj = cs.d[lane][j];
            for (int c = j + 1; c <= lane; ++c) cs.d[lane][c] = fma(-lrj, cs.d[c][j], cs.d[lane][c]);
          }
          __syncwarp();
        }
        if (lane == 0) cs.ok = ok;
      }
      __syncthreads();
      if (!cs.ok) return false;
      for (int e = tid; e < nb * nb; e += kThreads) {
        const int r = e / nb, c = e - r * nb;
        if (c <= r) M[(int64_t)(kb + r) * ld + kb + c] = cs.d[r][c];
      }
      // panel solve: rows below the diagonal block, X L_kk^T = A_panel
      for (int r = kb + nb + tid; r < rows; r += kThreads) {
        double* row = M + (int64_t)r * ld + kb;
        double x[kNB];
#pragma unroll
        for (int t = 0; t < kNB; ++t) x[t] = (t < nb) ? row[t] : 0.0;
#pragma unroll
        for (int t = 0; t < kNB; ++t) {
          if (t < nb) {
            double s = x[t];
#pragma unroll
            for (int q = 0; q < t; ++q) s = fma(-x[q], cs.d[t][q], s);
            x[t] = s * cs.inv[t];
          }
        }
#pragma unroll
        for (int t = 0; t < kNB; ++t)
          if (t < nb) row[t] = x[t];
      }
      __syncthreads();
    }
    // one deep update of everything right of the group (lower part and every
    // extra row) with the group's kLook panels
    const int rb = gend;
    for (int R = rb; R < rows; R += kTile)
      for (int C = rb; C < m && C < R + kTile; C += kTile)
        cta_gemm_tile<double, false, true>(rows, m, gend - g0, M + g0, ld, M + g0, ld, M, ld, R, C,
                                           -1.0, true, gs, m);
    __syncthreads();
  }
  return true;
}

// ---------------------------------------------------------------------------
// Triangular solves with the Cholesky factor for nrows rows of Y (leading
// dimension ldy; L is m x m lower triangular, leading dimension ld, only its
// lower triangle is read).  Columns go in blocks of kNB, grouped kSolveGroup
// blocks at a time as in the factorisation: inside a group every block first
// takes a left-looking update from the group's solved blocks (depth < 256),
// then a small in-register triangular solve (one thread per row); after the
// group one deep update of depth up to 256 carries it to the remaining
// columns, so Y is read and written once per group instead of once per block.
constexpr int kSolveGroup = 8;

// In-register solve of the nb-column block at c0 of every row, with the
// block's diagonal block of L staged in cs; forward (lower, L^T on the right)
// or backward (L on the right) order.
template <bool kForward>
__device__ __forceinline__ void solve_block(const double* L, int64_t ld, double* Y, int64_t ldy,
                                            int nrows, int c0, int nb, CholSmem& cs) {
  const int tid = threadIdx.x;
  for (int e = tid; e < nb * nb; e += kThreads) {
    const int r = e / nb, c = e - r * nb;
    cs.d[r][c] = (c <= r) ? L[(int64_t)(c0 + r) * ld + c0 + c] : 0.0;
  }
  __syncthreads();
  if (tid < nb) cs.inv[tid] = 1.0 / cs.d[tid][tid];
  __syncthreads();
  for (int r = tid; r < nrows; r += kThreads) {
    double* row = Y + (int64_t)r * ldy + c0;
    double x[kNB];
#pragma unroll
    for (int t = 0; t < kNB; ++t) x[t] = (t < nb) ? row[t] : 0.0;
    if (kForward) {
#pragma unroll
      for (int t = 0; t < kNB; ++t) {
        if (t < nb) {
          double sum = x[t];
#pragma unroll
          for (int q = 0; q < t; ++q) sum = fma(-x[q], cs.d[t][q], sum);
          x[t] = sum * cs.inv[t];
        }
      }
    } else {
#pragma unroll
      for (int t = kNB - 1; t >= 0; --t) {
        if (t < nb) {
          double sum = x[t];
#pragma unroll
          for (int q = t + 1; q < kNB; ++q)
            if (q < nb) sum = fma(-x[q], cs.d[q][t], sum);
          x[t] = sum * cs.inv[t];
        }
      }
    }
#pragma unroll
    for (int t = 0; t < kNB; ++t)
      if (t < nb) row[t] = x[t];
  }
  __syncthreads();
}

// Backward solve Y <- Y L^{-1}: column blocks from the right.
__device__ __forceinline__ void solve_right_lower(const double* L, int64_t ld, int m, double* Y,
                                                  int64_t ldy, int nrows, CholSmem& cs,
                                                  GemmSmem& gs) {
  const int nblk = (m + kNB - 1) / kNB;
  for (int gb_hi = nblk; gb_hi > 0;) {
    const int gb_lo = max(0, gb_hi - kSolveGroup);
    const int g0 = gb_lo * kNB, g1 = min(m, gb_hi * kNB);
    for (int cb = gb_hi - 1; cb >= gb_lo; --cb) {
      const int c0 = cb * kNB, nb = min(kNB, m - c0), cend = c0 + nb;
      if (cend < g1) {   // Y_blk -= X[:, cend:g1] L[cend:g1, blk]
        cta_gemm<double, false, false, 4>(nrows, nb, g1 - cend, Y + cend, ldy,
                                       L + (int64_t)cend * ld + c0, ld, Y + c0, ldy, -1.0, true, gs);
        __syncthreads();
      }
      solve_block<false>(L, ld, Y, ldy, nrows, c0, nb, cs);
    }
    if (g0 > 0) {        // Y[:, 0:g0] -= X[:, g0:g1] L[g0:g1, 0:g0]
      cta_gemm<double, false, false, 4>(nrows, g0, g1 - g0, Y + g0, ldy, L + (int64_t)g0 * ld, ld, Y,
                                     ldy, -1.0, true, gs);
      __syncthreads();
    }
    gb_hi = gb_lo;
  }
}

// Forward solve Y <- Y L^{-T}: column blocks from the left.
__device__ __forceinline__ void solve_right_lowerT(const double* L, int64_t ld, int m, double* Y,
                                                   int64_t ldy, int nrows, CholSmem& cs,
                                                   GemmSmem& gs) {
  for (int g0 = 0; g0 < m; g0 += kSolveGroup * kNB) {
    const int g1 = min(m, g0 + kSolveGroup * kNB);
    for (int kb = g0; kb < g1; kb += kNB) {
      const int nb = min(kNB, m - kb);
      if (kb > g0) {     // Y_blk -= X[:, g0:kb] L[blk, g0:kb]^T
        cta_gemm<double, false, true, 4>(nrows, nb, kb - g0, Y + g0, ldy, L + (int64_t)kb * ld + g0,
                                      ld, Y + kb, ldy, -1.0, true, gs);
        __syncthreads();
      }
      solve_block<true>(L, ld, Y, ldy, nrows, kb, nb, cs);
    }
    if (g1 < m) {        // Y[:, g1:m] -= X[:, g0:g1] L[g1:m, g0:g1]^T
      cta_gemm<double, false, true, 4>(nrows, m - g1, g1 - g0, Y + g0, ldy, L + (int64_t)g1 * ld + g0,
                                    ld, Y + g1, ldy, -1.0, true, gs);
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// Gather mode: sieve pair P's four factor blocks out of the per-orbital
// pair-extended blocks (Sec. "F12 integral transformations") into dst as
// packed p x m blocks [Ag_i, Ag_j, Af_i, Af_j].
//
// TMA path (tensor maps present): the pair's rows go in groups of four through
// tile::gather4 loads (4 arbitrary rows x 128 columns, column start rounded
// down to 16 bytes) into shared memory, up to 8 loads per mbarrier phase; the
// threads then pick the pair's columns out of each staged window.  Plain path
// (no maps, or columns spread over more than 32 windows): rows to warps,
// columns to lanes (the columns are atom runs, so reads are coalesced).
struct SieveCtl {
  unsigned long long mbar;  // TMA completion barrier
  int win[33];              // window start indices into the pair's column map
  int flag;                 // bounded wait expired
};

constexpr int kSieveW = 128;         // columns per gather4 box
constexpr int kSieveOps = 8;         // gather4 loads per phase (8 x 4 KB staging)
constexpr uint32_t kSieveWait = 1u << 26;

__device__ __forceinline__ void sieve_init(SieveCtl& sc) {
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(&sc.mbar))
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    sc.flag = 0;
  }
  __syncthreads();
}

// Returns false (uniformly) when a bounded TMA wait expired.
__device__ __forceinline__ bool sieve_pair(const FwdParams& prm, const PairDesc& pd, double* dst,
                                           GemmSmem& gs, SieveCtl& sc, uint32_t& phase) {
  static_assert(sizeof(GemmSmem) >= kSieveOps * 4 * kSieveW * sizeof(double), "sieve staging");
  const GatherDesc g = prm.gdesc[pd.pair];
  const int p = pd.p, m = pd.m;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int32_t* rows[2] = {prm.map_pao + g.map_pao, prm.map_pao + g.map_pao + p};
  const int32_t* cols[2] = {prm.map_aux + g.map_aux, prm.map_aux + g.map_aux + m};
  const int64_t off[2] = {g.off_i, g.off_j};
  const int32_t ldo[2] = {g.ld_i, g.ld_j};
  const int orb[2] = {g.orb_i, g.orb_j};
  double* tiles = gs.buf;   // kSieveOps x 4 x kSieveW doubles, 128-byte aligned
  const uint32_t tiles_s = (uint32_t)__cvta_generic_to_shared(tiles);
  const uint32_t mbar_s = (uint32_t)__cvta_generic_to_shared(&sc.mbar);
#pragma unroll 1
  for (int x = 0; x < 4; ++x) {
    const int side = x & 1;
    const int32_t* rw = rows[side];
    const int32_t* cl = cols[side];
    double* out = dst + (int64_t)x * p * m;
    const int c_lo = cl[0] & ~1;
    const int nw = (cl[m - 1] - c_lo) / kSieveW + 1;
    if (!prm.tmaps || nw > 32) {
      const double* src = (x < 2 ? prm.Bg : prm.Bf) + off[side];
      for (int r = warp; r < p; r += kThreads / 32) {
        const double* row = src + (int64_t)rw[r] * ldo[side];
        for (int c = lane; c < m; c += 32) out[(int64_t)r * m + c] = row[cl[c]];
      }
      __syncthreads();
      continue;
    }
    const char* tmap = static_cast<const char*>(prm.tmaps) + (size_t)(2 * orb[side] + (x >= 2)) * 128;
    // window w holds pair columns [win[w], win[w + 1])
    if (tid <= nw) {
      const int bound = c_lo + tid * kSieveW;
      int lo = 0, hi = m;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cl[mid] < bound) lo = mid + 1; else hi = mid;
      }
      sc.win[tid] = lo;
    }
    __syncthreads();
    const int ngroups = (p + 3) / 4;
    const int total = ngroups * nw;
    for (int op0 = 0; op0 < total; op0 += kSieveOps) {
      const int nops = min(kSieveOps, total - op0);
      if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmap) : "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar_s),
                     "r"((uint32_t)(nops * 4 * kSieveW * 8))
                     : "memory");
        for (int q = 0; q < nops && prm.debug_wait_polls == 0; ++q) {
          const int op = op0 + q, grp = op / nw, w = op - grp * nw;
          int r[4];
#pragma unroll
          for (int s4 = 0; s4 < 4; ++s4) r[s4] = rw[min(4 * grp + s4, p - 1)];
          const int xc = c_lo + w * kSieveW;
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
              " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(tiles_s + q * 4 * kSieveW * 8),
              "l"(tmap), "r"(xc), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(mbar_s)
              : "memory");
        }
        uint32_t done = 0;
        const uint32_t limit = prm.debug_wait_polls ? prm.debug_wait_polls : kSieveWait;
        for (uint32_t it = 0; it < limit && !done; ++it)
          asm volatile(
              "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
              " selp.u32 %0, 1, 0, p;\n}\n"
              : "=r"(done)
              : "r"(mbar_s), "r"(phase)
              : "memory");
        if (!done) sc.flag = 1;
      }
      __syncthreads();
      phase ^= 1u;
      if (sc.flag) return false;
      // pick the pair's columns out of the staged windows
      for (int q = 0; q < nops; ++q) {
        const int op = op0 + q, grp = op / nw, w = op - grp * nw;
        const int ca = sc.win[w], cb = sc.win[w + 1];
        const int xc = c_lo + w * kSieveW;
        const double* tq = tiles + q * 4 * kSieveW;
        const int width = cb - ca;
        for (int e = tid; e < 4 * width; e += kThreads) {
          const int s4 = e / width, c = ca + (e - s4 * width);
          const int r = 4 * grp + s4;
          if (r < p) out[(int64_t)r * m + c] = tq[s4 * kSieveW + (cl[c] - xc)];
        }
      }
      __syncthreads();
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// Fixed-order CTA sum of two per-thread values (deterministic for a fixed
// kThreads): butterfly within each warp, then warps in index order.
__device__ __forceinline__ void cta_sum2(double& a, double& b, double (*red)[kThreads / 32]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (lane == 0) { red[0][warp] = a; red[1][warp] = b; }
  __syncthreads();
  double sa = 0.0, sb = 0.0;
  for (int w = 0; w < kThreads / 32; ++w) { sa += red[0][w]; sb += red[1][w]; }
  __syncthreads();
  a = sa;
  b = sb;
}

// ---------------------------------------------------------------------------
// SOMO-augmented PNO space (Sec. "SOMO handling"): every PAO domain holds the
// s SOMOs and the PAO-to-PNO matrix is blockdiag(Q, I_s).  A pair's factor
// blocks carry the SOMO rows after its p PAO rows; its virtual space is the
// kq = k - s PNOs followed by the SOMOs.  The SOMOs are alpha-occupied, so the
// alpha virtuals are the PNOs only and the beta virtuals are all k.

// Rows kq .. k - 1 of At^x = Q_aug^T A^x: the SOMO rows p .. p + s - 1 of A^x
// (the identity block of Q_aug), copied exactly.
__device__ __forceinline__ void copy_somo_rows(const double* A, int p, int s, int m, double* At,
                                               int64_t ld, int kq) {
  for (int r = threadIdx.x >> 5; r < s; r += kThreads / 32)
    for (int c = threadIdx.x & 31; c < m; c += 32)
      At[(int64_t)(kq + r) * ld + c] = A[(int64_t)(p + r) * m + c];
}

// Rows p .. p + s - 1 of dA^x = Q_aug H: the SOMO rows kq .. k - 1 of H.
__device__ __forceinline__ void copy_somo_grad_rows(const double* H, int64_t ld, int kq, int s,
                                                    int m, double* dA, int p) {
  for (int r = threadIdx.x >> 5; r < s; r += kThreads / 32)
    for (int c = threadIdx.x & 31; c < m; c += 32)
      dA[(int64_t)(p + r) * m + c] = H[(int64_t)(kq + r) * ld + c];
}

// Energy weights of an augmented pair by virtual block q = 2 [a is a SOMO] +
// [b is a SOMO]: E_P = sum_ab wd(q) V_ab T_ab + wx(q) V_ab T_ba with
//   (i alpha, j beta): 3/8 V_ab T_ab over a alpha, b beta; 1/8 V_ab T_ba over a beta, b alpha
//   (j alpha, i beta): the same with the roles of a and b exchanged
//   same spin sigma:   1/4 V_ab (T_ab - T_ba) over a, b both sigma virtuals.
// Block 0 (both PNOs) gives the plain weights w_alpha, w_beta.
__device__ __forceinline__ void somo_block_weights(const PairDesc& pd, int q, double& wd,
                                                   double& wx) {
  const double c1 = pd.c1, c2 = pd.n_ab - pd.c1, naa = pd.n_aa, nbb = pd.n_bb;
  if (q == 0) {
    wd = 3.0 * pd.n_ab / 8.0 + (naa + nbb) / 4.0;
    wx = pd.n_ab / 8.0 - (naa + nbb) / 4.0;
  } else if (q == 1) {        // a PNO, b SOMO
    wd = 3.0 * c1 / 8.0 + nbb / 4.0;
    wx = c2 / 8.0 - nbb / 4.0;
  } else if (q == 2) {        // a SOMO, b PNO
    wd = 3.0 * c2 / 8.0 + nbb / 4.0;
    wx = c1 / 8.0 - nbb / 4.0;
  } else {                    // both SOMOs: beta-beta only
    wd = nbb / 4.0;
    wx = -nbb / 4.0;
  }
}

// Steps 4-5 of an augmented pair: block sums D_q = sum V_ab T_ab and
// X_q = sum V_ab T_ba over the four virtual blocks (fixed order), then the
// spin cases.  Every thread returns e[3]; D, X are the unrestricted totals.
__device__ __forceinline__ void somo_pair_energy(const PairDesc& pd, const double* V,
                                                 const double* T, double (*red)[kThreads / 32],
                                                 double e[3], double& D, double& X) {
  const int k = pd.k, kq = pd.k - pd.s;
  double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0, x0 = 0.0, x1 = 0.0, x2 = 0.0, x3 = 0.0;
  for (int el = threadIdx.x; el < k * k; el += kThreads) {
    const int a = el / k, b = el - a * k;
    const double v = V[el];
    const double td = v * T[el], tx = v * T[b * k + a];
    if (a < kq) {
      if (b < kq) { d0 += td; x0 += tx; } else { d1 += td; x1 += tx; }
    } else {
      if (b < kq) { d2 += td; x2 += tx; } else { d3 += td; x3 += tx; }
    }
  }
  cta_sum2(d0, x0, red);
  cta_sum2(d1, x1, red);
  cta_sum2(d2, x2, red);
  cta_sum2(d3, x3, red);
  const double c1 = pd.c1, c2 = pd.n_ab - pd.c1;
  // (i alpha, j beta): a in PNOs, b anywhere for D; a anywhere, b in PNOs for X
  e[0] = c1 * (3.0 * (d0 + d1) + (x0 + x2)) / 8.0 + c2 * (3.0 * (d0 + d2) + (x0 + x1)) / 8.0;
  e[1] = pd.n_aa * (d0 - x0) / 4.0;
  D = ((d0 + d1) + d2) + d3;
  X = ((x0 + x1) + x2) + x3;
  e[2] = pd.n_bb * (D - X) / 4.0;
}

// ---------------------------------------------------------------------------
// Streamed inputs: bounded wait of one thread for an arrival flag written by a
// copy on another stream.

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// True once ready[g] has reached epoch (wrap-safe comparison); false when
// timeout_ns passed first (the poll count is capped as well).
__device__ __forceinline__ bool wait_ready(const uint32_t* ready, int g, uint32_t epoch,
                                           uint64_t timeout_ns) {
  const uint64_t t0 = global_ns();
  const uint64_t max_polls = timeout_ns / 64 + 1024;
  const size_t addr = __cvta_generic_to_global(ready + g);
  for (uint64_t polls = 0;; ++polls) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(addr) : "memory");
    if ((int32_t)(v - epoch) >= 0) return true;
    if (polls >= max_polls || global_ns() - t0 > timeout_ns) return false;
    __nanosleep(128);
  }
}

// Thread 0 of the CTA: take the next queue slot; with streamed inputs wait for
// its group's flag.  A CTA's slots only grow, so its groups never go back and
// it polls once per new group; groups may land in any order.  Returns the
// slot, n_pairs when the queue is done or stopped, or -1 after an expired wait
// (the pair is marked status 3 and the stop flag set).
__device__ __forceinline__ long long next_slot(const FwdParams& prm, int& known_group) {
  long long sl = (prm.err && *prm.err != 0) ? prm.n_pairs : atomicAdd(prm.counter, 1);
  if (sl < prm.n_pairs && prm.ready) {
    const int g = prm.slot_group[sl];
    if (g > known_group) {
      if (wait_ready(prm.ready, g, prm.epoch, prm.arrival_timeout_ns)) {
        known_group = g;
      } else {
        prm.status[prm.desc[sl].pair] = 3;
        atomicExch(prm.err, 1);
        sl = -1;
      }
    }
  }
  return sl;
}

// ---------------------------------------------------------------------------
// Auxiliary metrics as full row-major blocks or as packed lower triangles
// (row r holds J[r][0..r] at r (r + 1) / 2): a symmetric metric then travels
// and rests in about half the bytes.

// Copy of a rows x cols block (lower = false) or of the lower triangle of a
// square block, diagonal included (lower = true), from global memory into the
// slab (row stride dld).  The source rows have stride sld, or, with packed
// (lower only), are the packed lower triangle (row r at r (r + 1) / 2).  All
// threads walk the region in row-major order, 256 elements apart, with eight
// loads in flight each before their stores: the copy is bound by memory
// latency, not bandwidth.
__device__ __forceinline__ void copy_region(const double* src, int64_t sld, int rows, int cols,
                                            bool lower, bool packed, double* dst, int64_t dld) {
  constexpr int kU = 8;
  if (rows <= 0 || cols <= 0) return;
  auto advance = [&](int& r, int& c, int step) {
    c += step;
    while (r < rows) {
      const int len = lower ? r + 1 : cols;
      if (c < len) break;
      c -= len;
      ++r;
    }
  };
  int r = 0, c = static_cast<int>(threadIdx.x);
  advance(r, c, 0);
  while (r < rows) {
    double v[kU];
    int rr = r, cc = c;
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t at = packed ? (int64_t)rr * (rr + 1) / 2 + cc : (int64_t)rr * sld + cc;
      v[u] = (rr < rows) ? src[at] : 0.0;
      advance(rr, cc, kThreads);
    }
    rr = r;
    cc = c;
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      if (rr < rows) dst[(int64_t)rr * dld + cc] = v[u];
      advance(rr, cc, kThreads);
    }
    r = rr;
    c = cc;
  }
}

// J_g (full or packed lower triangle) into the slab's leading m x m block:
// only the lower triangle, diagonal included, which is all the factorisation
// and the solves read; the entries above the diagonal are scratch.
__device__ __forceinline__ void load_metric(const double* J, int m, bool packed, double* M,
                                            int64_t ld) {
  copy_region(J, m, m, m, /*lower=*/true, packed, M, ld);
}

// Full symmetric m x m J_f (row stride ld) from its packed lower triangle.
__device__ __forceinline__ void unpack_metric(const double* J, int m, double* W, int64_t ld) {
  const int lane = threadIdx.x & 31;
  for (int r = threadIdx.x >> 5; r < m; r += kThreads / 32) {
    const double* row = J + (int64_t)r * (r + 1) / 2;
    for (int c = lane; c <= r; c += 32) {
      const double v = row[c];
      W[(int64_t)r * ld + c] = v;
      W[(int64_t)c * ld + r] = v;
    }
  }
}

}  // namespace pf12
