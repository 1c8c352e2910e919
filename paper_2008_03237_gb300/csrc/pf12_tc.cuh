// 5th-generation tensor-core (tcgen05) GEMM tile for the mixable contractions
// of the pair path, in split TF32 ("TF32x3"):  x = hi + lo with hi = tf32(x),
// lo = tf32(x - hi);  A B ~= A_hi B_hi + A_hi B_lo + A_lo B_hi, every product
// exact in the FP32 accumulator, which lives in tensor memory (TMEM).
//
// One CTA computes D (128 x N, N <= 128, N % 16 == 0 after padding) for
//   D[r][n] = sum_t A(r, t) B(n, t)
// with A(r, t) = TA ? A[t * lda + r] : A[r * lda + t] (FP64 in global memory)
// and  B(n, t) = TB ? B[t * ldb + n] : B[n * ldb + t];
// K is consumed in 32-wide chunks staged by all threads (FP64 -> FP32 -> tf32
// hi/lo, canonical K-major layout without swizzle; the FP64 <-> FP32
// conversions run on the integer pipes, not on the FP64 pipe that bounds the
// pair kernels), one thread issues the
// MMAs, a commit to an mbarrier signals completion, and after every chunk the
// FP32 accumulator is added into the FP64 output Out[n * ldo + r] (scaled by
// alpha): short FP32 spans keep the accumulator's rounding bias small.  Every wait is bounded; on expiry the routine returns false.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pf12_device.cuh"   // FP64 <-> FP32 conversions on the integer pipes

namespace pf12 {
namespace tc {

constexpr int kM = 128;        // rows per tile (TMEM lanes)
constexpr int kNmax = 128;     // columns per tile (TMEM columns allocated)
constexpr int kKC = 32;        // K chunk staged at once (4 MMA k-steps of 8)
constexpr int kPromote = 1;    // chunks accumulated in TMEM before the FP64 add
constexpr uint32_t kWaitLimit = 1u << 26;

// shared-memory staging: A hi/lo (128 x 32 tf32) and B hi/lo (128 x 32 tf32)
struct __align__(1024) Stage {
  uint32_t a_hi[kM * kKC];
  uint32_t a_lo[kM * kKC];
  uint32_t b_hi[kNmax * kKC];
  uint32_t b_lo[kNmax * kKC];
};

struct Ctrl {
  unsigned long long mbar;  // MMA completion barrier
  uint32_t tmem_base;       // TMEM address written by tcgen05.alloc
  uint32_t phase;           // next parity to wait for
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Canonical K-major layout without swizzle: 8-row x 16-byte core matrices,
// K-adjacent cores 128 B apart (leading byte offset), 8-row groups
// kKC/4 * 128 B apart (stride byte offset).  Byte offset of element (r, t):
__device__ __forceinline__ uint32_t kmajor_offset(int r, int t) {
  return (uint32_t)((r >> 3) * (kKC / 4) * 128 + (t >> 2) * 128 + (r & 7) * 16 + (t & 3) * 4);
}

// tcgen05 shared-memory matrix descriptor (no swizzle): start address,
// leading and stride byte offsets (all >> 4), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::tf32: D FP32, A and B TF32, both K-major,
// N >> 3 and M >> 4 in their fields.
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return u;
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Allocate kNmax TMEM columns (one warp, warp-uniform) and init the barrier.
__device__ __forceinline__ void setup(Ctrl& c) {
  const int warp = threadIdx.x >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&c.tmem_base)),
                 "r"((uint32_t)kNmax)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&c.mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    c.phase = 0;
  }
  fence_before();
  __syncthreads();
  fence_after();
}

// Free the TMEM columns (same warp as setup); all MMAs must have completed.
__device__ __forceinline__ void teardown(Ctrl& c) {
  fence_before();
  __syncthreads();
  fence_after();
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(c.tmem_base),
                 "r"((uint32_t)kNmax)
                 : "memory");
  }
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ bool mbar_wait(Ctrl& c, uint32_t limit = kWaitLimit) {
  const uint32_t addr = smem_addr(&c.mbar), par = c.phase;
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(par)
        : "memory");
    if (done) return true;
  }
  return false;
}

// One tile: Out[n * ldo + r0 + r] (+)= alpha * sum_t A(r0 + r, t) B(n0 + n, t)
// for r < min(128, M - r0), n < min(128, N - n0).  accumulate = false
// overwrites Out.  Called by all threads; returns false (uniformly) on a
// barrier timeout.
// debug_polls != 0 (tests only): issue no MMA, so nothing arrives on the
// barrier, and poll it debug_polls times: the bounded wait expires.
template <bool TA, bool TB>
__device__ bool gemm_tile(int M, int N, int K, const double* A, int64_t lda, const double* B,
                          int64_t ldb, double* Out, int64_t ldo, int r0, int n0, double alpha,
                          bool accumulate, Stage& st, Ctrl& c, int* s_flag,
                          uint32_t debug_polls = 0) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nthreads = blockDim.x;
  const int rows = min(kM, M - r0);
  const int ncols = min(kNmax, N - n0);
  const int npad = (ncols + 15) / 16 * 16;
  const uint32_t idesc = idesc_tf32(kM, npad);
  const uint32_t lbo = 128, sbo = (kKC / 4) * 128;
  bool first_in_span = true;
  const int nchunks = (K + kKC - 1) / kKC;
  for (int ch = 0; ch < nchunks; ++ch) {
    const int k0 = ch * kKC;
    // stage A: 128 x 32 (rows beyond M, K beyond K are zero)
    for (int e = tid; e < kM * kKC; e += nthreads) {
      int r, t;
      if (TA) { r = e % kM; t = e / kM; }   // coalesced along r
      else    { t = e % kKC; r = e / kKC; } // coalesced along t
      float x = 0.f;
      if (r < rows && k0 + t < K)
        x = f64_to_f32_rne(TA ? A[(int64_t)(k0 + t) * lda + r0 + r] : A[(int64_t)(r0 + r) * lda + k0 + t]);
      const uint32_t hi = to_tf32(x);
      const uint32_t lo = to_tf32(x - __uint_as_float(hi));
      const uint32_t off = kmajor_offset(r, t) >> 2;
      st.a_hi[off] = hi;
      st.a_lo[off] = lo;
    }
    // stage B: npad x 32
    for (int e = tid; e < npad * kKC; e += nthreads) {
      int n, t;
      if (TB) { n = e % npad; t = e / npad; }
      else    { t = e % kKC; n = e / kKC; }
      float x = 0.f;
      if (n < ncols && k0 + t < K)
        x = f64_to_f32_rne(TB ? B[(int64_t)(k0 + t) * ldb + n0 + n] : B[(int64_t)(n0 + n) * ldb + k0 + t]);
      const uint32_t hi = to_tf32(x);
      const uint32_t lo = to_tf32(x - __uint_as_float(hi));
      const uint32_t off = kmajor_offset(n, t) >> 2;
      st.b_hi[off] = hi;
      st.b_lo[off] = lo;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    fence_before();
    __syncthreads();
    fence_after();
    if (tid == 0 && debug_polls == 0) {
      const uint32_t d = c.tmem_base;
      const uint32_t ah = smem_addr(st.a_hi), al = smem_addr(st.a_lo);
      const uint32_t bh = smem_addr(st.b_hi), bl = smem_addr(st.b_lo);
#pragma unroll
      for (int ks = 0; ks < kKC / 8; ++ks) {
        const uint32_t koff = ks * 256;  // two 16-byte core columns per k-step of 8
        const uint64_t dah = smem_desc(ah + koff, lbo, sbo), dal = smem_desc(al + koff, lbo, sbo);
        const uint64_t dbh = smem_desc(bh + koff, lbo, sbo), dbl = smem_desc(bl + koff, lbo, sbo);
        const uint32_t acc0 = (first_in_span && ks == 0) ? 0u : 1u;
        mma_tf32(d, dah, dbh, idesc, acc0);
        mma_tf32(d, dah, dbl, idesc, 1u);
        mma_tf32(d, dal, dbh, idesc, 1u);
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_addr(&c.mbar))
          : "memory");
    }
    // one thread polls the barrier; the others park on the CTA barrier, so
    // the co-resident CTAs' FP64 work keeps the issue slots
    if (tid == 0 && !mbar_wait(c, debug_polls ? debug_polls : kWaitLimit)) *s_flag = 1;
    __syncthreads();
    if (tid == 0) c.phase ^= 1u;   // read again only after the next staging barrier
    if (*s_flag) return false;
    fence_after();
    first_in_span = false;
    const bool last = (ch == nchunks - 1);
    if (((ch + 1) % kPromote) == 0 || last) {
      // FP32 accumulator -> FP64 output: warp w reads TMEM lanes 32 (w % 4) ..,
      // columns split between warps w and w + 4
      const int q = warp & 3, half = warp >> 2, nw = blockDim.x >> 5;
      const int r = 32 * q + lane;
      const int cbeg = (nw >= 8) ? half * (npad / 2) : 0;
      const int cend = (nw >= 8) ? cbeg + npad / 2 : npad;
      for (int cb = cbeg; cb < cend; cb += 8) {
        uint32_t v[8];
        const uint32_t taddr = c.tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)cb;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
              "=r"(v[6]), "=r"(v[7])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (r < rows) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int n = cb + j;
            if (n < ncols) {
              double* po = Out + (int64_t)(n0 + n) * ldo + r0 + r;
              const double val = alpha * f32_to_f64(__uint_as_float(v[j]));
              *po = (accumulate || ch >= kPromote) ? *po + val : val;
            }
          }
        }
      }
      fence_before();
      __syncthreads();
      fence_after();
      first_in_span = true;
    } else {
      __syncthreads();
    }
  }
  return true;
}

// Whole product: Out^T (N x M, row n at Out + n * ldo) from 128 x 128 tiles.
template <bool TA, bool TB>
__device__ bool gemm(int M, int N, int K, const double* A, int64_t lda, const double* B, int64_t ldb,
                     double* Out, int64_t ldo, double alpha, bool accumulate, Stage& st, Ctrl& c,
                     int* s_flag, uint32_t debug_polls = 0) {
  for (int n0 = 0; n0 < N; n0 += kNmax)
    for (int r0 = 0; r0 < M; r0 += kM)
      if (!gemm_tile<TA, TB>(M, N, K, A, lda, B, ldb, Out, ldo, r0, n0, alpha, accumulate, st, c,
                             s_flag, debug_polls))
        return false;
  __syncthreads();
  return true;
}

}  // namespace tc
}  // namespace pf12
