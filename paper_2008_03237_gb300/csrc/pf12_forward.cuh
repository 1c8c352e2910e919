// Device code of the fused forward pair kernels (templates).  Each kernel
// variant is instantiated in its own translation unit (csrc/inst/fwd_*.cu), so
// that the variants compile in parallel; pf12_forward.cu dispatches to them.
#pragma once
#include <cuda_runtime.h>

#include "pf12_device.cuh"
#include "pf12_internal.h"
#if defined(PF12_FORWARD_TC)
#include "pf12_tc.cuh"
#endif

namespace pf12 {


// One pair, steps 1-5 (order of evaluation: At = Q^T A first, so that every
// FP64 solve has k right-hand sides).
//   M = [J_g ; At^g_i ; At^g_j]   ((m + 2k) x ld)  ->  [L ; Ct_i ; Ct_j]
//   F = [At^f_i ; At^f_j]         (2k x ld)        ->  [At^f_i - Ct_i J_f ; At^f_j]
//   V = (At^f_i - Ct_i J_f) Ct_j^T + Ct_i At^f_j^T
__device__ __forceinline__ void write_pair_energy(const FwdParams& prm, int64_t P, const double e[3],
                                                  double D, double X) {
  prm.e_pair[3 * P + 0] = e[0];
  prm.e_pair[3 * P + 1] = e[1];
  prm.e_pair[3 * P + 2] = e[2];
  prm.dx[2 * P] = D;
  prm.dx[2 * P + 1] = X;
  prm.status[P] = (isfinite(D) && isfinite(X)) ? 0 : 2;
}

template <typename TC, int LOOK = kLook>
__device__ bool pair_forward(const FwdParams& prm, const PairDesc& pd, double* ws, GemmSmem& gs,
                             CholSmem& cs, double (*red)[kThreads / 32], SieveCtl& sc,
                             uint32_t& phase) {
  const int tid = threadIdx.x;
  const int p = pd.p, k = pd.k, m = pd.m;
  const int64_t ld = (m + 3) / 4 * 4;
  double* M = ws;
  double* F = ws + (int64_t)(m + 2 * k) * ld;
  const double* Jg = prm.Jg + pd.off_mm;
  const double* Jf = prm.Jf + pd.off_mm;
  const double* Q = prm.Q + pd.off_pk;
  const double* T = prm.T + pd.off_kk;

  // J_g -> M; a packed J_f is unpacked into the slab for its product
  load_metric(Jg, m, prm.metric_packed, M, ld);
  const double* Jf_use = Jf;
  int64_t ld_jf = m;
  if (prm.metric_packed) {
    double* W = ws + fwd_jf_off(p, k, m, prm.gdesc != nullptr);
    unpack_metric(Jf, m, W, ld);
    Jf_use = W;
    ld_jf = ld;
  }

  // S1: packed factors, or (gather mode) the pair's blocks sieved out of the
  // per-orbital pair-extended blocks into the slab
  const double* Asrc[4] = {prm.Agi + pd.off_pm, prm.Agj + pd.off_pm, prm.Afi + pd.off_pm,
                           prm.Afj + pd.off_pm};
  if (prm.gdesc) {
    double* G = ws + fwd_sieve_off(k, m);
    if (!sieve_pair(prm, pd, G, gs, sc, phase)) return false;
    for (int x = 0; x < 4; ++x) Asrc[x] = G + (int64_t)x * p * m;
  }
  // S1': At^x = Q^T A^x  (k x m), A(a, mu) = Q[mu * k + a]
  // SOMO-augmented pair: the first kq rows through Q, the SOMO rows copied
  const int kq = k - pd.s;
  double* Adst[4] = {M + (int64_t)m * ld, M + (int64_t)(m + k) * ld, F, F + (int64_t)k * ld};
#pragma unroll 1
  for (int x = 0; x < 4; ++x) {
    cta_gemm<TC, true, false>(kq, m, p, Q, kq, Asrc[x], m, Adst[x], ld, 1.0, false, gs);
    if (pd.s) copy_somo_rows(Asrc[x], p, pd.s, m, Adst[x], ld, kq);
  }
  if (pd.s) __syncthreads();

  // S2: FP64 Cholesky of J_g with the forward solve of [At^g_i; At^g_j]
  const bool ok = chol_augmented<LOOK>(M, ld, m, m + 2 * k, cs, gs);
  if (!ok) {
    if (tid == 0) {
      const double nan = __longlong_as_double(0x7ff8000000000000ll);
      prm.status[pd.pair] = 1;
      prm.e_pair[3 * (int64_t)pd.pair + 0] = nan;
      prm.e_pair[3 * (int64_t)pd.pair + 1] = nan;
      prm.e_pair[3 * (int64_t)pd.pair + 2] = nan;
      prm.dx[2 * (int64_t)pd.pair] = nan;
      prm.dx[2 * (int64_t)pd.pair + 1] = nan;
    }
    return true;
  }
  double* Ci = M + (int64_t)m * ld;
  double* Cj = M + (int64_t)(m + k) * ld;
  // S2: FP64 backward solve  Ct = Y L^{-1}
  solve_right_lower(M, ld, m, Ci, ld, 2 * k, cs, gs);

  // S3: F_i <- At^f_i - Ct_i J_f ;  V = F_i Ct_j^T + Ct_i At^f_j^T
  double* Fi = F;
  double* Fj = F + (int64_t)k * ld;
  cta_gemm<TC, false, false>(k, m, m, Ci, ld, Jf_use, ld_jf, Fi, ld, -1.0, true, gs);
  double* V = prm.V + pd.off_kk;
  for (int r0 = 0; r0 < k; r0 += kTile)
    for (int c0 = 0; c0 < k; c0 += kTile) {
      cta_gemm_tile<TC, false, true>(k, k, m, Fi, ld, Cj, ld, V, k, r0, c0, 1.0, false, gs);
      cta_gemm_tile<TC, false, true>(k, k, m, Ci, ld, Fj, ld, V, k, r0, c0, 1.0, true, gs);
    }
  __syncthreads();
  if (pd.s) {   // augmented pair: spin cases restricted to their own virtuals
    double e[3], D, X;
    somo_pair_energy(pd, V, T, red, e, D, X);
    if (tid == 0) write_pair_energy(prm, pd.pair, e, D, X);
    return true;
  }

  // S4: d = <V, T>, x = <V, T^T>   (FP64, fixed order)
  double sd = 0.0, sx = 0.0;
  for (int e = tid; e < k * k; e += kThreads) {
    const int a = e / k, b = e - a * k;
    const double v = V[e];
    sd = fma(v, T[e], sd);
    sx = fma(v, T[b * k + a], sx);
  }
  cta_sum2(sd, sx, red);
  // S5: spin cases
  if (tid == 0) {
    const double e_ab = pd.n_ab * (3.0 * sd + sx) / 8.0;
    const double e_aa = pd.n_aa * (sd - sx) / 4.0;
    const double e_bb = pd.n_bb * (sd - sx) / 4.0;
    const int64_t P = pd.pair;
    prm.e_pair[3 * P + 0] = e_ab;
    prm.e_pair[3 * P + 1] = e_aa;
    prm.e_pair[3 * P + 2] = e_bb;
    prm.dx[2 * P] = sd;
    prm.dx[2 * P + 1] = sx;
    prm.status[P] = (isfinite(sd) && isfinite(sx)) ? 0 : 2;
  }
  return true;
}

template <typename TC, int MINB, int LOOK = kLook>
__global__ void __launch_bounds__(kThreads, MINB) pair_forward_kernel(FwdParams prm) {
  __shared__ GemmSmem gs;
  __shared__ CholSmem cs;
  __shared__ double red[2][kThreads / 32];
  __shared__ long long s_slot;
  __shared__ SieveCtl sc;
  uint32_t phase = 0;
  if (prm.gdesc) sieve_init(sc);
  double* ws = prm.work + (int64_t)blockIdx.x * prm.ws_stride;
  int known_group = -1;
  for (;;) {
    if (threadIdx.x == 0) s_slot = next_slot(prm, known_group);
    __syncthreads();
    const long long slot = s_slot;
    __syncthreads();
    if (slot < 0 || slot >= prm.n_pairs) break;
    const PairDesc pd = prm.desc[slot];
    if (!pair_forward<TC, LOOK>(prm, pd, ws, gs, cs, red, sc, phase)) {
      if (threadIdx.x == 0) {
        prm.status[pd.pair] = 3;
        atomicExch(prm.err, 1);
      }
      break;
    }
    __syncthreads();
  }
}

#if defined(PF12_FORWARD_TC)   // only the tensor-core variant's translation unit
// Mixed-precision pair with the dense contractions on the tensor cores:
// projections At^x = Q^T A^x and W = Ct_i J_f as tcgen05 split-TF32 GEMMs
// (transposed tiles: m on the 128-row MMA axis, k on N), everything FP64
// (Cholesky, solves, energy) unchanged.  Returns false after a bounded wait
// expired (the pair gets status 3 and the kernel stops taking pairs).
static __device__ bool pair_forward_tc(const FwdParams& prm, const PairDesc& pd, double* ws, GemmSmem& gs,
                                CholSmem& cs, double (*red)[kThreads / 32], tc::Stage& st,
                                tc::Ctrl& ctrl, int* s_flag, SieveCtl& sc, uint32_t& phase) {
  const int tid = threadIdx.x;
  const int p = pd.p, k = pd.k, m = pd.m;
  const int64_t ld = (m + 3) / 4 * 4;
  double* M = ws;
  double* F = ws + (int64_t)(m + 2 * k) * ld;
  const double* Jg = prm.Jg + pd.off_mm;
  const double* Jf = prm.Jf + pd.off_mm;
  const double* Q = prm.Q + pd.off_pk;
  const double* T = prm.T + pd.off_kk;
  load_metric(Jg, m, prm.metric_packed, M, ld);
  const double* Jf_use = Jf;
  int64_t ld_jf = m;
  if (prm.metric_packed) {
    double* W = ws + fwd_jf_off(p, k, m, prm.gdesc != nullptr);
    unpack_metric(Jf, m, W, ld);
    Jf_use = W;
    ld_jf = ld;
  }
  const double* Asrc[4] = {prm.Agi + pd.off_pm, prm.Agj + pd.off_pm, prm.Afi + pd.off_pm,
                           prm.Afj + pd.off_pm};
  if (prm.gdesc) {
    double* G = ws + fwd_sieve_off(k, m);
    if (!sieve_pair(prm, pd, G, gs, sc, phase)) return false;
    for (int x = 0; x < 4; ++x) Asrc[x] = G + (int64_t)x * p * m;
  }
  const int kq = k - pd.s;
  double* Adst[4] = {M + (int64_t)m * ld, M + (int64_t)(m + k) * ld, F, F + (int64_t)k * ld};
#pragma unroll 1
  for (int x = 0; x < 4; ++x) {
    if (!tc::gemm<true, true>(m, kq, p, Asrc[x], m, Q, kq, Adst[x], ld, 1.0, false, st, ctrl, s_flag,
                              prm.debug_wait_polls))
      return false;
    if (pd.s) copy_somo_rows(Asrc[x], p, pd.s, m, Adst[x], ld, kq);
  }
  __syncthreads();
  const bool ok = chol_augmented(M, ld, m, m + 2 * k, cs, gs);
  if (!ok) {
    if (tid == 0) {
      const double nan = __longlong_as_double(0x7ff8000000000000ll);
      prm.status[pd.pair] = 1;
      for (int q = 0; q < 3; ++q) prm.e_pair[3 * (int64_t)pd.pair + q] = nan;
      prm.dx[2 * (int64_t)pd.pair] = nan;
      prm.dx[2 * (int64_t)pd.pair + 1] = nan;
    }
    __syncthreads();
    return true;
  }
  double* Ci = M + (int64_t)m * ld;
  double* Cj = M + (int64_t)(m + k) * ld;
  solve_right_lower(M, ld, m, Ci, ld, 2 * k, cs, gs);
  double* Fi = F;
  double* Fj = F + (int64_t)k * ld;
  // F_i <- At^f_i - Ct_i J_f, computed as (J_f Ct_i^T)^T with J_f symmetric
  if (!tc::gemm<false, false>(m, k, m, Jf_use, ld_jf, Ci, ld, Fi, ld, -1.0, true, st, ctrl, s_flag))
    return false;
  double* V = prm.V + pd.off_kk;
  for (int r0 = 0; r0 < k; r0 += kTile)
    for (int c0 = 0; c0 < k; c0 += kTile) {
      cta_gemm_tile<float, false, true>(k, k, m, Fi, ld, Cj, ld, V, k, r0, c0, 1.0, false, gs);
      cta_gemm_tile<float, false, true>(k, k, m, Ci, ld, Fj, ld, V, k, r0, c0, 1.0, true, gs);
    }
  __syncthreads();
  if (pd.s) {
    double e[3], D, X;
    somo_pair_energy(pd, V, T, red, e, D, X);
    if (tid == 0) write_pair_energy(prm, pd.pair, e, D, X);
    return true;
  }
  double sd = 0.0, sx = 0.0;
  for (int e = tid; e < k * k; e += kThreads) {
    const int a = e / k, b = e - a * k;
    const double v = V[e];
    sd = fma(v, T[e], sd);
    sx = fma(v, T[b * k + a], sx);
  }
  cta_sum2(sd, sx, red);
  if (tid == 0) {
    const int64_t P = pd.pair;
    prm.e_pair[3 * P + 0] = pd.n_ab * (3.0 * sd + sx) / 8.0;
    prm.e_pair[3 * P + 1] = pd.n_aa * (sd - sx) / 4.0;
    prm.e_pair[3 * P + 2] = pd.n_bb * (sd - sx) / 4.0;
    prm.dx[2 * P] = sd;
    prm.dx[2 * P + 1] = sx;
    prm.status[P] = (isfinite(sd) && isfinite(sx)) ? 0 : 2;
  }
  return true;
}

// shared memory of the tensor-core variant: the staging tiles share space with
// the SIMT GEMM and Cholesky buffers (never live at the same time)
constexpr size_t kTcUnion = sizeof(tc::Stage) > sizeof(GemmSmem) + sizeof(CholSmem)
                                ? sizeof(tc::Stage)
                                : sizeof(GemmSmem) + sizeof(CholSmem);
constexpr size_t kTcSmem = kTcUnion + sizeof(tc::Ctrl) + 2 * (kThreads / 32) * sizeof(double) + 64;

template <int MINB>
__global__ void __launch_bounds__(kThreads, MINB) pair_forward_tc_kernel(FwdParams prm) {
  extern __shared__ __align__(1024) unsigned char smem[];
  tc::Stage& st = *reinterpret_cast<tc::Stage*>(smem);
  GemmSmem& gs = *reinterpret_cast<GemmSmem*>(smem);
  CholSmem& cs = *reinterpret_cast<CholSmem*>(smem + sizeof(GemmSmem));
  unsigned char* tail = smem + kTcUnion;
  tc::Ctrl& ctrl = *reinterpret_cast<tc::Ctrl*>(tail);
  double (*red)[kThreads / 32] = reinterpret_cast<double (*)[kThreads / 32]>(tail + sizeof(tc::Ctrl));
  long long* s_slot = reinterpret_cast<long long*>(tail + sizeof(tc::Ctrl) + 2 * (kThreads / 32) * sizeof(double));
  int* s_flag = reinterpret_cast<int*>(s_slot + 1);
  __shared__ SieveCtl sc;
  uint32_t phase = 0;
  if (prm.gdesc) sieve_init(sc);
  if (threadIdx.x == 0) *s_flag = 0;
  tc::setup(ctrl);
  double* ws = prm.work + (int64_t)blockIdx.x * prm.ws_stride;
  int known_group = -1;
  for (;;) {
    if (threadIdx.x == 0) *s_slot = next_slot(prm, known_group);
    __syncthreads();
    const long long slot = *s_slot;
    __syncthreads();
    if (slot < 0 || slot >= prm.n_pairs) break;
    const PairDesc pd = prm.desc[slot];
    if (!pair_forward_tc(prm, pd, ws, gs, cs, red, st, ctrl, s_flag, sc, phase)) {
      if (threadIdx.x == 0) {
        prm.status[pd.pair] = 3;
        atomicExch(prm.err, 1);
      }
      break;
    }
    __syncthreads();
  }
  tc::teardown(ctrl);
}
#endif  // PF12_FORWARD_TC

}  // namespace pf12
