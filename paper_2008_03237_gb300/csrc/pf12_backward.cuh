// Hand-written adjoint of the pair-F12 energy (one persistent fused launch),
// device templates; each variant is instantiated in csrc/inst/bwd_*.cu.
// Each pair's forward intermediates are recomputed, not stored; the two extra
// FP64 solves give Z^T = (At^f - Ct J_f) J_g^{-1}.  With G_V = dE (alpha T +
// beta T^T) (E_P = alpha d + beta x):
//   dT    = dE (alpha V + beta V^T)
//   H1 = G_V Ct_j,  H2 = G_V^T Ct_i,  H3 = G_V Z_j^T,  H4 = G_V^T Z_i^T   (k x m)
//   dAf_i = Q H1, dAf_j = Q H2, dAg_i = Q H3, dAg_j = Q H4                (p x m)
//   dQ    = Af_i H1^T + Af_j H2^T + Ag_i H3^T + Ag_j H4^T                 (p x k)
// which is the chain rule of V = Q^T K Q, K = A^f_i C_j^T + C_i A^f_j^T -
// C_i J_f C_j^T, C = A^g J_g^{-1} with J_g, J_f symmetric and held constant.
// SOMO-augmented pairs (Sec. "SOMO handling") use Q_aug = blockdiag(Q, I): the
// SOMO rows of dA are the SOMO rows of H, dQ takes the PNO rows of H only, and
// alpha, beta become per-block weights (alpha virtuals exclude the SOMOs).
#pragma once
#include <cuda_runtime.h>

#include "pf12_device.cuh"
#include "pf12_internal.h"

namespace pf12 {

template <typename TC>
__device__ bool pair_backward(const BwdParams& b, const PairDesc& pd, double* ws, GemmSmem& gs,
                              CholSmem& cs, SieveCtl& sc, uint32_t& phase) {
  const FwdParams& prm = b.f;
  const int tid = threadIdx.x;
  const int p = pd.p, k = pd.k, m = pd.m;
  const int64_t ld = (m + 3) / 4 * 4;
  const int64_t ldk = (k + 3) / 4 * 4;
  double* M = ws;                                // m + 2k rows
  double* F = M + (int64_t)(m + 2 * k) * ld;     // 2k rows
  double* R = F + 2 * (int64_t)k * ld;           // 2k rows
  double* GV = R + 2 * (int64_t)k * ld;          // k x ldk
  double* Vl = GV + (int64_t)k * ldk;            // k x ldk
  const double* Jg = prm.Jg + pd.off_mm;
  const double* Jf = prm.Jf + pd.off_mm;
  const double* Q = prm.Q + pd.off_pk;
  const double* T = prm.T + pd.off_kk;
  const double* Agi = prm.Agi + pd.off_pm;
  const double* Agj = prm.Agj + pd.off_pm;
  const double* Afi = prm.Afi + pd.off_pm;
  const double* Afj = prm.Afj + pd.off_pm;
  if (prm.gdesc) {   // gather mode: the pair's factor blocks sieved into the slab
    double* G = ws + bwd_sieve_off(k, m);
    if (!sieve_pair(prm, pd, G, gs, sc, phase)) return false;
    Agi = G;
    Agj = G + (int64_t)p * m;
    Afi = G + 2 * (int64_t)p * m;
    Afj = G + 3 * (int64_t)p * m;
  }

  load_metric(Jg, m, prm.metric_packed, M, ld);
  const double* Jf_use = Jf;
  int64_t ld_jf = m;
  if (prm.metric_packed) {   // full J_f for its product, unpacked into the slab
    double* W = ws + bwd_jf_off(p, k, m, prm.gdesc != nullptr);
    unpack_metric(Jf, m, W, ld);
    Jf_use = W;
    ld_jf = ld;
  }
  // SOMO-augmented pair: Q_aug = blockdiag(Q, I), Q is p x kq
  const int s = pd.s, kq = k - s;
  cta_gemm<TC, true, false>(kq, m, p, Q, kq, Agi, m, M + (int64_t)m * ld, ld, 1.0, false, gs);
  cta_gemm<TC, true, false>(kq, m, p, Q, kq, Agj, m, M + (int64_t)(m + k) * ld, ld, 1.0, false, gs);
  cta_gemm<TC, true, false>(kq, m, p, Q, kq, Afi, m, F, ld, 1.0, false, gs);
  cta_gemm<TC, true, false>(kq, m, p, Q, kq, Afj, m, F + (int64_t)k * ld, ld, 1.0, false, gs);
  if (s) {
    copy_somo_rows(Agi, p, s, m, M + (int64_t)m * ld, ld, kq);
    copy_somo_rows(Agj, p, s, m, M + (int64_t)(m + k) * ld, ld, kq);
    copy_somo_rows(Afi, p, s, m, F, ld, kq);
    copy_somo_rows(Afj, p, s, m, F + (int64_t)k * ld, ld, kq);
    __syncthreads();
  }

  if (!chol_augmented(M, ld, m, m + 2 * k, cs, gs)) {
    // no gradient exists for this pair: its blocks are written as zeros, so
    // values of an earlier call never survive in the caller's buffers
    const int64_t rows = (int64_t)(p + s) * m;
    double* outs[4] = {b.dAgi, b.dAgj, b.dAfi, b.dAfj};
    for (double* o : outs)
      if (o)
        for (int64_t e = tid; e < rows; e += kThreads) o[pd.off_pm + e] = 0.0;
    if (b.dQ)
      for (int64_t e = tid; e < (int64_t)p * kq; e += kThreads) b.dQ[pd.off_pk + e] = 0.0;
    if (b.dT)
      for (int64_t e = tid; e < (int64_t)k * k; e += kThreads) b.dT[pd.off_kk + e] = 0.0;
    if (tid == 0) prm.status[pd.pair] = 1;
    return true;
  }
  double* Ci = M + (int64_t)m * ld;
  double* Cj = M + (int64_t)(m + k) * ld;
  solve_right_lower(M, ld, m, Ci, ld, 2 * k, cs, gs);

  // R = At^f - Ct J_f  (both x at once: Ct_i, Ct_j are consecutive rows)
  for (int64_t e = tid; e < 2 * (int64_t)k * ld; e += kThreads) R[e] = F[e];
  __syncthreads();
  cta_gemm<TC, false, false>(2 * k, m, m, Ci, ld, Jf_use, ld_jf, R, ld, -1.0, true, gs);

  // V = R_i Ct_j^T + Ct_i At^f_j^T
  for (int r0 = 0; r0 < k; r0 += kTile)
    for (int c0 = 0; c0 < k; c0 += kTile) {
      cta_gemm_tile<TC, false, true>(k, k, m, R, ld, Cj, ld, Vl, ldk, r0, c0, 1.0, false, gs);
      cta_gemm_tile<TC, false, true>(k, k, m, Ci, ld, F + (int64_t)k * ld, ld, Vl, ldk, r0, c0, 1.0,
                                     true, gs);
    }
  __syncthreads();

  const double alpha = 3.0 * pd.n_ab / 8.0 + (pd.n_aa + pd.n_bb) / 4.0;
  const double beta = pd.n_ab / 8.0 - (pd.n_aa + pd.n_bb) / 4.0;
  double* dT = b.dT ? b.dT + pd.off_kk : nullptr;
  if (s == 0) {
    for (int e = tid; e < k * k; e += kThreads) {
      const int a = e / k, c = e - a * k;
      GV[a * ldk + c] = b.dE * (alpha * T[a * k + c] + beta * T[c * k + a]);
      if (dT) dT[e] = b.dE * (alpha * Vl[a * ldk + c] + beta * Vl[c * ldk + a]);
    }
  } else {   // augmented: weights by virtual block (PNO / SOMO of a and of c)
    for (int e = tid; e < k * k; e += kThreads) {
      const int a = e / k, c = e - a * k;
      double wd, wx, wd_t, wx_t;
      somo_block_weights(pd, 2 * (a >= kq) + (c >= kq), wd, wx);
      somo_block_weights(pd, 2 * (c >= kq) + (a >= kq), wd_t, wx_t);
      GV[a * ldk + c] = b.dE * (wd * T[a * k + c] + wx * T[c * k + a]);
      if (dT) dT[e] = b.dE * (wd * Vl[a * ldk + c] + wx_t * Vl[c * ldk + a]);
    }
  }
  __syncthreads();

  // Z^T = R J_g^{-1}: forward then backward FP64 solve on the 2k rows of R
  solve_right_lowerT(M, ld, m, R, ld, 2 * k, cs, gs);
  solve_right_lower(M, ld, m, R, ld, 2 * k, cs, gs);
  double* Zi = R;
  double* Zj = R + (int64_t)k * ld;

  double* H1 = F;
  double* H2 = F + (int64_t)k * ld;
  double* dQ = b.dQ ? b.dQ + pd.off_pk : nullptr;
  // H1 = G_V Ct_j, H2 = G_V^T Ct_i
  cta_gemm<TC, false, false>(k, m, k, GV, ldk, Cj, ld, H1, ld, 1.0, false, gs);
  cta_gemm<TC, true, false>(k, m, k, GV, ldk, Ci, ld, H2, ld, 1.0, false, gs);
  if (b.dAfi) cta_gemm<TC, false, false>(p, m, kq, Q, kq, H1, ld, b.dAfi + pd.off_pm, m, 1.0, false, gs);
  if (b.dAfj) cta_gemm<TC, false, false>(p, m, kq, Q, kq, H2, ld, b.dAfj + pd.off_pm, m, 1.0, false, gs);
  if (s) {
    if (b.dAfi) copy_somo_grad_rows(H1, ld, kq, s, m, b.dAfi + pd.off_pm, p);
    if (b.dAfj) copy_somo_grad_rows(H2, ld, kq, s, m, b.dAfj + pd.off_pm, p);
  }
  if (dQ) {
    cta_gemm<TC, false, true>(p, kq, m, Afi, m, H1, ld, dQ, kq, 1.0, false, gs);
    cta_gemm<TC, false, true>(p, kq, m, Afj, m, H2, ld, dQ, kq, 1.0, true, gs);
  }
  if (s) __syncthreads();   // H1, H2 are overwritten next
  // H3 = G_V Z_j^T, H4 = G_V^T Z_i^T
  cta_gemm<TC, false, false>(k, m, k, GV, ldk, Zj, ld, H1, ld, 1.0, false, gs);
  cta_gemm<TC, true, false>(k, m, k, GV, ldk, Zi, ld, H2, ld, 1.0, false, gs);
  if (b.dAgi) cta_gemm<TC, false, false>(p, m, kq, Q, kq, H1, ld, b.dAgi + pd.off_pm, m, 1.0, false, gs);
  if (b.dAgj) cta_gemm<TC, false, false>(p, m, kq, Q, kq, H2, ld, b.dAgj + pd.off_pm, m, 1.0, false, gs);
  if (s) {
    if (b.dAgi) copy_somo_grad_rows(H1, ld, kq, s, m, b.dAgi + pd.off_pm, p);
    if (b.dAgj) copy_somo_grad_rows(H2, ld, kq, s, m, b.dAgj + pd.off_pm, p);
  }
  if (dQ) {
    cta_gemm<TC, false, true>(p, kq, m, Agi, m, H1, ld, dQ, kq, 1.0, true, gs);
    cta_gemm<TC, false, true>(p, kq, m, Agj, m, H2, ld, dQ, kq, 1.0, true, gs);
  }
  if (s) __syncthreads();
  if (tid == 0) prm.status[pd.pair] = 0;
  return true;
}

template <typename TC, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) pair_backward_kernel(BwdParams b) {
  __shared__ GemmSmem gs;
  __shared__ CholSmem cs;
  __shared__ long long s_slot;
  __shared__ SieveCtl sc;
  uint32_t phase = 0;
  if (b.f.gdesc) sieve_init(sc);
  double* ws = b.f.work + (int64_t)blockIdx.x * b.f.ws_stride;
  for (;;) {
    if (threadIdx.x == 0)
      s_slot = (b.f.err && *b.f.err != 0) ? b.f.n_pairs : atomicAdd(b.f.counter + 1, 1);
    __syncthreads();
    const long long slot = s_slot;
    __syncthreads();
    if (slot >= b.f.n_pairs) break;
    const PairDesc pd = b.f.desc[slot];
    if (!pair_backward<TC>(b, pd, ws, gs, cs, sc, phase)) {
      if (threadIdx.x == 0) {
        b.f.status[pd.pair] = 3;
        atomicExch(b.f.err, 1);
      }
      break;
    }
    __syncthreads();
  }
}

}  // namespace pf12
