// Fused persistent kernel of the complete pair F12 energy E_(2)F12 (Sec. "The
// PNO-based CCSD(T)F12bar Method"): for every pair, in one CTA,
//   1. FP64 Cholesky of J_g with the forward solve riding along and the FP64
//      backward solve, for the Coulomb densities of i and j with every PAO and
//      the occupied i, j, and of the Fock-transformed i_F, j_F (Eq. XAppr):
//        M = [J_g; A^g_i; A^g_j; A^g_iF; A^g_jF] -> [L; C_i; C_j; C_iF; C_jF]
//   2. robust fits (same coefficients, three operators):
//        V kernel over the extended basis Q_x = blockdiag(Q, I_2), projected
//          first: Vh = At^f_i Ct_j^T + Ct_i (At^f_j - Ct_j J_f)^T
//        geminal over the PAO domain: K_R = A^r_i C_j^T + C_i W1^T,
//          W1 = A^r_j - C_j J_r;  K_RiF = A^r_iF C_j^T + C_iF W1^T;
//          K_RjF = A^r_i C_jF^T + C_i W2^T, W2 = A^r_jF - C_jF J_r
//   3. the Q_ij projector (Eq. Qij): R_pno = Q^T K_R Q, R_Q = K_R - Q R_pno Q^T,
//      and Vh -= sum_cd R_pno[c, d] (c p|d q) from the PNO-pair factors B,
//      taken in chunks of kFullChunk auxiliary functions:
//        H[c][x][q] = sum_d R_pno[c, d] B[d][x][q],  Vh += -sum_c B[c]^T H[c]
//   4. the Fock coupling of Eq. C: Ft = F_v Q - Q (Q^T F_v Q),
//      C = Ft^T (K_R Q) + (K_R^T Q)^T Ft
//   5. B of Eq. B through S1 = R_Q F_v, S2 = F_v R_Q, and the X terms of
//      Eq. XAppr as inner products of K_RjF, K_RiF with R_Q and R_Q^T
//   6. the 14 spatial terms (fixed-order FP64 CTA sums) and the spin-adapted
//      pair energies (Eqs. F12energy_sf*).
// Cholesky, solves and every energy sum are FP64; the products follow TC.
// Each variant is instantiated in its own translation unit (csrc/inst/full_*.cu).
#pragma once
#include <cuda_runtime.h>

#include "pf12_device.cuh"
#include "pf12_internal.h"

namespace pf12 {

// rows x cols block from global memory (row stride sld) into the slab (row stride dld)
__device__ __forceinline__ void copy_block(const double* src, int64_t sld, int rows, int cols,
                                           double* dst, int64_t dld) {
  copy_region(src, sld, rows, cols, /*lower=*/false, /*packed=*/false, dst, dld);
}

// Q_x^T A for a (p + 2)-row block: the PNO rows through Q, rows p, p + 1 copied
template <typename TC>
__device__ __forceinline__ void project_ext(const double* Q, int p, int k, int m, const double* A,
                                            int64_t lda, double* out, int64_t ldo, GemmSmem& gs) {
  cta_gemm<TC, true, false>(k, m, p, Q, k, A, lda, out, ldo, 1.0, false, gs);
  copy_block(A + (int64_t)p * lda, lda, 2, m, out + (int64_t)k * ldo, ldo);
  __syncthreads();
}

template <typename TC>
__device__ void pair_full(const FullParams& prm, const FullDesc& pd, double* ws, GemmSmem& gs,
                          CholSmem& cs, double (*red)[kThreads / 32]) {
  const int tid = threadIdx.x;
  const int p = pd.p, k = pd.k, m = pd.m, k2 = k + 2;
  const int64_t ld = (m + 3) / 4 * 4, lq = (p + 3) / 4 * 4;
  const FullSlab sl = full_slab(p, k, m);
  double* M = ws + sl.M;
  const int64_t r_i = m, r_j = m + p + 2, r_iF = m + 2 * p + 4, r_jF = m + 3 * p + 4;
  const int nrhs = 4 * p + 4;
  const double* Jg = prm.Jg + pd.off_mm;
  const double* Jf = prm.Jf + pd.off_mm;
  const double* Jr = prm.Jr + pd.off_mm;
  const double* Q = prm.Q + pd.off_pk;
  const double* T = prm.T + pd.off_kk;
  const double* Fv = prm.Fv + pd.off_pp;
  const double* Sg = prm.S + pd.off_s;
  const double* B = prm.B + pd.off_b;
  const double* Agi = prm.Agi + pd.off_pm;
  const double* Agj = prm.Agj + pd.off_pm;
  const double* Afi = prm.Afi + pd.off_pm;
  const double* Afj = prm.Afj + pd.off_pm;
  const double* Ari = prm.Ari + pd.off_pm;
  const double* Arj = prm.Arj + pd.off_pm;
  const double* AgiF = prm.AgiF + pd.off_pm;
  const double* AgjF = prm.AgjF + pd.off_pm;
  const double* AriF = prm.AriF + pd.off_pm;
  const double* ArjF = prm.ArjF + pd.off_pm;

  // 1. J_g and the Coulomb factors into the slab; FP64 factorisation + solves
  load_metric(Jg, m, false, M, ld);   // lower triangle: all the factorisation reads
  copy_block(Agi, m, p + 2, m, M + r_i * ld, ld);
  copy_block(Agj, m, p + 2, m, M + r_j * ld, ld);
  copy_block(AgiF, m, p, m, M + r_iF * ld, ld);
  copy_block(AgjF, m, p, m, M + r_jF * ld, ld);
  __syncthreads();
  if (!chol_augmented(M, ld, m, m + nrhs, cs, gs)) {
    if (tid == 0) {
      const double nan = __longlong_as_double(0x7ff8000000000000ll);
      prm.status[pd.pair] = 1;
      for (int q = 0; q < 3; ++q) prm.e_pair[3 * (int64_t)pd.pair + q] = nan;
      for (int q = 0; q < kFullTerms; ++q) prm.terms[(int64_t)kFullTerms * pd.pair + q] = nan;
    }
    return;
  }
  solve_right_lower(M, ld, m, M + r_i * ld, ld, nrhs, cs, gs);
  const double* Ci = M + r_i * ld;
  const double* Cj = M + r_j * ld;
  const double* CiF = M + r_iF * ld;
  const double* CjF = M + r_jF * ld;

  // 2a. V kernel over the extended basis, projected before its products
  double* Atfi = ws + sl.Atfi;
  double* Atfj = ws + sl.Atfj;
  double* Cti = ws + sl.Cti;
  double* Ctj = ws + sl.Ctj;
  project_ext<TC>(Q, p, k, m, Afi, m, Atfi, ld, gs);
  project_ext<TC>(Q, p, k, m, Afj, m, Atfj, ld, gs);
  project_ext<TC>(Q, p, k, m, Ci, ld, Cti, ld, gs);
  project_ext<TC>(Q, p, k, m, Cj, ld, Ctj, ld, gs);
  cta_gemm<TC, false, false>(k2, m, m, Ctj, ld, Jf, m, Atfj, ld, -1.0, true, gs);
  double* Vh = ws + sl.Vh;
  cta_gemm<TC, false, true>(k2, k2, m, Atfi, ld, Ctj, ld, Vh, k2, 1.0, false, gs);
  cta_gemm<TC, false, true>(k2, k2, m, Cti, ld, Atfj, ld, Vh, k2, 1.0, true, gs);

  // 2b. geminal kernels over the PAO domain
  double* W1 = ws + sl.W1;
  double* W2 = ws + sl.W2;
  copy_block(Arj, m, p, m, W1, ld);
  copy_block(ArjF, m, p, m, W2, ld);
  __syncthreads();
  cta_gemm<TC, false, false>(p, m, m, Cj, ld, Jr, m, W1, ld, -1.0, true, gs);
  cta_gemm<TC, false, false>(p, m, m, CjF, ld, Jr, m, W2, ld, -1.0, true, gs);
  double* KR = ws + sl.KR;
  double* KRiF = ws + sl.KRiF;
  double* KRjF = ws + sl.KRjF;
  cta_gemm<TC, false, true>(p, p, m, Ari, m, Cj, ld, KR, lq, 1.0, false, gs);
  cta_gemm<TC, false, true>(p, p, m, Ci, ld, W1, ld, KR, lq, 1.0, true, gs);
  cta_gemm<TC, false, true>(p, p, m, AriF, m, Cj, ld, KRiF, lq, 1.0, false, gs);
  cta_gemm<TC, false, true>(p, p, m, CiF, ld, W1, ld, KRiF, lq, 1.0, true, gs);
  cta_gemm<TC, false, true>(p, p, m, Ari, m, CjF, ld, KRjF, lq, 1.0, false, gs);
  cta_gemm<TC, false, true>(p, p, m, Ci, ld, W2, ld, KRjF, lq, 1.0, true, gs);

  // 3-4. PNO projections, Fock coupling, projected geminal
  double* Y = ws + sl.Y;
  double* Zt = ws + sl.Zt;
  double* FvQ = ws + sl.FvQ;
  double* Ft = ws + sl.Ft;
  double* U = ws + sl.U;
  double* Rpno = ws + sl.Rpno;
  double* QtFQ = ws + sl.QtFQ;
  double* Cm = ws + sl.Cm;
  double* RQ = ws + sl.RQ;
  cta_gemm<TC, false, false>(p, k, p, KR, lq, Q, k, Y, k, 1.0, false, gs);     // K_R Q
  cta_gemm<TC, true, false>(p, k, p, KR, lq, Q, k, Zt, k, 1.0, false, gs);     // K_R^T Q
  cta_gemm<TC, false, false>(p, k, p, Fv, p, Q, k, FvQ, k, 1.0, false, gs);    // F_v Q
  cta_gemm<TC, true, false>(k, k, p, Q, k, Y, k, Rpno, k, 1.0, false, gs);     // Q^T K_R Q
  cta_gemm<TC, true, false>(k, k, p, Q, k, FvQ, k, QtFQ, k, 1.0, false, gs);   // Q^T F_v Q
  for (int64_t e = tid; e < (int64_t)p * k; e += kThreads) Ft[e] = FvQ[e];
  __syncthreads();
  cta_gemm<TC, false, false>(p, k, k, Q, k, QtFQ, k, Ft, k, -1.0, true, gs);   // (1 - QQ^T) F_v Q
  cta_gemm<TC, false, false>(p, k, k, Q, k, Rpno, k, U, k, 1.0, false, gs);    // Q R_pno
  cta_gemm<TC, true, false>(k, k, p, Ft, k, Y, k, Cm, k, 1.0, false, gs);      // Ft^T K_R Q
  cta_gemm<TC, true, false>(k, k, p, Zt, k, Ft, k, Cm, k, 1.0, true, gs);      // + Q^T K_R Ft
  for (int64_t e = tid; e < (int64_t)p * lq; e += kThreads) RQ[e] = KR[e];
  __syncthreads();
  cta_gemm<TC, false, true>(p, p, k, U, k, Q, k, RQ, lq, -1.0, true, gs);      // K_R - Q R_pno Q^T

  // 3. PNO-projector term of V, chunk by chunk over the auxiliary functions
  double* H = ws + sl.H;
  const int64_t ldb = (int64_t)m * k2;       // B[c] is an m x (k + 2) block
  for (int x0 = 0; x0 < m; x0 += kFullChunk) {
    const int w = min(kFullChunk, m - x0);
    const int64_t ldh = (int64_t)w * k2;
    cta_gemm<TC, false, false>(k, w * k2, k, Rpno, k, B + (int64_t)x0 * k2, ldb, H, ldh, 1.0,
                               false, gs);
    for (int c = 0; c < k; ++c)
      cta_gemm<TC, true, false>(k2, k2, w, B + c * ldb + (int64_t)x0 * k2, k2, H + c * ldh, k2,
                                Vh, k2, -1.0, true, gs);
  }

  // 5. Fock products of the projected geminal
  double* S1 = ws + sl.S1;
  double* S2 = ws + sl.S2;
  cta_gemm<TC, false, false>(p, p, p, RQ, lq, Fv, p, S1, lq, 1.0, false, gs);  // R_Q F_v
  cta_gemm<TC, false, false>(p, p, p, Fv, p, RQ, lq, S2, lq, 1.0, false, gs);  // F_v R_Q

  // 6. the spatial terms, fixed-order FP64 sums
  const double* si = Sg;
  const double* sj = Sg + k;
  double d = 0.0, x = 0.0, sd = 0.0, sx = 0.0, cd = 0.0, cx = 0.0;
  for (int e = tid; e < k * k; e += kThreads) {
    const int a = e / k, b = e - a * k;
    const double v = Vh[a * k2 + b];
    d = fma(v, T[e], d);
    x = fma(v, T[b * k + a], x);
    cd = fma(Cm[e], T[e], cd);
    cx = fma(Cm[e], T[b * k + a], cx);
  }
  for (int b = tid; b < k; b += kThreads) {
    // direct: Vh[i, s_j] + Vh[s_i, j];  exchange: Vh[j, s_i] + Vh[s_j, i]
    sd = fma(Vh[k * k2 + b], sj[b], sd);
    sd = fma(si[b], Vh[b * k2 + k + 1], sd);
    sx = fma(Vh[(k + 1) * k2 + b], si[b], sx);
    sx = fma(sj[b], Vh[b * k2 + k], sx);
  }
  double b1 = 0.0, b2 = 0.0, bx = 0.0, xjd = 0.0, xjx = 0.0, xid = 0.0, xix = 0.0;
  for (int64_t e = tid; e < (int64_t)p * p; e += kThreads) {
    const int a = (int)(e / p), b = (int)(e - (int64_t)a * p);
    const int64_t ab = (int64_t)a * lq + b, ba = (int64_t)b * lq + a;
    const double r = RQ[ab], rt = RQ[ba];
    b1 = fma(S1[ab], r, b1);
    b2 = fma(S2[ab], r, b2);
    bx = fma(S1[ab], rt, bx);
    xjd = fma(KRjF[ab], r, xjd);
    xjx = fma(KRjF[ab], rt, xjx);
    xid = fma(KRiF[ab], r, xid);
    xix = fma(KRiF[ab], rt, xix);
  }
  cta_sum2(d, x, red);
  cta_sum2(sd, sx, red);
  cta_sum2(cd, cx, red);
  cta_sum2(b1, b2, red);
  cta_sum2(bx, xjd, red);
  cta_sum2(xjx, xid, red);
  double zero = 0.0;
  cta_sum2(xix, zero, red);
  if (tid == 0) {
    double tm[kFullTerms];
    tm[0] = Vh[k * k2 + k + 1];     // Vh[i, j]
    tm[1] = Vh[(k + 1) * k2 + k];   // Vh[j, i]
    tm[2] = d;
    tm[3] = x;
    tm[4] = sd;
    tm[5] = sx;
    tm[6] = cd;
    tm[7] = cx;
    tm[8] = b1 + b2;
    tm[9] = 2.0 * bx;
    tm[10] = xjd;
    tm[11] = xjx;
    tm[12] = xid;
    tm[13] = xix;
    const int64_t P = pd.pair;
    bool fin = true;
    for (int q = 0; q < kFullTerms; ++q) {
      prm.terms[kFullTerms * P + q] = tm[q];
      fin = fin && isfinite(tm[q]);
    }
    const double vd = 0.5 * (tm[0] + tm[2] + tm[4]) + tm[6];
    const double vx = 0.5 * (tm[1] + tm[3] + tm[5]) + tm[7];
    const double bd = tm[8] - tm[10] - tm[12];
    const double bxx = tm[9] - tm[11] - tm[13];
    const double e_os = 0.75 * vd + 0.25 * vx + (10.0 * bd + 6.0 * bxx) / 64.0;
    const double e_ss = 0.5 * (vd - vx) + (bd - bxx) / 16.0;
    prm.e_pair[3 * P + 0] = pd.n_ab * e_os;
    prm.e_pair[3 * P + 1] = pd.n_aa * e_ss;
    prm.e_pair[3 * P + 2] = pd.n_bb * e_ss;
    prm.status[P] = fin ? 0 : 2;
  }
}

template <typename TC, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) pair_full_kernel(FullParams prm) {
  __shared__ GemmSmem gs;
  __shared__ CholSmem cs;
  __shared__ double red[2][kThreads / 32];
  __shared__ long long s_slot;
  double* ws = prm.work + (int64_t)blockIdx.x * prm.ws_stride;
  for (;;) {
    if (threadIdx.x == 0) s_slot = atomicAdd(prm.counter, 1);
    __syncthreads();
    const long long slot = s_slot;
    __syncthreads();
    if (slot >= prm.n_pairs) break;
    const FullDesc pd = prm.desc[slot];
    pair_full<TC>(prm, pd, ws, gs, cs, red);
    __syncthreads();
  }
}

}  // namespace pf12
