// Fused forward pair kernel: one persistent launch evaluates, for every pair,
// the projections onto the PNOs, the FP64 Cholesky of J_g with the forward
// solve riding along, the FP64 backward solve, the robust-fit V and the pair
// energies.  Pairs are taken from a cost-sorted queue through one atomic
// counter (no inter-CTA waits).
#include <cuda_runtime.h>

#include "pf12_device.cuh"
#include "pf12_internal.h"

namespace pf12 {

// One pair, steps 1-5 (order of evaluation: At = Q^T A first, so that every
// FP64 solve has k right-hand sides).
//   M = [J_g ; At^g_i ; At^g_j]   ((m + 2k) x ld)  ->  [L ; Ct_i ; Ct_j]
//   F = [At^f_i ; At^f_j]         (2k x ld)        ->  [At^f_i - Ct_i J_f ; At^f_j]
//   V = (At^f_i - Ct_i J_f) Ct_j^T + Ct_i At^f_j^T
template <typename TC>
__device__ void pair_forward(const FwdParams& prm, const PairDesc& pd, double* ws, GemmSmem& gs,
                             CholSmem& cs, double (*red)[kThreads / 32]) {
  const int tid = threadIdx.x;
  const int p = pd.p, k = pd.k, m = pd.m;
  const int64_t ld = (m + 3) / 4 * 4;
  double* M = ws;
  double* F = ws + (int64_t)(m + 2 * k) * ld;
  const double* Jg = prm.Jg + pd.off_mm;
  const double* Jf = prm.Jf + pd.off_mm;
  const double* Q = prm.Q + pd.off_pk;
  const double* T = prm.T + pd.off_kk;

  // J_g -> M (rows of m contiguous doubles)
  for (int r = tid >> 5; r < m; r += kThreads / 32)
    for (int c = tid & 31; c < m; c += 32) M[(int64_t)r * ld + c] = Jg[(int64_t)r * m + c];

  // S1': At^x = Q^T A^x  (k x m), A(a, mu) = Q[mu * k + a]
  const double* Asrc[4] = {prm.Agi + pd.off_pm, prm.Agj + pd.off_pm, prm.Afi + pd.off_pm,
                           prm.Afj + pd.off_pm};
  double* Adst[4] = {M + (int64_t)m * ld, M + (int64_t)(m + k) * ld, F, F + (int64_t)k * ld};
#pragma unroll 1
  for (int x = 0; x < 4; ++x)
    cta_gemm<TC, true, false>(k, m, p, Q, k, Asrc[x], m, Adst[x], ld, 1.0, false, gs);

  // S2: FP64 Cholesky of J_g with the forward solve of [At^g_i; At^g_j]
  const bool ok = chol_augmented(M, ld, m, m + 2 * k, cs, gs);
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
    return;
  }
  double* Ci = M + (int64_t)m * ld;
  double* Cj = M + (int64_t)(m + k) * ld;
  // S2: FP64 backward solve  Ct = Y L^{-1}
  solve_right_lower(M, ld, m, Ci, ld, 2 * k, cs, gs);

  // S3: F_i <- At^f_i - Ct_i J_f ;  V = F_i Ct_j^T + Ct_i At^f_j^T
  double* Fi = F;
  double* Fj = F + (int64_t)k * ld;
  cta_gemm<TC, false, false>(k, m, m, Ci, ld, Jf, m, Fi, ld, -1.0, true, gs);
  double* V = prm.V + pd.off_kk;
  for (int r0 = 0; r0 < k; r0 += kTile)
    for (int c0 = 0; c0 < k; c0 += kTile) {
      cta_gemm_tile<TC, false, true>(k, k, m, Fi, ld, Cj, ld, V, k, r0, c0, 1.0, false, gs);
      cta_gemm_tile<TC, false, true>(k, k, m, Ci, ld, Fj, ld, V, k, r0, c0, 1.0, true, gs);
    }
  __syncthreads();

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
}

template <typename TC>
__global__ void __launch_bounds__(kThreads, 2) pair_forward_kernel(FwdParams prm) {
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
    const PairDesc pd = prm.desc[slot];
    pair_forward<TC>(prm, pd, ws, gs, cs, red);
    __syncthreads();
  }
}

cudaError_t launch_forward(const FwdParams& prm, int precision, int n_ctas, cudaStream_t s) {
  if (precision == 0)
    pair_forward_kernel<double><<<n_ctas, kThreads, 0, s>>>(prm);
  else
    pair_forward_kernel<float><<<n_ctas, kThreads, 0, s>>>(prm);
  return cudaGetLastError();
}

int forward_blocks_per_sm(int precision) {
  int n = 0;
  if (precision == 0)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pair_forward_kernel<double>, kThreads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pair_forward_kernel<float>, kThreads, 0);
  return n;
}

// Deterministic total: thread t sums a contiguous range of pairs in order,
// then a fixed shared-memory tree.  out3 = (E, number of non-OK pairs, first
// non-OK pair or -1).
__global__ void __launch_bounds__(1024) energy_total_kernel(const double* e_pair,
                                                            const int32_t* status, int64_t n,
                                                            double* out3) {
  __shared__ double s_sum[1024];
  __shared__ long long s_bad[1024];
  __shared__ long long s_first[1024];
  const int t = threadIdx.x;
  const int64_t chunk = (n + 1023) / 1024;
  const int64_t beg = t * chunk, end = min(n, beg + chunk);
  double acc = 0.0;
  long long bad = 0, first = -1;
  for (int64_t P = beg; P < end; ++P) {
    acc += e_pair[3 * P] + e_pair[3 * P + 1] + e_pair[3 * P + 2];
    if (status[P] != 0) {
      if (first < 0) first = P;
      ++bad;
    }
  }
  s_sum[t] = acc;
  s_bad[t] = bad;
  s_first[t] = first;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if (t < w) {
      s_sum[t] += s_sum[t + w];
      s_bad[t] += s_bad[t + w];
      const long long f = s_first[t + w];
      if (f >= 0 && (s_first[t] < 0 || f < s_first[t])) s_first[t] = f;
    }
    __syncthreads();
  }
  if (t == 0) {
    out3[0] = s_sum[0];
    out3[1] = (double)s_bad[0];
    out3[2] = (double)s_first[0];
  }
}

cudaError_t launch_energy_total(const double* e_pair, const int32_t* status, int64_t n_pairs,
                                double* out3, cudaStream_t s) {
  energy_total_kernel<<<1, 1024, 0, s>>>(e_pair, status, n_pairs, out3);
  return cudaGetLastError();
}

}  // namespace pf12
