// Fused forward pair kernel: one persistent launch evaluates, for every pair,
// the projections onto the PNOs, the FP64 Cholesky of J_g with the forward
// solve riding along, the FP64 backward solve, the robust-fit V and the pair
// energies.  Pairs are taken from a cost-sorted queue through one atomic
// counter (no inter-CTA waits).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "../../include/pairf12.h"
#include "pf12_device.cuh"
#include "pf12_internal.h"
#include "pf12_tc.cuh"

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

template <typename TC>
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

template <typename TC, int MINB>
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
    if (!pair_forward<TC>(prm, pd, ws, gs, cs, red, sc, phase)) {
      if (threadIdx.x == 0) {
        prm.status[pd.pair] = 3;
        atomicExch(prm.err, 1);
      }
      break;
    }
    __syncthreads();
  }
}

// Mixed-precision pair with the dense contractions on the tensor cores:
// projections At^x = Q^T A^x and W = Ct_i J_f as tcgen05 split-TF32 GEMMs
// (transposed tiles: m on the 128-row MMA axis, k on N), everything FP64
// (Cholesky, solves, energy) unchanged.  Returns false after a bounded wait
// expired (the pair gets status 3 and the kernel stops taking pairs).
__device__ bool pair_forward_tc(const FwdParams& prm, const PairDesc& pd, double* ws, GemmSmem& gs,
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

// Tile/occupancy variants the autotuner chooses from: variant 0 / 1 run the
// SIMT kernel at MINB = 2 / 3 CTAs per SM (more resident pairs per SM hide the
// serial phases of each pair's factorisation; fewer leave more registers per
// thread); variant 2 (mixed precision only) is the tensor-core kernel at 3.
static cudaError_t tc_attr() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(pair_forward_tc_kernel<3>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
  // prefer the largest shared-memory carveout so that three 66 KB CTAs fit per SM
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(pair_forward_tc_kernel<3>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess) done = true;
  return e;
}

cudaError_t launch_forward(const FwdParams& prm, int precision, int variant, int n_ctas,
                           cudaStream_t s) {
  if (precision == 0) {
    if (variant == 1) pair_forward_kernel<double, 3><<<n_ctas, kThreads, 0, s>>>(prm);
    else pair_forward_kernel<double, 2><<<n_ctas, kThreads, 0, s>>>(prm);
  } else if (variant == 2) {
    cudaError_t e = tc_attr();
    if (e != cudaSuccess) return e;
    pair_forward_tc_kernel<3><<<n_ctas, kThreads, kTcSmem, s>>>(prm);
  } else {
    if (variant == 1) pair_forward_kernel<float, 3><<<n_ctas, kThreads, 0, s>>>(prm);
    else pair_forward_kernel<float, 2><<<n_ctas, kThreads, 0, s>>>(prm);
  }
  return cudaGetLastError();
}

int forward_blocks_per_sm(int precision, int variant) {
  int n = 0;
  if (precision == 0) {
    if (variant == 1)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pair_forward_kernel<double, 3>, kThreads, 0);
    else if (variant == 0)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pair_forward_kernel<double, 2>, kThreads, 0);
  } else if (variant == 2) {
    if (tc_attr() != cudaSuccess) return 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pair_forward_tc_kernel<3>, kThreads, kTcSmem);
    // resource model (registers, shared memory with the per-CTA reserve,
    // threads); the runtime's answer for this dynamic-smem kernel can be lower
    cudaFuncAttributes fa{};
    int dev = 0, smem_sm = 0, regs_sm = 0, thr_sm = 0, reserve = 0;
    if (cudaFuncGetAttributes(&fa, pair_forward_tc_kernel<3>) == cudaSuccess &&
        cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&reserve, cudaDevAttrReservedSharedMemoryPerBlock, dev) == cudaSuccess) {
      const int by_regs = regs_sm / std::max(1, fa.numRegs * kThreads);
      const int by_smem = smem_sm / (int)(fa.sharedSizeBytes + kTcSmem + reserve);
      const int by_thr = thr_sm / kThreads;
      n = std::max(n, std::min(by_regs, std::min(by_smem, by_thr)));
    }
    n = std::min(n, 4);  // 4 x 128 TMEM columns per SM at most
  } else {
    if (variant == 1)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pair_forward_kernel<float, 3>, kThreads, 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pair_forward_kernel<float, 2>, kThreads, 0);
  }
  return n;
}

// Deterministic total: thread t sums a contiguous range of pairs in order,
// then a fixed shared-memory tree.  out3 = (E, number of non-OK pairs, first
// non-OK pair or -1).
__global__ void __launch_bounds__(1024) energy_total_kernel(const double* e_pair,
                                                            const int32_t* status, int64_t n,
                                                            const int32_t* err, double* out3) {
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
    out3[3] = (err && *err) ? 1.0 : 0.0;
  }
}

cudaError_t launch_energy_total(const double* e_pair, const int32_t* status, int64_t n_pairs,
                                const int32_t* err, double* out3, cudaStream_t s) {
  energy_total_kernel<<<1, 1024, 0, s>>>(e_pair, status, n_pairs, err, out3);
  return cudaGetLastError();
}

// Streamed inputs, before the autotuner's sample launches (whose pairs come
// from every group): one thread waits for every group's flag in turn.
__global__ void wait_ready_kernel(const uint32_t* ready, int32_t n_groups, uint32_t epoch,
                                  uint64_t timeout_ns, int32_t* err) {
  if (threadIdx.x != 0) return;
  for (int32_t g = 0; g < n_groups; ++g)
    if (!wait_ready(ready, g, epoch, timeout_ns)) {
      atomicExch(err, 1);
      return;
    }
}

cudaError_t launch_wait_ready(const uint32_t* ready, int32_t n_groups, uint32_t epoch,
                              uint64_t timeout_ns, int32_t* err, cudaStream_t s) {
  wait_ready_kernel<<<1, 32, 0, s>>>(ready, n_groups, epoch, timeout_ns, err);
  return cudaGetLastError();
}

}  // namespace pf12

// ---------------------------------------------------------------------------
// Allocation-free variant of the forward path (pf12_energy_noalloc).
//
// Some callers cannot call cudaMalloc at all: code running inside a memory
// pool or arena they do not own, plugins of a host program that owns every
// device allocation, or callers that have just been refused more memory and
// still need an energy.  For them the whole scratch of one forward pass (work
// queue head, per-pair status and contractions, pair descriptors and the
// per-CTA Cholesky/solve slabs) lives in this file-scope device array.  Every
// GPU that loads the library holds it until the process exits.
namespace {

constexpr size_t kNoallocScratchBytes = size_t(64) << 20;  // 64 MiB
static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchBytes / sizeof(double)];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};   // device address of g_noalloc_scratch, per device

inline size_t round256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" int pf12_energy_noalloc(int32_t n_orb, const int8_t* kind, int64_t n_pairs,
                                   const int32_t* pi, const int32_t* pj, const int32_t* n_pao,
                                   const int32_t* n_pno, const int32_t* n_aux,
                                   const pf12_tensors* t, int32_t precision, void* stream,
                                   double* V_dev, double* e_pair_dev, double* E_host) {
  using namespace pf12;
  if (precision != PF12_FP64 && precision != PF12_MIXED_FP32) return PF12_ERR_UNSUPPORTED;
  if (n_pairs < 0 || n_orb < 0) return PF12_ERR_INVALID_ARG;
  if (n_pairs == 0) {
    if (E_host) *E_host = 0.0;
    return PF12_OK;
  }
  if (!kind || !pi || !pj || !n_pao || !n_pno || !n_aux || !t || !V_dev || !e_pair_dev)
    return PF12_ERR_INVALID_ARG;
  const double* ptrs[8] = {t->Ag_i, t->Ag_j, t->Af_i, t->Af_j, t->Jg, t->Jf, t->Q, t->T};
  for (const double* p : ptrs)
    if (!p || (reinterpret_cast<uintptr_t>(p) & 15u)) return PF12_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(V_dev) & 15u) || !t->off_pm || !t->off_mm || !t->off_pk ||
      !t->off_kk)
    return PF12_ERR_INVALID_ARG;
  for (int32_t o = 0; o < n_orb; ++o)
    if (kind[o] != 0 && kind[o] != 1) return PF12_ERR_INVALID_ARG;

  // sizes: every pair checked, the largest slab found
  int64_t max_ws = 0;
  for (int64_t P = 0; P < n_pairs; ++P) {
    const int32_t i = pi[P], j = pj[P], p = n_pao[P], k = n_pno[P], m = n_aux[P];
    if (i < 0 || j < 0 || i >= n_orb || j >= n_orb || i > j) return PF12_ERR_INVALID_ARG;
    if (p < 1 || k < 1 || m < 1 || k > p || m > kMaxAux || k > kMaxPno) return PF12_ERR_INVALID_ARG;
    const int64_t offs[4] = {t->off_pm[P], t->off_mm[P], t->off_pk[P], t->off_kk[P]};
    const int64_t sizes[4] = {(int64_t)p * m, (int64_t)m * m, (int64_t)p * k, (int64_t)k * k};
    const int64_t lens[4] = {t->len_pm, t->len_mm, t->len_pk, t->len_kk};
    for (int q = 0; q < 4; ++q)
      if (offs[q] < 0 || (offs[q] & 1) || offs[q] + sizes[q] > lens[q]) return PF12_ERR_INVALID_ARG;
    max_ws = std::max(max_ws, fwd_ws(p, k, m));
  }
  // scratch layout: counter | status | dx | out3 | descriptors | slabs
  const size_t off_status = 256;
  const size_t off_dx = off_status + round256(sizeof(int32_t) * n_pairs);
  const size_t off_out3 = off_dx + round256(sizeof(double) * 2 * n_pairs);
  const size_t off_desc = off_out3 + 256;
  const size_t off_work = off_desc + round256(sizeof(PairDesc) * n_pairs);
  const size_t stride = round256(sizeof(double) * (size_t)max_ws);
  if (off_work + stride > kNoallocScratchBytes) return PF12_ERR_INVALID_ARG;  // beyond the maximum

  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PF12_ERR_CUDA;
  char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return PF12_ERR_CUDA;
      g_noalloc_ptr[dev] = ptr;
    }
    base = static_cast<char*>(g_noalloc_ptr[dev]);
  }
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PF12_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // descriptors in the caller's pair order, staged through a small stack buffer
  PairDesc stage[64];
  for (int64_t P0 = 0; P0 < n_pairs; P0 += 64) {
    const int64_t nb = std::min<int64_t>(64, n_pairs - P0);
    for (int64_t q = 0; q < nb; ++q) {
      const int64_t P = P0 + q;
      PairDesc& d = stage[q];
      d.off_pm = t->off_pm[P];
      d.off_mm = t->off_mm[P];
      d.off_pk = t->off_pk[P];
      d.off_kk = t->off_kk[P];
      d.p = n_pao[P];
      d.k = n_pno[P];
      d.m = n_aux[P];
      d.pair = (int32_t)P;
      const int bi = kind[pi[P]] == 0, bj = kind[pj[P]] == 0;
      if (pi[P] == pj[P]) {
        d.n_ab = (int8_t)bi;
        d.n_aa = d.n_bb = 0;
      } else {
        d.n_ab = (int8_t)(bi + bj);
        d.n_aa = 1;
        d.n_bb = (int8_t)(bi * bj);
      }
      d.w_alpha = 3.0f * d.n_ab / 8.0f + (d.n_aa + d.n_bb) / 4.0f;
      d.w_beta = d.n_ab / 8.0f - (d.n_aa + d.n_bb) / 4.0f;
      d.c1 = (int8_t)(kind[pj[P]] == 0);
      d.s = 0;
    }
    // pageable source: the copy has consumed `stage` when the call returns
    if (cudaMemcpyAsync(base + off_desc + sizeof(PairDesc) * P0, stage, sizeof(PairDesc) * nb,
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
      return PF12_ERR_CUDA;
  }
  // the queue head must start at zero; status, dx and slabs are fully written
  if (cudaMemsetAsync(base, 0, 256, s) != cudaSuccess) return PF12_ERR_CUDA;

  const int bps = std::max(1, forward_blocks_per_sm(precision, 0));
  int64_t n_ctas = std::min<int64_t>(n_pairs, (int64_t)bps * n_sm);
  n_ctas = std::min<int64_t>(n_ctas, (int64_t)((kNoallocScratchBytes - off_work) / stride));
  FwdParams f{};
  f.Agi = t->Ag_i;
  f.Agj = t->Ag_j;
  f.Afi = t->Af_i;
  f.Afj = t->Af_j;
  f.Jg = t->Jg;
  f.Jf = t->Jf;
  f.Q = t->Q;
  f.T = t->T;
  f.desc = reinterpret_cast<const PairDesc*>(base + off_desc);
  f.n_pairs = n_pairs;
  f.V = V_dev;
  f.e_pair = e_pair_dev;
  f.dx = reinterpret_cast<double*>(base + off_dx);
  f.status = reinterpret_cast<int32_t*>(base + off_status);
  f.work = reinterpret_cast<double*>(base + off_work);
  f.ws_stride = (int64_t)(stride / sizeof(double));
  f.counter = reinterpret_cast<int32_t*>(base);
  if (launch_forward(f, precision, 0, (int)n_ctas, s) != cudaSuccess) return PF12_ERR_CUDA;
  double* out3 = reinterpret_cast<double*>(base + off_out3);
  if (launch_energy_total(e_pair_dev, f.status, n_pairs, nullptr, out3, s) != cudaSuccess) return PF12_ERR_CUDA;
  double h3[3] = {0, 0, 0};
  if (cudaMemcpyAsync(h3, out3, sizeof h3, cudaMemcpyDeviceToHost, s) != cudaSuccess) return PF12_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return PF12_ERR_CUDA;
  if (E_host) *E_host = h3[0];
  if (h3[1] > 0) {
    int32_t st = 0;
    if (cudaMemcpy(&st, f.status + (int64_t)h3[2], sizeof st, cudaMemcpyDeviceToHost) != cudaSuccess)
      return PF12_ERR_CUDA;
    return st == PF12_PAIR_NOT_SPD ? PF12_ERR_NOT_SPD : PF12_ERR_NONFINITE;
  }
  return std::isfinite(h3[0]) ? PF12_OK : PF12_ERR_NONFINITE;
}
