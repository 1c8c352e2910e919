// Host side of the fused forward pair kernel (device code: pf12_forward.cuh):
// variant dispatch, the deterministic energy total, the arrival wait used
// before tuning on streamed inputs, and the allocation-free entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "../../include/pairf12.h"
#include "pf12_device.cuh"
#include "pf12_internal.h"

namespace pf12 {

// Forward variants the autotuner chooses from (kFwdLook, kFwdCtasPerSm):
// variant 0 / 1 run the SIMT kernel at MINB = 2 / 3 CTAs per SM (more resident
// pairs per SM hide the serial phases of each pair's factorisation; fewer
// leave more registers per thread); variant 2 (mixed precision only) is the
// tensor-core kernel at 3; variant 3 is variant 1 with Cholesky look-ahead
// groups of 16 panels instead of 8.  Each variant lives in its own
// translation unit under csrc/inst/.
cudaError_t launch_forward(const FwdParams& prm, int precision, int variant, int n_ctas,
                           cudaStream_t s) {
  if (precision == 0) {
    if (variant == 3) return launch_fwd_f64_3_l16(prm, n_ctas, s);
    if (variant == 1) return launch_fwd_f64_3(prm, n_ctas, s);
    return launch_fwd_f64_2(prm, n_ctas, s);
  }
  if (variant == 3) return launch_fwd_f32_3_l16(prm, n_ctas, s);
  if (variant == 2) return launch_fwd_tc_3(prm, n_ctas, s);
  if (variant == 1) return launch_fwd_f32_3(prm, n_ctas, s);
  return launch_fwd_f32_2(prm, n_ctas, s);
}

int forward_blocks_per_sm(int precision, int variant) {
  if (precision == 0) {
    if (variant == 3) return occupancy_fwd_f64_3_l16();
    if (variant == 1) return occupancy_fwd_f64_3();
    if (variant == 0) return occupancy_fwd_f64_2();
    return 0;
  }
  if (variant == 3) return occupancy_fwd_f32_3_l16();
  if (variant == 2) return occupancy_fwd_tc_3();
  if (variant == 1) return occupancy_fwd_f32_3();
  return occupancy_fwd_f32_2();
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
  // every call copies from host stack memory, synchronises the stream and
  // reads the result back: a capturing stream cannot take that, so refuse it
  // before any other CUDA call touches (and would invalidate) the capture
  {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cap) != cudaSuccess) {
      cudaGetLastError();
      return PF12_ERR_CUDA;
    }
    if (cap != cudaStreamCaptureStatusNone) return PF12_ERR_UNSUPPORTED;
  }
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
