// Host side of the C ABI declared in include/pairf12.h: argument checks, pair
// metadata and cost-sorted work queue, workspace sizing, CUDA-graph capture of
// the fused forward launch, deterministic energy total, timers.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/pairf12.h"
#include "pf12_internal.h"

using pf12::PairDesc;

namespace {
// Named host range around each entry point, visible to NVTX-aware profilers
// (header-only NVTX: a no-op unless a tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

struct pf12_ctx {
  int precision = PF12_FP64;
  cudaStream_t stream = nullptr;
  cudaStream_t capture_stream = nullptr;
  size_t ws_cap = 0;
  std::string err = "no error";
  int n_sm = 0;

  // pair metadata
  int64_t n_pairs = 0;
  bool uploaded = false, fitted = false;
  pf12_tensors t{};
  std::vector<int64_t> off_kk;
  std::vector<int32_t> pk;  // n_pno per pair (caller order)
  PairDesc* d_desc = nullptr;
  double* d_V = nullptr;        // len_kk
  double* d_epair = nullptr;    // 3 n
  double* d_dx = nullptr;       // 2 n
  int32_t* d_status = nullptr;  // n
  double* d_out3 = nullptr;     // energy total
  int32_t* d_counter = nullptr;
  double* d_work = nullptr;
  size_t work_bytes = 0;
  int64_t ws_stride = 0, ws_stride_bwd = 0;
  int n_ctas = 0, n_ctas_bwd = 0;
  int64_t max_fwd_ws = 0, max_bwd_ws = 0;

  // autotuner: forward kernel variant (occupancy), its CTA counts, tuning sample
  int variant = -1;
  int forced = -1;
  int bwd_variant = -1;
  int n_ctas_bwd_v[pf12::kBwdVariants] = {};
  double tune_bwd_ms[pf12::kBwdVariants] = {};
  int n_ctas_v[pf12::kFwdVariants] = {};
  std::string tuner_cache;
  std::string tune_key;
  double tune_ms[pf12::kFwdVariants] = {};
  PairDesc* d_desc_sample = nullptr;
  int64_t n_sample = 0;

  // gather mode
  bool gather = false;
  int32_t n_orb = 0;
  std::vector<int64_t> g_off_pm;   // library-computed packed offsets of per-pair gradient blocks
  int64_t g_len_pm = 0, g_len_orb = 0;
  const double *g_Bg = nullptr, *g_Bf = nullptr;
  pf12::GatherDesc* d_gdesc = nullptr;
  PairDesc* d_desc_by_pair = nullptr;
  int32_t *d_map_pao = nullptr, *d_map_aux = nullptr;
  int64_t* d_orb_ptr = nullptr;
  int32_t* d_orb_list = nullptr;
  int64_t* d_off_orb = nullptr;
  int32_t* d_ld_orb = nullptr;
  double* d_dA = nullptr;          // 4 x g_len_pm, allocated by the first gather backward
  unsigned char* d_tmaps = nullptr;  // 2 x n_orb TMA tensor maps (128 B each) of the orbital blocks
  size_t cap_tmaps = 0;
  bool use_tma = false;
  bool sieve_plain = false;        // option: sieve with plain loads only
  bool augment = false;            // option: SOMO-augmented PNO space
  bool packed = false;             // option: metrics as packed lower triangles
  uint32_t debug_wait_polls = 0;   // test hook (pf12_opts.debug_wait_timeout)

  // streamed inputs (pf12_set_arrival): the queue is ordered group by group
  std::vector<PairDesc> h_desc;    // caller order, kept from the upload
  std::vector<double> h_cost;
  std::vector<int64_t> arr_end;    // group ends in the caller's pair order
  const uint32_t* arr_ready = nullptr;
  uint32_t arr_epoch = 0;
  bool arr_dirty = false;          // queue order to rebuild before the next fit
  int32_t* d_slot_group = nullptr;
  size_t cap_sg = 0;

  // full mode: the complete pair energy (pf12_upload_full)
  bool full = false;
  pf12_full_tensors ft{};
  pf12::FullDesc* d_fdesc = nullptr;
  pf12::FullDesc* d_fdesc_sample = nullptr;
  double* d_terms = nullptr;
  size_t cap_fdesc = 0, cap_fsample = 0, cap_terms = 0;
  int n_ctas_full_v[pf12::kFullVariants] = {};

  // graph of the forward launch
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;

  // capacities (elements) of the device buffers: re-uploads reuse them and only
  // grow, so a re-upload issues no cudaFree (which would synchronise the device
  // and stall copies running on other streams)
  size_t cap_desc = 0, cap_sample = 0, cap_V = 0, cap_ep = 0, cap_dx = 0, cap_st = 0, cap_work = 0, cap_gdesc = 0,
         cap_dbp = 0, cap_mp = 0, cap_ma = 0, cap_optr = 0, cap_olist = 0, cap_oorb = 0,
         cap_ld = 0, cap_dA = 0;
  bool fixed_allocated = false;
  std::string prev_key;      // tuning key of the previous upload (variant kept if equal)
  int prev_variant = -1;
  std::string prev_bwd_key;  // the same for the adjoint's variant
  int prev_bwd_variant = -1;

  // timers
  cudaEvent_t ev[6] = {};
  bool t_fit = false, t_energy = false, t_bwd = false;
  double flops64 = 0, flops_mix = 0, bytes_in = 0;
};

namespace {

int fail(pf12_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(pf12_ctx* c, cudaError_t e, const char* where) {
  return fail(c, PF12_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define PF12_CUDA(ctx, call)                               \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

// Forget the pair list (buffers are kept for the next upload).
void free_pairs(pf12_ctx* c) {
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->graph_exec = nullptr;
  c->graph = nullptr;
  if (c->variant >= 0) {
    c->prev_key = c->tune_key;
    c->prev_variant = c->variant;
  }
  if (c->bwd_variant >= 0) {
    c->prev_bwd_key = c->tune_key;
    c->prev_bwd_variant = c->bwd_variant;
  }
  c->variant = -1;
  c->bwd_variant = -1;
  c->n_sample = 0;
  c->arr_end.clear();
  c->arr_ready = nullptr;
  c->arr_dirty = false;
  c->gather = false;
  c->full = false;
  c->uploaded = c->fitted = false;
  c->n_pairs = 0;
}

void release_all(pf12_ctx* c) {
  free_pairs(c);
  void* ptrs[] = {c->d_desc, c->d_gdesc, c->d_desc_by_pair, c->d_map_pao, c->d_map_aux,
                  c->d_orb_ptr, c->d_orb_list, c->d_off_orb, c->d_ld_orb, c->d_dA,
                  c->d_desc_sample, c->d_V, c->d_epair, c->d_dx, c->d_status, c->d_out3,
                  c->d_counter, c->d_work, c->d_tmaps, c->d_slot_group, c->d_fdesc,
                  c->d_fdesc_sample, c->d_terms};
  for (void* q : ptrs)
    if (q) cudaFree(q);
}

template <typename T>
cudaError_t grow(T*& p, size_t& cap, size_t count) {
  count = std::max<size_t>(count, 1);
  if (p && count <= cap) return cudaSuccess;
  if (p) cudaFree(p);
  p = nullptr;
  cap = 0;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p), sizeof(T) * count);
  if (e == cudaSuccess) cap = count;
  else p = nullptr;
  return e;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

pf12::FwdParams fwd_params(pf12_ctx* c) {
  pf12::FwdParams f{};
  f.Agi = c->t.Ag_i;
  f.Agj = c->t.Ag_j;
  f.Afi = c->t.Af_i;
  f.Afj = c->t.Af_j;
  f.Jg = c->t.Jg;
  f.Jf = c->t.Jf;
  f.Q = c->t.Q;
  f.T = c->t.T;
  f.desc = c->d_desc;
  f.n_pairs = c->n_pairs;
  f.V = c->d_V;
  f.e_pair = c->d_epair;
  f.dx = c->d_dx;
  f.status = c->d_status;
  f.work = c->d_work;
  f.ws_stride = c->ws_stride;
  f.counter = c->d_counter;
  f.err = c->d_counter + 2;
  f.debug_wait_polls = c->debug_wait_polls;
  f.metric_packed = c->packed ? 1 : 0;
  if (c->gather) {
    f.tmaps = c->use_tma ? c->d_tmaps : nullptr;
    f.gdesc = c->d_gdesc;
    f.Bg = c->g_Bg;
    f.Bf = c->g_Bf;
    f.map_pao = c->d_map_pao;
    f.map_aux = c->d_map_aux;
  }
  return f;
}

}  // namespace

extern "C" {

int pf12_create(pf12_ctx** out, const pf12_opts* o) {
  if (!out) return PF12_ERR_INVALID_ARG;
  *out = nullptr;
  pf12_ctx* c = new pf12_ctx();
  if (o) {
    if (o->precision != PF12_FP64 && o->precision != PF12_MIXED_FP32) {
      delete c;
      return PF12_ERR_UNSUPPORTED;
    }
    c->precision = o->precision;
    c->stream = static_cast<cudaStream_t>(o->cuda_stream);
    c->ws_cap = o->workspace_bytes;
    if (o->tuner_cache) c->tuner_cache = o->tuner_cache;
    if (o->force_variant >= pf12::kFwdVariants) {
      delete c;
      return PF12_ERR_UNSUPPORTED;
    }
    c->forced = o->force_variant;
    c->sieve_plain = o->sieve_plain != 0;
    c->augment = o->augment_somo != 0;
    c->packed = o->metric_packed != 0;
    c->debug_wait_polls = o->debug_wait_timeout ? 4096u : 0u;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking);
  for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = cudaEventCreate(&c->ev[i]);
  if (e != cudaSuccess) {
    delete c;
    return PF12_ERR_CUDA;
  }
  *out = c;
  return PF12_OK;
}

int pf12_set_stream(pf12_ctx* c, void* s) {
  if (!c) return PF12_ERR_INVALID_ARG;
  c->stream = static_cast<cudaStream_t>(s);
  return PF12_OK;
}

static int upload_impl(pf12_ctx* c, int32_t n_orb, const int8_t* kind, int64_t n_pairs,
                       const int32_t* pi, const int32_t* pj, const int32_t* n_pao,
                       const int32_t* n_pno, const int32_t* n_aux, const pf12_tensors* t_in,
                       const pf12_gather_tensors* g) {
  NvtxRange nvtx("pf12_upload_pairs");
  if (!c) return PF12_ERR_INVALID_ARG;
  free_pairs(c);
  if (n_pairs < 0 || n_orb < 0) return fail(c, PF12_ERR_INVALID_ARG, "negative count");
  if (n_pairs > 0 && (!kind || !pi || !pj || !n_pao || !n_pno || !n_aux || (!t_in && !g)))
    return fail(c, PF12_ERR_INVALID_ARG, "null metadata pointer");
  pf12_tensors tg{};
  const pf12_tensors* t = t_in;
  if (g && n_pairs > 0) {
    // gather mode: factors come from per-orbital blocks; per-pair gradient
    // blocks (backward) use a library-computed packed layout
    const double* ptrs[6] = {g->Bg, g->Bf, g->Jg, g->Jf, g->Q, g->T};
    for (const double* p : ptrs)
      if (!p || !aligned16(p)) return fail(c, PF12_ERR_INVALID_ARG, "tensor pointer null or not 16-byte aligned");
    if (!g->off_orb || !g->ext_pao || !g->ext_aux || !g->ext_ld || !g->map_pao || !g->map_aux ||
        !g->off_map_pao || !g->off_map_aux || !g->off_mm || !g->off_pk || !g->off_kk)
      return fail(c, PF12_ERR_INVALID_ARG, "null gather-mode array");
    for (int32_t o = 0; o < n_orb; ++o)
      if (g->off_orb[o] < 0 || g->ext_pao[o] < 0 || g->ext_aux[o] < 0 || g->ext_ld[o] < g->ext_aux[o] ||
          g->off_orb[o] + (int64_t)g->ext_pao[o] * g->ext_ld[o] > g->len_orb)
        return fail(c, PF12_ERR_INVALID_ARG, "orbital block outside Bg/Bf or ld < M");
    c->g_off_pm.assign(n_pairs, 0);
    int64_t acc = 0;
    for (int64_t P = 0; P < n_pairs; ++P) {
      c->g_off_pm[P] = acc;
      acc += ((int64_t)std::max(n_pao[P], 0) * std::max(n_aux[P], 0) + 31) / 32 * 32;
    }
    tg.Jg = g->Jg;
    tg.Jf = g->Jf;
    tg.Q = g->Q;
    tg.T = g->T;
    tg.off_pm = c->g_off_pm.data();
    tg.off_mm = g->off_mm;
    tg.off_pk = g->off_pk;
    tg.off_kk = g->off_kk;
    tg.len_pm = acc;
    tg.len_mm = g->len_mm;
    tg.len_pk = g->len_pk;
    tg.len_kk = g->len_kk;
    t = &tg;
  } else if (n_pairs > 0) {
    const double* ptrs[8] = {t->Ag_i, t->Ag_j, t->Af_i, t->Af_j, t->Jg, t->Jf, t->Q, t->T};
    for (const double* p : ptrs)
      if (!p || !aligned16(p)) return fail(c, PF12_ERR_INVALID_ARG, "tensor pointer null or not 16-byte aligned");
    if (!t->off_pm || !t->off_mm || !t->off_pk || !t->off_kk)
      return fail(c, PF12_ERR_INVALID_ARG, "null offset array");
  }
  int32_t n_somo = 0;
  for (int32_t o = 0; o < n_orb; ++o) {
    if (kind[o] != 0 && kind[o] != 1) return fail(c, PF12_ERR_INVALID_ARG, "orb_kind must be 0 or 1");
    n_somo += kind[o];
  }
  const bool gm = g != nullptr;
  if (gm && c->augment && n_somo > 0)
    return fail(c, PF12_ERR_UNSUPPORTED, "SOMO augmentation is available in packed mode only");
  // SOMO-augmented PNO space: every pair gains the n_somo SOMO rows / virtuals
  const int32_t s_aug = c->augment ? n_somo : 0;
  std::vector<pf12::GatherDesc> gdesc(gm ? n_pairs : 0);

  std::vector<PairDesc> desc(n_pairs);
  std::vector<double> cost(n_pairs);
  double f64 = 0, fmix = 0, bytes = 0;
  int64_t max_fwd = 0, max_bwd = 0;
  c->off_kk.assign(n_pairs, 0);
  c->pk.assign(n_pairs, 0);
  for (int64_t P = 0; P < n_pairs; ++P) {
    const int32_t i = pi[P], j = pj[P], p = n_pao[P], kq = n_pno[P], m = n_aux[P];
    const int32_t k = kq + s_aug, pr = p + s_aug;   // virtual dimension, factor rows
    char buf[160];
    if (i < 0 || j < 0 || i >= n_orb || j >= n_orb || i > j) {
      snprintf(buf, sizeof buf, "pair %lld: need 0 <= i <= j < n_orb", (long long)P);
      return fail(c, PF12_ERR_INVALID_ARG, buf);
    }
    if (p < 1 || kq < 1 || m < 1 || kq > p || m > pf12::kMaxAux || k > pf12::kMaxPno) {
      snprintf(buf, sizeof buf, "pair %lld: sizes p=%d k=%d m=%d out of range", (long long)P, p, kq, m);
      return fail(c, PF12_ERR_INVALID_ARG, buf);
    }
    const int64_t offs[4] = {t->off_pm[P], t->off_mm[P], t->off_pk[P], t->off_kk[P]};
    const int64_t mm = c->packed ? (int64_t)m * (m + 1) / 2 : (int64_t)m * m;
    const int64_t sizes[4] = {(int64_t)pr * m, mm, (int64_t)p * kq, (int64_t)k * k};
    const int64_t lens[4] = {t->len_pm, t->len_mm, t->len_pk, t->len_kk};
    for (int q = 0; q < 4; ++q)
      if (offs[q] < 0 || (offs[q] & 1) || offs[q] + sizes[q] > lens[q]) {
        snprintf(buf, sizeof buf, "pair %lld: offset %d misaligned or block outside its buffer", (long long)P, q);
        return fail(c, PF12_ERR_INVALID_ARG, buf);
      }
    PairDesc& d = desc[P];
    d.off_pm = offs[0];
    d.off_mm = offs[1];
    d.off_pk = offs[2];
    d.off_kk = offs[3];
    d.p = p;
    d.k = k;
    d.m = m;
    d.pair = (int32_t)P;
    const int ki = kind[i], kj = kind[j];
    const int ai = 1, bi = ki == 0, aj = 1, bj = kj == 0;
    if (i == j) {
      d.n_ab = (int8_t)(ai * bi);
      d.n_aa = d.n_bb = 0;
    } else {
      d.n_ab = (int8_t)(ai * bj + aj * bi);
      d.n_aa = (int8_t)(ai * aj);
      d.n_bb = (int8_t)(bi * bj);
    }
    d.w_alpha = 3.0f * d.n_ab / 8.0f + (d.n_aa + d.n_bb) / 4.0f;
    d.w_beta = d.n_ab / 8.0f - (d.n_aa + d.n_bb) / 4.0f;
    d.c1 = (int8_t)(kj == 0);
    d.s = s_aug;
    const double dm = m, dk = k, dp = p, dkq = kq, dpr = pr;
    const double c64 = dm * dm * dm / 3.0 + 4.0 * dk * dm * dm;
    const double cmix = 8.0 * dp * dkq * dm + 2.0 * dk * dm * dm + 4.0 * dk * dk * dm;
    cost[P] = c64 + cmix / 8.0;
    f64 += c64;
    fmix += cmix;
    bytes += 8.0 * (4.0 * dpr * dm + 2.0 * (double)mm + dp * dkq + dk * dk);
    max_fwd = std::max(max_fwd, pf12::fwd_ws(p, k, m, gm, c->packed));
    max_bwd = std::max(max_bwd, pf12::bwd_ws(p, k, m, gm, c->packed));
    c->off_kk[P] = offs[3];
    c->pk[P] = k;
    if (gm) {
      // maps: in range for the two orbitals' blocks and strictly increasing
      const int64_t op = g->off_map_pao[P], oa = g->off_map_aux[P];
      if (op < 0 || oa < 0 || op + 2 * (int64_t)p > g->len_map_pao || oa + 2 * (int64_t)m > g->len_map_aux) {
        snprintf(buf, sizeof buf, "pair %lld: index map outside its array", (long long)P);
        return fail(c, PF12_ERR_INVALID_ARG, buf);
      }
      const int32_t orb[2] = {i, j};
      for (int side = 0; side < 2; ++side) {
        const int32_t* rows = g->map_pao + op + (int64_t)side * p;
        const int32_t* cols = g->map_aux + oa + (int64_t)side * m;
        bool okm = true;
        for (int r = 0; r < p; ++r)
          okm &= rows[r] >= 0 && rows[r] < g->ext_pao[orb[side]] && (r == 0 || rows[r] > rows[r - 1]);
        for (int q = 0; q < m; ++q)
          okm &= cols[q] >= 0 && cols[q] < g->ext_aux[orb[side]] && (q == 0 || cols[q] > cols[q - 1]);
        if (!okm) {
          snprintf(buf, sizeof buf, "pair %lld: map out of range or not strictly increasing", (long long)P);
          return fail(c, PF12_ERR_INVALID_ARG, buf);
        }
      }
      pf12::GatherDesc& gd = gdesc[P];
      gd.off_i = g->off_orb[i];
      gd.off_j = g->off_orb[j];
      gd.map_pao = op;
      gd.map_aux = oa;
      gd.ld_i = g->ext_ld[i];
      gd.ld_j = g->ext_ld[j];
      gd.orb_i = i;
      gd.orb_j = j;
    }
  }
  // longest-processing-time order for the persistent queue (ties: list order)
  std::vector<int64_t> order(n_pairs);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return cost[a] > cost[b]; });
  std::vector<PairDesc> sorted(n_pairs);
  for (int64_t s = 0; s < n_pairs; ++s) sorted[s] = desc[order[s]];
  c->h_desc = desc;
  c->h_cost = cost;

  if (t) c->t = *t;
  c->n_pairs = n_pairs;
  c->flops64 = f64 + (c->precision == PF12_FP64 ? fmix : 0.0);
  c->flops_mix = fmix;
  c->bytes_in = bytes;
  c->max_fwd_ws = max_fwd;
  c->max_bwd_ws = max_bwd;

  // workspace: one slab per persistent CTA, shared by forward and backward;
  // sized for the forward variant with the most resident CTAs
  const int64_t stride = (max_fwd + 31) / 32 * 32;
  const int64_t stride_b = (max_bwd + 31) / 32 * 32;
  int64_t cap_f = INT64_MAX, cap_b = INT64_MAX;
  if (c->ws_cap) {
    cap_f = (int64_t)(c->ws_cap / 8) / std::max<int64_t>(stride, 1);
    cap_b = (int64_t)(c->ws_cap / 8) / std::max<int64_t>(stride_b, 1);
    if (n_pairs > 0 && (cap_f < 1 || cap_b < 1))
      return fail(c, PF12_ERR_OOM, "workspace_bytes too small for the largest pair");
  }
  int64_t want = 1;
  for (int v = 0; v < pf12::kFwdVariants; ++v) {
    const int bps = pf12::forward_blocks_per_sm(c->precision, v);
    cudaGetLastError();
    if (bps <= 0) {       // variant not available for this precision
      c->n_ctas_v[v] = 0;
      continue;
    }
    int64_t n_v = std::min<int64_t>(n_pairs, (int64_t)bps * c->n_sm);
    n_v = std::max<int64_t>(1, std::min(n_v, cap_f));
    c->n_ctas_v[v] = (int)n_v;
    want = std::max(want, n_v);
  }
  int64_t want_b = 1;
  for (int v = 0; v < pf12::kBwdVariants; ++v) {
    const int bps_b = std::max(1, pf12::backward_blocks_per_sm(c->precision, v));
    int64_t n_v = std::min<int64_t>(n_pairs, (int64_t)bps_b * c->n_sm);
    n_v = std::max<int64_t>(1, std::min(n_v, cap_b));
    c->n_ctas_bwd_v[v] = (int)n_v;
    want_b = std::max(want_b, n_v);
  }
  c->n_ctas = c->n_ctas_v[0];
  c->n_ctas_bwd = c->n_ctas_bwd_v[0];
  c->ws_stride = stride;
  c->ws_stride_bwd = stride_b;
  const size_t work_doubles = (size_t)std::max(want * stride, want_b * stride_b);

  // tuning sample: pairs spread evenly over the cost-sorted list, eight per CTA
  // of the widest variant, so that the last wave's tail is a small share of
  // the timed launch (with three per CTA, tail noise of +-2 % decided between
  // variants whose full-list rates differ by 5 %)
  std::vector<PairDesc> sample;
  const int64_t n_s = std::min<int64_t>(n_pairs, 8 * (int64_t)want);
  for (int64_t q = 0; q < n_s; ++q) sample.push_back(sorted[(q * n_pairs) / std::max<int64_t>(n_s, 1)]);
  {
    std::vector<int> ms, ks;
    for (int64_t P = 0; P < n_pairs; ++P) { ms.push_back(n_aux[P]); ks.push_back(n_pno[P]); }
    std::sort(ms.begin(), ms.end());
    std::sort(ks.begin(), ks.end());
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, dev);
    char key[256];
    // coarse size signature: lists that differ only a little (batches of one
    // stream, repeated uploads) share their tuning
    snprintf(key, sizeof key, "%s|sm%d|prec%d|m%d|k%d|gather%d", prop.name, c->n_sm, c->precision,
             n_pairs ? ms[n_pairs / 2] / 200 * 200 : 0, n_pairs ? ks[n_pairs / 2] / 20 * 20 : 0,
             (int)gm);
    c->tune_key = key;
    for (char& ch : c->tune_key)
      if (ch == ' ') ch = '_';
  }
  if (c->forced < 0 && c->prev_variant >= 0 && c->prev_key == c->tune_key &&
      c->n_ctas_v[c->prev_variant] > 0) {
    c->variant = c->prev_variant;     // same size signature as the last list: keep its tuning
    c->n_ctas = c->n_ctas_v[c->variant];
  }
  if (c->prev_bwd_variant >= 0 && c->prev_bwd_key == c->tune_key &&
      c->n_ctas_bwd_v[c->prev_bwd_variant] > 0)
    c->bwd_variant = c->prev_bwd_variant;

  const size_t n = (size_t)std::max<int64_t>(n_pairs, 1);
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = grow(c->d_desc, c->cap_desc, n);
  if (e == cudaSuccess) e = grow(c->d_V, c->cap_V, (size_t)std::max<int64_t>(t ? t->len_kk : 0, 2));
  if (e == cudaSuccess) e = grow(c->d_epair, c->cap_ep, 3 * n);
  if (e == cudaSuccess) e = grow(c->d_dx, c->cap_dx, 2 * n);
  if (e == cudaSuccess) e = grow(c->d_status, c->cap_st, n);
  if (e == cudaSuccess && !c->fixed_allocated) {
    e = cudaMalloc(&c->d_out3, sizeof(double) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_counter, sizeof(int32_t) * 4);
    if (e == cudaSuccess) c->fixed_allocated = true;
  }
  if (e == cudaSuccess && n_pairs > 0) e = grow(c->d_work, c->cap_work, work_doubles);
  if (e == cudaSuccess && n_s > 0) e = grow(c->d_desc_sample, c->cap_sample, (size_t)n_s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_pairs(c);
    return fail(c, e == cudaErrorMemoryAllocation ? PF12_ERR_OOM : PF12_ERR_CUDA,
                std::string("device allocation: ") + cudaGetErrorString(e));
  }
  c->work_bytes = sizeof(double) * work_doubles;
  PF12_CUDA(c, cudaMemcpyAsync(c->d_desc, sorted.data(), sizeof(PairDesc) * n_pairs,
                               cudaMemcpyHostToDevice, c->stream));
  if (n_s > 0)
    PF12_CUDA(c, cudaMemcpyAsync(c->d_desc_sample, sample.data(), sizeof(PairDesc) * n_s,
                                 cudaMemcpyHostToDevice, c->stream));
  c->n_sample = n_s;
  if (t && t->len_kk > 0) PF12_CUDA(c, cudaMemsetAsync(c->d_V, 0, sizeof(double) * t->len_kk, c->stream));
  PF12_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(int32_t) * n, c->stream));
  PF12_CUDA(c, cudaMemsetAsync(c->d_counter, 0, sizeof(int32_t) * 4, c->stream));
  PF12_CUDA(c, cudaMemsetAsync(c->d_epair, 0, sizeof(double) * 3 * n, c->stream));
  if (gm && n_pairs > 0) {
    // device copies of the maps, descriptors and the per-orbital scatter lists
    std::vector<int64_t> orb_ptr(n_orb + 1, 0);
    for (int64_t P = 0; P < n_pairs; ++P) {
      ++orb_ptr[pi[P] + 1];
      ++orb_ptr[pj[P] + 1];
    }
    for (int32_t o = 0; o < n_orb; ++o) orb_ptr[o + 1] += orb_ptr[o];
    std::vector<int32_t> orb_list(2 * n_pairs);
    std::vector<int64_t> fill(orb_ptr.begin(), orb_ptr.end() - 1);
    for (int64_t P = 0; P < n_pairs; ++P) {
      orb_list[fill[pi[P]]++] = (int32_t)(2 * P);
      orb_list[fill[pj[P]]++] = (int32_t)(2 * P + 1);
    }
    std::vector<int64_t> off_orb(g->off_orb, g->off_orb + n_orb);
    std::vector<int32_t> ld_orb(g->ext_ld, g->ext_ld + n_orb);
    cudaError_t e2 = cudaSuccess;
    if (e2 == cudaSuccess) e2 = grow(c->d_gdesc, c->cap_gdesc, (size_t)n_pairs);
    if (e2 == cudaSuccess) e2 = grow(c->d_desc_by_pair, c->cap_dbp, (size_t)n_pairs);
    if (e2 == cudaSuccess) e2 = grow(c->d_map_pao, c->cap_mp, (size_t)g->len_map_pao);
    if (e2 == cudaSuccess) e2 = grow(c->d_map_aux, c->cap_ma, (size_t)g->len_map_aux);
    if (e2 == cudaSuccess) e2 = grow(c->d_orb_ptr, c->cap_optr, (size_t)n_orb + 1);
    if (e2 == cudaSuccess) e2 = grow(c->d_orb_list, c->cap_olist, 2 * (size_t)n_pairs);
    if (e2 == cudaSuccess) e2 = grow(c->d_off_orb, c->cap_oorb, (size_t)n_orb);
    if (e2 == cudaSuccess) e2 = grow(c->d_ld_orb, c->cap_ld, (size_t)n_orb);
    if (e2 != cudaSuccess) {
      cudaGetLastError();
      free_pairs(c);
      return fail(c, PF12_ERR_OOM, std::string("device allocation: ") + cudaGetErrorString(e2));
    }
    PF12_CUDA(c, cudaMemcpyAsync(c->d_gdesc, gdesc.data(), sizeof(pf12::GatherDesc) * n_pairs, cudaMemcpyHostToDevice, c->stream));
    PF12_CUDA(c, cudaMemcpyAsync(c->d_desc_by_pair, desc.data(), sizeof(PairDesc) * n_pairs, cudaMemcpyHostToDevice, c->stream));
    PF12_CUDA(c, cudaMemcpyAsync(c->d_map_pao, g->map_pao, sizeof(int32_t) * g->len_map_pao, cudaMemcpyHostToDevice, c->stream));
    PF12_CUDA(c, cudaMemcpyAsync(c->d_map_aux, g->map_aux, sizeof(int32_t) * g->len_map_aux, cudaMemcpyHostToDevice, c->stream));
    PF12_CUDA(c, cudaMemcpyAsync(c->d_orb_ptr, orb_ptr.data(), sizeof(int64_t) * (n_orb + 1), cudaMemcpyHostToDevice, c->stream));
    PF12_CUDA(c, cudaMemcpyAsync(c->d_orb_list, orb_list.data(), sizeof(int32_t) * 2 * n_pairs, cudaMemcpyHostToDevice, c->stream));
    PF12_CUDA(c, cudaMemcpyAsync(c->d_off_orb, off_orb.data(), sizeof(int64_t) * n_orb, cudaMemcpyHostToDevice, c->stream));
    PF12_CUDA(c, cudaMemcpyAsync(c->d_ld_orb, ld_orb.data(), sizeof(int32_t) * n_orb, cudaMemcpyHostToDevice, c->stream));
    // TMA tensor maps of the orbital blocks for the gather4 sieve: rank 2,
    // (ld_o columns, P_o rows), box 128 x 1; every block must start and stride
    // on 16 bytes, else the sieve keeps plain loads
    c->use_tma = false;
    bool eligible = !c->sieve_plain;
    for (int32_t o = 0; o < n_orb && eligible; ++o)
      eligible = (g->off_orb[o] % 2 == 0) && (g->ext_ld[o] % 2 == 0);
    using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    EncodeFn encode = nullptr;
    if (eligible) {
      void* fn = nullptr;
      cudaDriverEntryPointQueryResult q{};
      if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                           &q) == cudaSuccess &&
          q == cudaDriverEntryPointSuccess && fn)
        encode = reinterpret_cast<EncodeFn>(fn);
      cudaGetLastError();
    }
    if (encode) {
      std::vector<CUtensorMap> maps(2 * (size_t)n_orb);
      std::memset(maps.data(), 0, maps.size() * sizeof(CUtensorMap));
      bool ok = true;
      for (int32_t o = 0; o < n_orb && ok; ++o) {
        if (g->ext_pao[o] <= 0 || g->ext_ld[o] <= 0) continue;   // orbital without pairs
        const cuuint64_t dims[2] = {(cuuint64_t)g->ext_ld[o], (cuuint64_t)g->ext_pao[o]};
        const cuuint64_t strides[1] = {(cuuint64_t)g->ext_ld[o] * sizeof(double)};
        const cuuint32_t box[2] = {128, 1};
        const cuuint32_t estr[2] = {1, 1};
        const double* bases[2] = {g->Bg + g->off_orb[o], g->Bf + g->off_orb[o]};
        for (int q2 = 0; q2 < 2 && ok; ++q2)
          ok = encode(&maps[2 * o + q2], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
                      const_cast<double*>(bases[q2]), dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
               CUDA_SUCCESS;
      }
      if (ok && grow(c->d_tmaps, c->cap_tmaps, maps.size() * sizeof(CUtensorMap)) == cudaSuccess) {
        PF12_CUDA(c, cudaMemcpyAsync(c->d_tmaps, maps.data(), maps.size() * sizeof(CUtensorMap),
                                     cudaMemcpyHostToDevice, c->stream));
        c->use_tma = true;
      }
      cudaGetLastError();
    }
    c->gather = true;
    c->n_orb = n_orb;
    c->g_Bg = g->Bg;
    c->g_Bf = g->Bf;
    c->g_len_pm = t->len_pm;
    c->g_len_orb = g->len_orb;
  }
  PF12_CUDA(c, cudaStreamSynchronize(c->stream));
  c->uploaded = true;
  return PF12_OK;
}

int pf12_upload_pairs(pf12_ctx* c, int32_t n_orb, const int8_t* kind, int64_t n_pairs,
                      const int32_t* pi, const int32_t* pj, const int32_t* n_pao,
                      const int32_t* n_pno, const int32_t* n_aux, const pf12_tensors* t) {
  return upload_impl(c, n_orb, kind, n_pairs, pi, pj, n_pao, n_pno, n_aux, t, nullptr);
}

int pf12_upload_pairs_gather(pf12_ctx* c, int32_t n_orb, const int8_t* kind, int64_t n_pairs,
                             const int32_t* pi, const int32_t* pj, const int32_t* n_pao,
                             const int32_t* n_pno, const int32_t* n_aux,
                             const pf12_gather_tensors* g) {
  if (!g) return fail(c, PF12_ERR_INVALID_ARG, "null gather tensors");
  return upload_impl(c, n_orb, kind, n_pairs, pi, pj, n_pao, n_pno, n_aux, nullptr, g);
}

}  // extern "C"

namespace {

// Longest wait for an input group's arrival flag (short under the test hook).
uint64_t arrival_timeout(const pf12_ctx* c) {
  return c->debug_wait_polls ? 2000000ull : 60000000000ull;
}

// Queue order of the persistent launch: longest pair first (ties in list
// order); with streamed inputs group by group, longest first within a group,
// plus the group of every queue slot.
int apply_queue_order(pf12_ctx* c) {
  const int64_t n = c->n_pairs;
  std::vector<int32_t> group(n, 0);
  if (c->arr_ready)
    for (int64_t P = 0, g = 0; P < n; ++P) {
      while (P >= c->arr_end[g]) ++g;
      group[P] = (int32_t)g;
    }
  std::vector<int64_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    if (group[a] != group[b]) return group[a] < group[b];
    return c->h_cost[a] > c->h_cost[b];
  });
  std::vector<PairDesc> sorted(n);
  std::vector<int32_t> slot_group(n);
  for (int64_t q = 0; q < n; ++q) {
    sorted[q] = c->h_desc[order[q]];
    slot_group[q] = group[order[q]];
  }
  PF12_CUDA(c, grow(c->d_slot_group, c->cap_sg, (size_t)n));
  // pageable sources: both copies have consumed the vectors when they return
  PF12_CUDA(c, cudaMemcpyAsync(c->d_desc, sorted.data(), sizeof(PairDesc) * n,
                               cudaMemcpyHostToDevice, c->stream));
  PF12_CUDA(c, cudaMemcpyAsync(c->d_slot_group, slot_group.data(), sizeof(int32_t) * n,
                               cudaMemcpyHostToDevice, c->stream));
  c->arr_dirty = false;
  return PF12_OK;
}

// Autotuner: time every forward variant on the cost-spread sample of this pair
// list (one warm-up launch on a single pair, then one timed launch) and keep
// the fastest; the tensor-core variant only when it wins by 2 %.  Results are cached per (GPU, precision, size signature) in the optional
// tuner_cache file, one "key variant ms0 ms1 ms2" line per entry.
int tune(pf12_ctx* c) {
  if (c->forced >= 0) {
    if (c->n_ctas_v[c->forced] <= 0)
      return fail(c, PF12_ERR_UNSUPPORTED, "forced variant not available for this precision");
    c->variant = c->forced;
    return PF12_OK;
  }
  if (!c->tuner_cache.empty()) {
    FILE* f = fopen(c->tuner_cache.c_str(), "r");
    if (f) {
      char line[1024], key[512];
      int v = -1;
      while (fgets(line, sizeof line, f))
        if (sscanf(line, "%511s %d", key, &v) == 2 && c->tune_key == key && v >= 0 &&
            v < pf12::kFwdVariants && c->n_ctas_v[v] > 0)
          c->variant = v;
      fclose(f);
    }
    if (c->variant >= 0) return PF12_OK;
  }
  // small lists: one wave of CTAs at most, nothing to tune
  if (c->n_pairs <= c->n_ctas_v[0] || c->n_sample == 0) {
    c->variant = 0;
    return PF12_OK;
  }
  if (c->arr_ready)   // streamed inputs: the sample spans every group: wait for all of them
    PF12_CUDA(c, pf12::launch_wait_ready(c->arr_ready, (int32_t)c->arr_end.size(), c->arr_epoch,
                                         arrival_timeout(c), c->d_counter + 2, c->stream));
  pf12::FwdParams f = fwd_params(c);
  f.desc = c->d_desc_sample;
  int best = -1;
  for (int v = 0; v < pf12::kFwdVariants; ++v) {
    c->tune_ms[v] = 0.0;
    if (c->n_ctas_v[v] <= 0) continue;
    f.n_pairs = 1;
    PF12_CUDA(c, cudaMemsetAsync(c->d_counter, 0, sizeof(int32_t), c->stream));
    PF12_CUDA(c, pf12::launch_forward(f, c->precision, v, 1, c->stream));
    // median of three timed launches on the sample: one launch's tail varies
    // by about 2 % from run to run, as much as the variants differ
    f.n_pairs = c->n_sample;
    float t[3];
    for (int r = 0; r < 3; ++r) {
      PF12_CUDA(c, cudaMemsetAsync(c->d_counter, 0, sizeof(int32_t), c->stream));
      PF12_CUDA(c, cudaEventRecord(c->ev[0], c->stream));
      PF12_CUDA(c, pf12::launch_forward(f, c->precision, v, c->n_ctas_v[v], c->stream));
      PF12_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
      PF12_CUDA(c, cudaEventSynchronize(c->ev[1]));
      PF12_CUDA(c, cudaEventElapsedTime(&t[r], c->ev[0], c->ev[1]));
    }
    std::sort(t, t + 3);
    const float ms = t[1];
    c->tune_ms[v] = ms;
    // the tensor-core variant rounds its operands to split TF32 and carries the
    // larger error (about 10x the SIMT FP32 path's): it has to win by 2 %
    const float need = v == 2 ? 0.98f : 1.0f;
    if (best < 0 || ms < need * c->tune_ms[best]) best = v;
  }
  c->variant = best < 0 ? 0 : best;
  if (!c->tuner_cache.empty()) {
    FILE* fo = fopen(c->tuner_cache.c_str(), "a");
    if (fo) {
      fprintf(fo, "%s %d", c->tune_key.c_str(), c->variant);
      for (int v = 0; v < pf12::kFwdVariants; ++v) fprintf(fo, " %.3f", c->tune_ms[v]);
      fprintf(fo, "\n");
      fclose(fo);
    }
  }
  return PF12_OK;
}

}  // namespace

namespace {

// ------------------------------------------------------------------ full mode

pf12::FullParams full_params(pf12_ctx* c) {
  pf12::FullParams f{};
  const pf12_full_tensors& t = c->ft;
  f.Agi = t.Ag_i;
  f.Agj = t.Ag_j;
  f.Afi = t.Af_i;
  f.Afj = t.Af_j;
  f.Ari = t.Ar_i;
  f.Arj = t.Ar_j;
  f.AgiF = t.AgF_i;
  f.AgjF = t.AgF_j;
  f.AriF = t.ArF_i;
  f.ArjF = t.ArF_j;
  f.Jg = t.Jg;
  f.Jf = t.Jf;
  f.Jr = t.Jr;
  f.Q = t.Q;
  f.T = t.T;
  f.Fv = t.Fv;
  f.S = t.S;
  f.B = t.B;
  f.desc = c->d_fdesc;
  f.n_pairs = c->n_pairs;
  f.e_pair = c->d_epair;
  f.terms = c->d_terms;
  f.status = c->d_status;
  f.work = c->d_work;
  f.ws_stride = c->ws_stride;
  f.counter = c->d_counter;
  return f;
}

// Algorithmic work of one full-mode pair: FP64 (factorisation + solves on the
// 4p + 4 right-hand sides) and the mixable products, in the kernel's order.
void full_work(double p, double k, double m, double& f64, double& fmix) {
  const double k2 = k + 2;
  f64 = m * m * m / 3.0 + 2.0 * (4.0 * p + 4.0) * m * m;
  fmix = 4 * 2 * p * k * m + 2 * k2 * m * m + 2 * 2 * k2 * k2 * m   // V kernel, projected
         + 2 * 2 * p * m * m + 6 * 2 * p * p * m                     // geminal kernels
         + 4 * 2 * p * p * k + 6 * 2 * p * k * k                     // projections, C, R_Q
         + 2 * k * k * k2 * m + 2 * k * k2 * k2 * m                  // projector term
         + 2 * 2 * p * p * p;                                        // F R_Q, R_Q F
}

int tune_full(pf12_ctx* c) {
  if (c->forced >= 0) {
    if (c->forced >= pf12::kFullVariants || c->n_ctas_full_v[c->forced] <= 0)
      return fail(c, PF12_ERR_UNSUPPORTED, "forced variant not available in full mode");
    c->variant = c->forced;
    return PF12_OK;
  }
  if (c->n_pairs <= c->n_ctas_full_v[0] || c->n_sample == 0) {
    c->variant = 0;
    return PF12_OK;
  }
  pf12::FullParams f = full_params(c);
  f.desc = c->d_fdesc_sample;
  int best = 0;
  for (int v = 0; v < pf12::kFullVariants; ++v) {
    if (c->n_ctas_full_v[v] <= 0) continue;
    f.n_pairs = 1;
    PF12_CUDA(c, cudaMemsetAsync(c->d_counter, 0, sizeof(int32_t), c->stream));
    PF12_CUDA(c, pf12::launch_full(f, c->precision, v, 1, c->stream));
    f.n_pairs = c->n_sample;
    float ms = 0;
    PF12_CUDA(c, cudaMemsetAsync(c->d_counter, 0, sizeof(int32_t), c->stream));
    PF12_CUDA(c, cudaEventRecord(c->ev[0], c->stream));
    PF12_CUDA(c, pf12::launch_full(f, c->precision, v, c->n_ctas_full_v[v], c->stream));
    PF12_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
    PF12_CUDA(c, cudaEventSynchronize(c->ev[1]));
    PF12_CUDA(c, cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
    c->tune_ms[v] = ms;
    if (ms < c->tune_ms[best]) best = v;
  }
  c->variant = best;
  return PF12_OK;
}

int fit_full(pf12_ctx* c) {
  if (c->variant < 0) {
    const int rc = tune_full(c);
    if (rc != PF12_OK) return rc;
    c->n_ctas = c->n_ctas_full_v[c->variant];
  }
  if (!c->graph_exec) {
    PF12_CUDA(c, cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemsetAsync(c->d_counter, 0, sizeof(int32_t), c->capture_stream);
    if (e == cudaSuccess)
      e = pf12::launch_full(full_params(c), c->precision, c->variant, c->n_ctas, c->capture_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->capture_stream, &g);
    if (e != cudaSuccess) return cuda_fail(c, e, "capture full launch");
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "end capture");
    c->graph = g;
    PF12_CUDA(c, cudaGraphInstantiate(&c->graph_exec, g, 0));
  }
  PF12_CUDA(c, cudaEventRecord(c->ev[0], c->stream));
  PF12_CUDA(c, cudaGraphLaunch(c->graph_exec, c->stream));
  PF12_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
  c->t_fit = true;
  c->fitted = true;
  return PF12_OK;
}

}  // namespace

extern "C" {

int pf12_upload_full(pf12_ctx* c, int32_t n_orb, const int8_t* kind, int64_t n_pairs,
                     const int32_t* pi, const int32_t* pj, const int32_t* n_pao,
                     const int32_t* n_pno, const int32_t* n_aux, const pf12_full_tensors* t) {
  NvtxRange nvtx("pf12_upload_full");
  if (!c) return PF12_ERR_INVALID_ARG;
  free_pairs(c);
  if (n_pairs < 0 || n_orb < 0) return fail(c, PF12_ERR_INVALID_ARG, "negative count");
  if (c->augment || c->packed)
    return fail(c, PF12_ERR_UNSUPPORTED, "full mode takes plain PNO spaces and full metrics");
  if (n_pairs > 0 && (!kind || !pi || !pj || !n_pao || !n_pno || !n_aux || !t))
    return fail(c, PF12_ERR_INVALID_ARG, "null metadata pointer");
  if (n_pairs > 0) {
    const double* ptrs[18] = {t->Ag_i, t->Ag_j, t->Af_i, t->Af_j, t->Ar_i, t->Ar_j,
                              t->AgF_i, t->AgF_j, t->ArF_i, t->ArF_j, t->Jg, t->Jf, t->Jr,
                              t->Q, t->T, t->Fv, t->S, t->B};
    for (const double* q : ptrs)
      if (!q || !aligned16(q)) return fail(c, PF12_ERR_INVALID_ARG, "tensor pointer null or not 16-byte aligned");
    if (!t->off_pm || !t->off_mm || !t->off_pk || !t->off_kk || !t->off_pp || !t->off_s || !t->off_b)
      return fail(c, PF12_ERR_INVALID_ARG, "null offset array");
  }
  for (int32_t o = 0; o < n_orb; ++o)
    if (kind[o] != 0 && kind[o] != 1) return fail(c, PF12_ERR_INVALID_ARG, "orb_kind must be 0 or 1");
  std::vector<pf12::FullDesc> desc(n_pairs);
  std::vector<double> cost(n_pairs);
  double f64 = 0, fmix = 0, bytes = 0;
  int64_t max_ws = 0;
  for (int64_t P = 0; P < n_pairs; ++P) {
    const int32_t i = pi[P], j = pj[P], p = n_pao[P], k = n_pno[P], m = n_aux[P];
    char buf[160];
    if (i < 0 || j < 0 || i >= n_orb || j >= n_orb || i > j) {
      snprintf(buf, sizeof buf, "pair %lld: need 0 <= i <= j < n_orb", (long long)P);
      return fail(c, PF12_ERR_INVALID_ARG, buf);
    }
    if (p < 1 || k < 1 || m < 1 || k > p || m > pf12::kMaxAux || k > pf12::kMaxPno) {
      snprintf(buf, sizeof buf, "pair %lld: sizes p=%d k=%d m=%d out of range", (long long)P, p, k, m);
      return fail(c, PF12_ERR_INVALID_ARG, buf);
    }
    const int64_t offs[7] = {t->off_pm[P], t->off_mm[P], t->off_pk[P], t->off_kk[P],
                             t->off_pp[P], t->off_s[P], t->off_b[P]};
    const int64_t sizes[7] = {(int64_t)(p + 2) * m, (int64_t)m * m, (int64_t)p * k,
                              (int64_t)k * k, (int64_t)p * p, 2 * (int64_t)k,
                              (int64_t)k * m * (k + 2)};
    const int64_t lens[7] = {t->len_pm, t->len_mm, t->len_pk, t->len_kk, t->len_pp, t->len_s,
                             t->len_b};
    for (int q = 0; q < 7; ++q)
      if (offs[q] < 0 || (offs[q] & 1) || offs[q] + sizes[q] > lens[q]) {
        snprintf(buf, sizeof buf, "pair %lld: offset %d misaligned or block outside its buffer", (long long)P, q);
        return fail(c, PF12_ERR_INVALID_ARG, buf);
      }
    pf12::FullDesc& d = desc[P];
    d.off_pm = offs[0];
    d.off_mm = offs[1];
    d.off_pk = offs[2];
    d.off_kk = offs[3];
    d.off_pp = offs[4];
    d.off_s = offs[5];
    d.off_b = offs[6];
    d.p = p;
    d.k = k;
    d.m = m;
    d.pair = (int32_t)P;
    const int bi = kind[i] == 0, bj = kind[j] == 0;
    if (i == j) {
      d.n_ab = (int8_t)bi;
      d.n_aa = d.n_bb = 0;
    } else {
      d.n_ab = (int8_t)(bi + bj);
      d.n_aa = 1;
      d.n_bb = (int8_t)(bi * bj);
    }
    double c64, cmix;
    full_work(p, k, m, c64, cmix);
    cost[P] = c64 + cmix / 8.0;
    f64 += c64;
    fmix += cmix;
    bytes += 8.0 * (10.0 * (p + 2) * m + 3.0 * m * m + (double)p * k + (double)k * k +
                    (double)p * p + 2.0 * k + (double)k * m * (k + 2));
    max_ws = std::max(max_ws, pf12::full_slab(p, k, m).total);
  }
  std::vector<int64_t> order(n_pairs);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return cost[a] > cost[b]; });
  std::vector<pf12::FullDesc> sorted(n_pairs);
  for (int64_t q = 0; q < n_pairs; ++q) sorted[q] = desc[order[q]];
  const int64_t stride = (max_ws + 31) / 32 * 32;
  int64_t cap = INT64_MAX;
  if (c->ws_cap) {
    cap = (int64_t)(c->ws_cap / 8) / std::max<int64_t>(stride, 1);
    if (n_pairs > 0 && cap < 1) return fail(c, PF12_ERR_OOM, "workspace_bytes too small for the largest pair");
  }
  int64_t want = 1;
  for (int v = 0; v < pf12::kFullVariants; ++v) {
    const int bps = pf12::full_blocks_per_sm(c->precision, v);
    cudaGetLastError();
    int64_t n_v = std::min<int64_t>(n_pairs, (int64_t)std::max(bps, 0) * c->n_sm);
    n_v = bps <= 0 ? 0 : std::max<int64_t>(1, std::min(n_v, cap));
    c->n_ctas_full_v[v] = (int)n_v;
    want = std::max(want, n_v);
  }
  std::vector<pf12::FullDesc> sample;
  const int64_t n_s = std::min<int64_t>(n_pairs, 4 * want);
  for (int64_t q = 0; q < n_s; ++q) sample.push_back(sorted[(q * n_pairs) / std::max<int64_t>(n_s, 1)]);
  const size_t n = (size_t)std::max<int64_t>(n_pairs, 1);
  cudaError_t e = grow(c->d_fdesc, c->cap_fdesc, n);
  if (e == cudaSuccess) e = grow(c->d_fdesc_sample, c->cap_fsample, (size_t)std::max<int64_t>(n_s, 1));
  if (e == cudaSuccess) e = grow(c->d_epair, c->cap_ep, 3 * n);
  if (e == cudaSuccess) e = grow(c->d_terms, c->cap_terms, (size_t)pf12::kFullTerms * n);
  if (e == cudaSuccess) e = grow(c->d_status, c->cap_st, n);
  if (e == cudaSuccess && !c->fixed_allocated) {
    e = cudaMalloc(&c->d_out3, sizeof(double) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_counter, sizeof(int32_t) * 4);
    if (e == cudaSuccess) c->fixed_allocated = true;
  }
  if (e == cudaSuccess && n_pairs > 0) e = grow(c->d_work, c->cap_work, (size_t)(want * stride));
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_pairs(c);
    return fail(c, e == cudaErrorMemoryAllocation ? PF12_ERR_OOM : PF12_ERR_CUDA,
                std::string("device allocation: ") + cudaGetErrorString(e));
  }
  if (n_pairs > 0) {
    PF12_CUDA(c, cudaMemcpyAsync(c->d_fdesc, sorted.data(), sizeof(pf12::FullDesc) * n_pairs,
                                 cudaMemcpyHostToDevice, c->stream));
    PF12_CUDA(c, cudaMemcpyAsync(c->d_fdesc_sample, sample.data(), sizeof(pf12::FullDesc) * n_s,
                                 cudaMemcpyHostToDevice, c->stream));
  }
  PF12_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(int32_t) * n, c->stream));
  PF12_CUDA(c, cudaMemsetAsync(c->d_counter, 0, sizeof(int32_t) * 4, c->stream));
  PF12_CUDA(c, cudaMemsetAsync(c->d_epair, 0, sizeof(double) * 3 * n, c->stream));
  PF12_CUDA(c, cudaStreamSynchronize(c->stream));
  c->ft = *t;
  c->full = true;
  c->tune_key = "full";     // a later amplitude-only upload never reuses this tuning
  c->n_pairs = n_pairs;
  c->n_sample = n_s;
  c->ws_stride = stride;
  c->work_bytes = sizeof(double) * (size_t)(want * stride);
  c->flops64 = f64 + (c->precision == PF12_FP64 ? fmix : 0.0);
  c->flops_mix = fmix;
  c->bytes_in = bytes;
  c->n_ctas = c->n_ctas_full_v[0];
  for (int v = 0; v < pf12::kFwdVariants; ++v) c->n_ctas_v[v] = v < pf12::kFullVariants ? c->n_ctas_full_v[v] : 0;
  c->uploaded = true;
  return PF12_OK;
}

int pf12_full_terms(pf12_ctx* c, double* terms_dev) {
  if (!c || !terms_dev) return fail(c, PF12_ERR_INVALID_ARG, "null argument");
  if (!c->full) return fail(c, PF12_ERR_INVALID_ARG, "pf12_full_terms needs pf12_upload_full");
  if (!c->fitted) return fail(c, PF12_ERR_INVALID_ARG, "pf12_full_terms before pf12_fit");
  if (c->n_pairs == 0) return PF12_OK;
  PF12_CUDA(c, cudaMemcpyAsync(terms_dev, c->d_terms, sizeof(double) * pf12::kFullTerms * c->n_pairs,
                               cudaMemcpyDeviceToDevice, c->stream));
  return PF12_OK;
}

int pf12_set_arrival(pf12_ctx* c, int32_t n_groups, const int64_t* group_end,
                     const uint32_t* ready_dev, uint32_t epoch) {
  if (!c) return PF12_ERR_INVALID_ARG;
  if (!c->uploaded) return fail(c, PF12_ERR_INVALID_ARG, "pf12_set_arrival before pf12_upload_pairs");
  if (c->full) return fail(c, PF12_ERR_UNSUPPORTED, "streamed inputs are not offered in full mode");
  if (n_groups == 0 || c->n_pairs == 0) {
    const bool was = c->arr_ready != nullptr;
    c->arr_ready = nullptr;
    c->arr_end.clear();
    return was ? apply_queue_order(c) : PF12_OK;   // back to the plain cost order
  }
  if (c->gather) return fail(c, PF12_ERR_UNSUPPORTED, "streamed inputs are available in packed mode only");
  if (n_groups < 0 || !group_end || !ready_dev || (reinterpret_cast<uintptr_t>(ready_dev) & 3u))
    return fail(c, PF12_ERR_INVALID_ARG, "n_groups < 0, null group_end, or null / unaligned ready flags");
  for (int32_t g = 0; g < n_groups; ++g)
    if (group_end[g] <= (g ? group_end[g - 1] : 0) || group_end[g] > c->n_pairs)
      return fail(c, PF12_ERR_INVALID_ARG, "group_end must increase strictly within (0, n_pairs]");
  if (group_end[n_groups - 1] != c->n_pairs)
    return fail(c, PF12_ERR_INVALID_ARG, "the last group must end at n_pairs");
  std::vector<int64_t> ends(group_end, group_end + n_groups);
  const bool reorder = !c->arr_ready || ends != c->arr_end || c->arr_dirty;
  c->arr_end = ends;
  c->arr_ready = ready_dev;
  c->arr_epoch = epoch;
  // reorder now, before the caller issues its copies: the descriptor copies
  // come from pageable memory and would otherwise queue behind them
  return reorder ? apply_queue_order(c) : PF12_OK;
}

int pf12_fit(pf12_ctx* c) {
  NvtxRange nvtx("pf12_fit");
  if (!c) return PF12_ERR_INVALID_ARG;
  if (!c->uploaded) return fail(c, PF12_ERR_INVALID_ARG, "pf12_fit before pf12_upload_pairs");
  if (c->n_pairs == 0) {
    c->fitted = true;
    return PF12_OK;
  }
  if (c->full) return fit_full(c);
  if (c->arr_dirty) {
    const int rc = apply_queue_order(c);
    if (rc != PF12_OK) return rc;
  }
  const uint64_t arrival_timeout_ns = arrival_timeout(c);
  if (c->variant < 0) {
    const int rc = tune(c);
    if (rc != PF12_OK) return rc;
    c->n_ctas = c->n_ctas_v[c->variant];
  }
  if (c->arr_ready) {
    // streamed inputs: direct launch (the epoch changes from call to call)
    pf12::FwdParams f = fwd_params(c);
    f.ready = c->arr_ready;
    f.slot_group = c->d_slot_group;
    f.epoch = c->arr_epoch;
    f.arrival_timeout_ns = arrival_timeout_ns;
    PF12_CUDA(c, cudaEventRecord(c->ev[0], c->stream));
    PF12_CUDA(c, cudaMemsetAsync(c->d_counter, 0, sizeof(int32_t), c->stream));
    PF12_CUDA(c, pf12::launch_forward(f, c->precision, c->variant, c->n_ctas, c->stream));
    PF12_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
    c->t_fit = true;
    c->fitted = true;
    return PF12_OK;
  }
  if (!c->graph_exec) {
    // capture on the library's own stream (nothing executes), replay on the caller's
    PF12_CUDA(c, cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemsetAsync(c->d_counter, 0, sizeof(int32_t), c->capture_stream);
    if (e == cudaSuccess)
      e = pf12::launch_forward(fwd_params(c), c->precision, c->variant, c->n_ctas, c->capture_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->capture_stream, &g);
    if (e != cudaSuccess) return cuda_fail(c, e, "capture forward");
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "end capture");
    c->graph = g;
    PF12_CUDA(c, cudaGraphInstantiate(&c->graph_exec, g, 0));
  }
  PF12_CUDA(c, cudaEventRecord(c->ev[0], c->stream));
  PF12_CUDA(c, cudaGraphLaunch(c->graph_exec, c->stream));
  PF12_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
  c->t_fit = true;
  c->fitted = true;
  return PF12_OK;
}

int pf12_build_v(pf12_ctx* c, double* V_dev) {
  if (!c || !V_dev) return fail(c, PF12_ERR_INVALID_ARG, "null argument");
  if (c->full) return fail(c, PF12_ERR_UNSUPPORTED, "full mode keeps no V (use pf12_full_terms)");
  if (!c->fitted) return fail(c, PF12_ERR_INVALID_ARG, "pf12_build_v before pf12_fit");
  if (c->n_pairs == 0) return PF12_OK;
  for (int64_t P = 0; P < c->n_pairs; ++P) {
    const size_t kk = (size_t)c->pk[P] * c->pk[P];
    // one copy per pair keeps the caller's padding untouched
    PF12_CUDA(c, cudaMemcpyAsync(V_dev + c->off_kk[P], c->d_V + c->off_kk[P], kk * sizeof(double),
                                 cudaMemcpyDeviceToDevice, c->stream));
  }
  return PF12_OK;
}

int pf12_energy(pf12_ctx* c, double* e_pair_dev, double* E_host) {
  NvtxRange nvtx("pf12_energy");
  if (!c) return PF12_ERR_INVALID_ARG;
  if (!c->fitted) return fail(c, PF12_ERR_INVALID_ARG, "pf12_energy before pf12_fit");
  if (c->n_pairs == 0) {
    if (E_host) *E_host = 0.0;
    return PF12_OK;
  }
  PF12_CUDA(c, cudaEventRecord(c->ev[2], c->stream));
  PF12_CUDA(c, pf12::launch_energy_total(c->d_epair, c->d_status, c->n_pairs, c->d_counter + 2,
                                         c->d_out3, c->stream));
  PF12_CUDA(c, cudaEventRecord(c->ev[3], c->stream));
  c->t_energy = true;
  if (e_pair_dev)
    PF12_CUDA(c, cudaMemcpyAsync(e_pair_dev, c->d_epair, sizeof(double) * 3 * c->n_pairs,
                                 cudaMemcpyDeviceToDevice, c->stream));
  if (!E_host) return PF12_OK;
  double out3[4];
  PF12_CUDA(c, cudaMemcpyAsync(out3, c->d_out3, sizeof out3, cudaMemcpyDeviceToHost, c->stream));
  PF12_CUDA(c, cudaStreamSynchronize(c->stream));
  *E_host = out3[0];
  if (out3[3] != 0.0) {
    *E_host = std::nan("");
    return fail(c, PF12_ERR_TIMEOUT,
                "a bounded device wait expired (tensor-core or TMA barrier, or input arrival); "
                "pairs after it were not evaluated; upload again before the next fit");
  }
  if (out3[1] > 0) {
    char buf[128];
    snprintf(buf, sizeof buf, "%lld pair(s) failed, first pair %lld", (long long)out3[1], (long long)out3[2]);
    c->err = buf;
    int32_t st = 0;
    PF12_CUDA(c, cudaMemcpy(&st, c->d_status + (int64_t)out3[2], sizeof st, cudaMemcpyDeviceToHost));
    return st == PF12_PAIR_NOT_SPD ? PF12_ERR_NOT_SPD : PF12_ERR_NONFINITE;
  }
  if (!std::isfinite(out3[0])) return fail(c, PF12_ERR_NONFINITE, "total energy not finite");
  return PF12_OK;
}

}  // extern "C"

namespace {

// Adjoint tuner: like the forward tuner, on the same cost-spread sample (the
// sample's gradient blocks are overwritten by the real launch that follows).
// The choice is kept across uploads with the same size signature and cached
// in the tuner_cache file under the forward key plus "|bwd"; without that, a
// streamed run re-timed the adjoint on every batch (C-quartet lattice: 140 s
// per forward + adjoint step instead of about 90 s).
int tune_backward(pf12_ctx* c, pf12::BwdParams b) {
  if (c->n_pairs <= c->n_ctas_bwd_v[0] || c->n_sample == 0) {
    c->bwd_variant = 0;
    return PF12_OK;
  }
  const std::string key = c->tune_key + "|bwd";
  if (!c->tuner_cache.empty()) {     // same file as the forward tuner, own key
    FILE* f = fopen(c->tuner_cache.c_str(), "r");
    if (f) {
      char line[1024], k[512];
      int v = -1;
      while (fgets(line, sizeof line, f))
        if (sscanf(line, "%511s %d", k, &v) == 2 && key == k && v >= 0 && v < pf12::kBwdVariants &&
            c->n_ctas_bwd_v[v] > 0)
          c->bwd_variant = v;
      fclose(f);
    }
    if (c->bwd_variant >= 0) return PF12_OK;
  }
  b.f.desc = c->d_desc_sample;
  int best = 0;
  for (int v = 0; v < pf12::kBwdVariants; ++v) {
    b.f.n_pairs = 1;
    PF12_CUDA(c, cudaMemsetAsync(c->d_counter + 1, 0, sizeof(int32_t), c->stream));
    PF12_CUDA(c, pf12::launch_backward(b, c->precision, v, 1, c->stream));
    b.f.n_pairs = c->n_sample;
    PF12_CUDA(c, cudaMemsetAsync(c->d_counter + 1, 0, sizeof(int32_t), c->stream));
    PF12_CUDA(c, cudaEventRecord(c->ev[4], c->stream));
    PF12_CUDA(c, pf12::launch_backward(b, c->precision, v, c->n_ctas_bwd_v[v], c->stream));
    PF12_CUDA(c, cudaEventRecord(c->ev[5], c->stream));
    PF12_CUDA(c, cudaEventSynchronize(c->ev[5]));
    float ms = 0;
    PF12_CUDA(c, cudaEventElapsedTime(&ms, c->ev[4], c->ev[5]));
    c->tune_bwd_ms[v] = ms;
    if (ms < c->tune_bwd_ms[best]) best = v;
  }
  c->bwd_variant = best;
  if (!c->tuner_cache.empty()) {
    FILE* fo = fopen(c->tuner_cache.c_str(), "a");
    if (fo) {
      fprintf(fo, "%s %d %.3f %.3f 0\n", key.c_str(), best, c->tune_bwd_ms[0], c->tune_bwd_ms[1]);
      fclose(fo);
    }
  }
  return PF12_OK;
}

}  // namespace

extern "C" {

int pf12_backward(pf12_ctx* c, double dE, double* dAgi, double* dAgj, double* dAfi, double* dAfj,
                  double* dQ, double* dT) {
  NvtxRange nvtx("pf12_backward");
  if (!c) return PF12_ERR_INVALID_ARG;
  if (c->full) return fail(c, PF12_ERR_UNSUPPORTED, "no adjoint of the full pair energy");
  if (!c->uploaded) return fail(c, PF12_ERR_INVALID_ARG, "pf12_backward before pf12_upload_pairs");
  if (c->gather) return fail(c, PF12_ERR_INVALID_ARG, "gather mode: use pf12_backward_gather");
  if (c->n_pairs == 0) return PF12_OK;
  pf12::BwdParams b{};
  b.f = fwd_params(c);
  b.f.work = c->d_work;
  b.f.ws_stride = c->ws_stride_bwd;
  b.dE = dE;
  b.dAgi = dAgi;
  b.dAgj = dAgj;
  b.dAfi = dAfi;
  b.dAfj = dAfj;
  b.dQ = dQ;
  b.dT = dT;
  const void* outs[6] = {dAgi, dAgj, dAfi, dAfj, dQ, dT};
  for (const void* p : outs)
    if (p && !aligned16(p)) return fail(c, PF12_ERR_INVALID_ARG, "gradient pointer not 16-byte aligned");
  if (c->bwd_variant < 0) {
    const int rc = tune_backward(c, b);
    if (rc != PF12_OK) return rc;
  }
  PF12_CUDA(c, cudaEventRecord(c->ev[4], c->stream));
  PF12_CUDA(c, cudaMemsetAsync(c->d_counter + 1, 0, sizeof(int32_t), c->stream));
  PF12_CUDA(c, pf12::launch_backward(b, c->precision, c->bwd_variant, c->n_ctas_bwd_v[c->bwd_variant],
                                     c->stream));
  PF12_CUDA(c, cudaEventRecord(c->ev[5], c->stream));
  c->t_bwd = true;
  return PF12_OK;
}

int pf12_backward_gather(pf12_ctx* c, double dE, double* dBg, double* dBf, double* dQ, double* dT) {
  NvtxRange nvtx("pf12_backward_gather");
  if (!c) return PF12_ERR_INVALID_ARG;
  if (c->full) return fail(c, PF12_ERR_UNSUPPORTED, "no adjoint of the full pair energy");
  if (!c->uploaded || !c->gather)
    return fail(c, PF12_ERR_INVALID_ARG, "pf12_backward_gather needs pf12_upload_pairs_gather");
  if (c->n_pairs == 0) return PF12_OK;
  const void* outs[4] = {dBg, dBf, dQ, dT};
  for (const void* p : outs)
    if (p && !aligned16(p)) return fail(c, PF12_ERR_INVALID_ARG, "gradient pointer not 16-byte aligned");
  const bool want_b = dBg || dBf;
  if (want_b) {
    cudaError_t e = grow(c->d_dA, c->cap_dA, 4 * (size_t)std::max<int64_t>(c->g_len_pm, 1));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(c, PF12_ERR_OOM, "per-pair gradient scratch");
    }
  }
  pf12::BwdParams b{};
  b.f = fwd_params(c);
  b.f.work = c->d_work;
  b.f.ws_stride = c->ws_stride_bwd;
  b.dE = dE;
  if (want_b) {
    b.dAgi = c->d_dA;
    b.dAgj = c->d_dA + c->g_len_pm;
    b.dAfi = c->d_dA + 2 * c->g_len_pm;
    b.dAfj = c->d_dA + 3 * c->g_len_pm;
  }
  b.dQ = dQ;
  b.dT = dT;
  if (c->bwd_variant < 0) {
    const int rc = tune_backward(c, b);
    if (rc != PF12_OK) return rc;
  }
  PF12_CUDA(c, cudaEventRecord(c->ev[4], c->stream));
  PF12_CUDA(c, cudaMemsetAsync(c->d_counter + 1, 0, sizeof(int32_t), c->stream));
  PF12_CUDA(c, pf12::launch_backward(b, c->precision, c->bwd_variant, c->n_ctas_bwd_v[c->bwd_variant],
                                     c->stream));
  if (want_b) {
    // both orbital gradients are produced; a NULL one goes to a throwaway copy
    double* gb = dBg;
    double* gf = dBf;
    double* tmp = nullptr;
    if (!gb || !gf) {
      PF12_CUDA(c, cudaMallocAsync(reinterpret_cast<void**>(&tmp), sizeof(double) * std::max<int64_t>(c->g_len_orb, 1), c->stream));
      if (!gb) gb = tmp;
      if (!gf) gf = tmp;
    }
    PF12_CUDA(c, cudaMemsetAsync(gb, 0, sizeof(double) * c->g_len_orb, c->stream));
    if (gf != gb) PF12_CUDA(c, cudaMemsetAsync(gf, 0, sizeof(double) * c->g_len_orb, c->stream));
    PF12_CUDA(c, pf12::launch_scatter(b.dAgi, b.dAgj, b.dAfi, b.dAfj, c->d_desc_by_pair, c->d_gdesc,
                                      c->d_map_pao, c->d_map_aux, c->d_orb_ptr, c->d_orb_list,
                                      c->d_off_orb, c->d_ld_orb, c->n_orb, gb, gf, c->stream));
    if (tmp) PF12_CUDA(c, cudaFreeAsync(tmp, c->stream));
  }
  PF12_CUDA(c, cudaEventRecord(c->ev[5], c->stream));
  c->t_bwd = true;
  return PF12_OK;
}

int pf12_pair_status(pf12_ctx* c, int32_t* status_host) {
  if (!c || !status_host) return fail(c, PF12_ERR_INVALID_ARG, "null argument");
  if (c->n_pairs == 0) return PF12_OK;
  PF12_CUDA(c, cudaMemcpyAsync(status_host, c->d_status, sizeof(int32_t) * c->n_pairs,
                               cudaMemcpyDeviceToHost, c->stream));
  PF12_CUDA(c, cudaStreamSynchronize(c->stream));
  return PF12_OK;
}

int pf12_stats(pf12_ctx* c, pf12_stats_t* s) {
  if (!c || !s) return fail(c, PF12_ERR_INVALID_ARG, "null argument");
  std::memset(s, 0, sizeof *s);
  PF12_CUDA(c, cudaStreamSynchronize(c->stream));
  float ms = 0;
  if (c->t_fit && cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]) == cudaSuccess) s->ms_fit = ms;
  if (c->t_energy && cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]) == cudaSuccess) s->ms_energy = ms;
  if (c->t_bwd && cudaEventElapsedTime(&ms, c->ev[4], c->ev[5]) == cudaSuccess) s->ms_backward = ms;
  cudaGetLastError();
  s->flops_fp64 = c->flops64;
  s->flops_mixed = c->flops_mix;
  s->bytes_in = c->bytes_in;
  s->n_pairs = c->n_pairs;
  s->n_ctas = c->n_ctas;
  s->launches_fit = c->n_pairs > 0 ? 1 : 0;
  s->tile_config = c->variant;
  for (int v = 0; v < pf12::kFwdVariants; ++v) {
    s->tune_ms[v] = c->tune_ms[v];
    s->ctas_variant[v] = c->n_ctas_v[v];
  }
  if (c->variant >= 0 && !c->full) {
    s->look_depth = pf12::kFwdLook[c->variant];
    s->ctas_per_sm = pf12::kFwdCtasPerSm[c->variant];
    s->tensor_cores = c->variant == 2;
  } else if (c->variant >= 0) {
    s->look_depth = 8;   // full mode: the default look-ahead
    s->ctas_per_sm = c->variant == 1 ? 3 : 2;
    s->tensor_cores = 0;
  }
  s->gemm_tile = pf12::kTile;
  s->gemm_k_chunk = pf12::kBK;
  s->panel_width = pf12::kNB;
  s->bwd_variant = c->bwd_variant;
  s->sieve_tma = c->gather && c->use_tma;
  for (int v = 0; v < 2; ++v) s->tune_bwd_ms[v] = c->tune_bwd_ms[v];
  s->graph_used = c->graph_exec != nullptr;
  return PF12_OK;
}

const char* pf12_last_error(const pf12_ctx* c) { return c ? c->err.c_str() : "null context"; }

void pf12_destroy(pf12_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  release_all(c);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  delete c;
}

}  // extern "C"
