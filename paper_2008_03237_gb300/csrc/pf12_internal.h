// Internal declarations shared by the host API and the kernel translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pf12 {

constexpr int kThreads = 256;   // threads per CTA of every pair kernel
constexpr int kTile = 64;       // output tile edge of the CTA GEMM
constexpr int kBK = 32;         // K chunk of the CTA GEMM
constexpr int kNB = 32;         // Cholesky / solve panel width
constexpr int kMaxAux = 4096;   // m limit (workspace and index arithmetic in int32)
constexpr int kMaxPno = 256;    // k limit

// One entry per pair, in the persistent kernel's (cost-sorted) order.
// SOMO-augmented pairs (s > 0): the factor blocks have p + s rows (the s SOMO
// rows last), Q is p x (k - s), and V, T are k x k with the SOMO virtuals last.
struct PairDesc {
  int64_t off_pm, off_mm, off_pk, off_kk;  // element offsets into the packed inputs
  int32_t p, k, m, pair;                   // PAO rows, virtual dimension, aux size, caller's index
  float w_alpha, w_beta;                   // E_P = w_alpha d + w_beta x (as FP64 below)
  int8_t n_ab, n_aa, n_bb;                 // spin-case multiplicities
  int8_t c1;                               // 1 if (i alpha, j beta) is occupied; c2 = n_ab - c1
  int32_t s;                               // SOMO rows / virtuals of the augmented space (0: none)
};
static_assert(sizeof(PairDesc) == 64, "PairDesc layout");

// Gather mode: where pair P's factors live inside the per-orbital blocks.
struct GatherDesc {
  int64_t off_i, off_j;      // element offsets of orbital i's and j's blocks
  int64_t map_pao, map_aux;  // offsets of the pair's 2p row / 2m column indices
  int32_t ld_i, ld_j;        // row strides of those blocks
  int32_t orb_i, orb_j;      // orbital indices (tensor-map lookup)
};

struct FwdParams {
  const double *Agi, *Agj, *Afi, *Afj, *Jg, *Jf, *Q, *T;
  const PairDesc* desc;
  int64_t n_pairs;
  double* V;          // ctx-owned, same layout as T
  double* e_pair;     // n_pairs x 3, indexed by the caller's pair index
  double* dx;         // n_pairs x 2 (d, x), caller's index
  int32_t* status;    // n_pairs, caller's index
  double* work;       // n_ctas * ws_stride doubles
  int64_t ws_stride;  // doubles per CTA
  int32_t* counter;   // work-queue head, zeroed before each launch
  int32_t* err;       // set when a bounded device wait expired (zeroed at upload)
  // gather mode (null in packed mode): A blocks are sieved from per-orbital blocks
  const GatherDesc* gdesc;   // indexed by the caller's pair index
  const double *Bg, *Bf;     // per-orbital extended blocks (Coulomb, F12)
  const int32_t *map_pao, *map_aux;
  // TMA tensor maps of the orbital blocks ([2o] Bg, [2o + 1] Bf, 128 bytes each,
  // box 128 columns x 1 row) or null: the sieve then uses plain loads
  const void* tmaps;
  // test hook: nonzero = issue no tensor-core / TMA work before the first
  // barrier wait and give that wait this many polls, so it expires
  uint32_t debug_wait_polls;
  // streamed inputs (ready == null: every input is resident before the
  // launch).  The pair in queue slot s belongs to arrival group slot_group[s];
  // a CTA reads that pair's inputs only after ready[group] has reached epoch
  // (written by the caller's copy stream after the group's copies), waiting at
  // most arrival_timeout_ns.
  const uint32_t* ready;
  const int32_t* slot_group;
  uint32_t epoch;
  uint64_t arrival_timeout_ns;
  // 1: J_g and J_f blocks are packed lower triangles (row r holds J[r][0..r]
  // at r (r + 1) / 2); J_f is unpacked into the slab before its product
  int32_t metric_packed;
};

struct BwdParams {
  FwdParams f;
  double dE;
  double *dAgi, *dAgj, *dAfi, *dAfj, *dQ, *dT;
};

// Complete pair energy (full mode): every term of E_(2)F12 per pair.  Factor
// blocks are (p + 2) x m (PAO rows, then the occupied i, j); see
// pf12_full_tensors in include/pairf12.h for the inputs.
struct FullDesc {
  int64_t off_pm, off_mm, off_pk, off_kk, off_pp, off_s, off_b;
  int32_t p, k, m, pair;
  int8_t n_ab, n_aa, n_bb, pad_;
  int32_t pad2_;
};
static_assert(sizeof(FullDesc) == 80, "FullDesc layout");

constexpr int kFullTerms = 14;   // spatial terms per pair (order of oracle TERM_NAMES)
constexpr int kFullChunk = 128;  // auxiliary functions per chunk of the projector term

struct FullParams {
  const double *Agi, *Agj, *Afi, *Afj, *Ari, *Arj, *AgiF, *AgjF, *AriF, *ArjF;
  const double *Jg, *Jf, *Jr, *Q, *T, *Fv, *S, *B;
  const FullDesc* desc;
  int64_t n_pairs;
  double* e_pair;     // n_pairs x 3, caller's index
  double* terms;      // n_pairs x kFullTerms, caller's index
  int32_t* status;    // n_pairs, caller's index
  double* work;       // n_ctas * ws_stride doubles
  int64_t ws_stride;
  int32_t* counter;   // work-queue head
};

// Slab of one full-mode pair (doubles): offsets of its regions, ld = m rounded
// up to 4, lq = p rounded up to 4.
struct FullSlab {
  int64_t M, W1, W2, Atfi, Atfj, Cti, Ctj, KR, KRiF, KRjF, RQ, S1, S2, Y, Zt, FvQ, Ft, U,
      Rpno, QtFQ, Cm, Vh, H, total;
};
inline __host__ __device__ int64_t slab_take(int64_t& o, int64_t n) {
  const int64_t at = o;
  o += (n + 31) / 32 * 32;   // every region starts on 256 bytes
  return at;
}
inline __host__ __device__ FullSlab full_slab(int p, int k, int m) {
  const int64_t ld = (m + 3) / 4 * 4, lq = (p + 3) / 4 * 4, k2 = k + 2;
  FullSlab s{};
  int64_t o = 0;
#define take(n) slab_take(o, (n))
  s.M = take((int64_t)(m + 4 * p + 4) * ld);
  s.W1 = take((int64_t)p * ld);
  s.W2 = take((int64_t)p * ld);
  s.Atfi = take(k2 * ld);
  s.Atfj = take(k2 * ld);
  s.Cti = take(k2 * ld);
  s.Ctj = take(k2 * ld);
  s.KR = take((int64_t)p * lq);
  s.KRiF = take((int64_t)p * lq);
  s.KRjF = take((int64_t)p * lq);
  s.RQ = take((int64_t)p * lq);
  s.S1 = take((int64_t)p * lq);
  s.S2 = take((int64_t)p * lq);
  s.Y = take((int64_t)p * k);
  s.Zt = take((int64_t)p * k);
  s.FvQ = take((int64_t)p * k);
  s.Ft = take((int64_t)p * k);
  s.U = take((int64_t)p * k);
  s.Rpno = take((int64_t)k * k);
  s.QtFQ = take((int64_t)k * k);
  s.Cm = take((int64_t)k * k);
  s.Vh = take(k2 * k2);
  s.H = take((int64_t)k * kFullChunk * k2);
#undef take
  s.total = o + 64;
  return s;
}

constexpr int kFullVariants = 2;   // 2 / 3 CTAs per SM
cudaError_t launch_full(const FullParams& prm, int precision, int variant, int n_ctas,
                        cudaStream_t s);
int full_blocks_per_sm(int precision, int variant);
cudaError_t launch_full_f64_2(const FullParams& prm, int n_ctas, cudaStream_t s);
cudaError_t launch_full_f64_3(const FullParams& prm, int n_ctas, cudaStream_t s);
cudaError_t launch_full_f32_2(const FullParams& prm, int n_ctas, cudaStream_t s);
cudaError_t launch_full_f32_3(const FullParams& prm, int n_ctas, cudaStream_t s);
int occupancy_full_f64_2();
int occupancy_full_f64_3();
int occupancy_full_f32_2();
int occupancy_full_f32_3();

// per-CTA workspace (doubles) for a pair of sizes (p, k, m), forward / backward
inline int64_t ld_of(int m) { return (int64_t)((m + 3) / 4 * 4); }
// offset of the sieved A blocks (4 x p x m) inside a forward slab
inline __host__ __device__ int64_t fwd_sieve_off(int k, int m) {
  const int64_t ld = (m + 3) / 4 * 4;
  return ((int64_t)(m + 2 * k) * ld + 2 * (int64_t)k * ld + 31) / 32 * 32;
}
// offset of the unpacked J_f (m x ld) inside a forward slab (packed metrics)
inline __host__ __device__ int64_t fwd_jf_off(int p, int k, int m, bool gather) {
  return fwd_sieve_off(k, m) + (gather ? (4 * (int64_t)p * m + 64 + 31) / 32 * 32 : 0);
}
inline int64_t fwd_ws(int p, int k, int m, bool gather = false, bool packed = false) {
  int64_t ld = ld_of(m);
  if (packed) return fwd_jf_off(p, k, m, gather) + (int64_t)m * ld + 64;
  return (int64_t)(m + 2 * k) * ld + 2 * (int64_t)k * ld + 64 +
         (gather ? 4 * (int64_t)p * m + 64 : 0);
}
inline __host__ __device__ int64_t bwd_sieve_off(int k, int m) {
  const int64_t ld = (m + 3) / 4 * 4, ldk = (k + 3) / 4 * 4;
  return ((int64_t)(m + 6 * k) * ld + 2 * (int64_t)k * ldk + 31) / 32 * 32;
}
inline __host__ __device__ int64_t bwd_jf_off(int p, int k, int m, bool gather) {
  return bwd_sieve_off(k, m) + (gather ? (4 * (int64_t)p * m + 64 + 31) / 32 * 32 : 0);
}
inline int64_t bwd_ws(int p, int k, int m, bool gather = false, bool packed = false) {
  int64_t ld = ld_of(m);
  int64_t ldk = (k + 3) / 4 * 4;
  if (packed) return bwd_jf_off(p, k, m, gather) + (int64_t)m * ld + 64;
  // M = [J_g -> L; Ct_i; Ct_j] (m + 2k rows), F (2k rows: At^f, then H),
  // R (2k rows: At^f - Ct J_f, then Z^T), G_V and V (k x k each)
  return (int64_t)(m + 6 * k) * ld + 2 * (int64_t)k * ldk + 64 +
         (gather ? 4 * (int64_t)p * m + 64 : 0);
}

// Per-variant launchers and occupancy queries (one translation unit each,
// csrc/inst/, compiled in parallel): f64 / f32 = product type, 2 / 3 = CTAs
// per SM, tc = tcgen05 split-TF32 contractions.
cudaError_t launch_fwd_f64_2(const FwdParams& prm, int n_ctas, cudaStream_t s);
cudaError_t launch_fwd_f64_3(const FwdParams& prm, int n_ctas, cudaStream_t s);
cudaError_t launch_fwd_f32_2(const FwdParams& prm, int n_ctas, cudaStream_t s);
cudaError_t launch_fwd_f32_3(const FwdParams& prm, int n_ctas, cudaStream_t s);
cudaError_t launch_fwd_tc_3(const FwdParams& prm, int n_ctas, cudaStream_t s);
cudaError_t launch_fwd_f64_3_l16(const FwdParams& prm, int n_ctas, cudaStream_t s);
cudaError_t launch_fwd_f32_3_l16(const FwdParams& prm, int n_ctas, cudaStream_t s);
int occupancy_fwd_f64_3_l16();
int occupancy_fwd_f32_3_l16();
int occupancy_fwd_f64_2();
int occupancy_fwd_f64_3();
int occupancy_fwd_f32_2();
int occupancy_fwd_f32_3();
int occupancy_fwd_tc_3();
cudaError_t launch_bwd_f64_2(const BwdParams& prm, int n_ctas, cudaStream_t s);
cudaError_t launch_bwd_f64_3(const BwdParams& prm, int n_ctas, cudaStream_t s);
cudaError_t launch_bwd_f32_2(const BwdParams& prm, int n_ctas, cudaStream_t s);
cudaError_t launch_bwd_f32_3(const BwdParams& prm, int n_ctas, cudaStream_t s);
int occupancy_bwd_f64_2();
int occupancy_bwd_f64_3();
int occupancy_bwd_f32_2();
int occupancy_bwd_f32_3();

// Forward variants (tile shapes) the autotuner chooses from:
//   0: SIMT, 2 CTAs/SM, look-ahead 8    1: SIMT, 3 CTAs/SM, look-ahead 8
//   2: tcgen05 contractions, 3 CTAs/SM, look-ahead 8 (mixed precision only)
//   3: SIMT, 3 CTAs/SM, look-ahead 16
constexpr int kFwdVariants = 4;
constexpr int kFwdLook[kFwdVariants] = {8, 8, 8, 16};
constexpr int kFwdCtasPerSm[kFwdVariants] = {2, 3, 3, 3};
cudaError_t launch_forward(const FwdParams& prm, int precision, int variant, int n_ctas,
                           cudaStream_t s);
constexpr int kBwdVariants = 2;
cudaError_t launch_backward(const BwdParams& prm, int precision, int variant, int n_ctas,
                            cudaStream_t s);
// One thread waits (bounded, per flag) until every ready[g], g < n_groups,
// has reached epoch; sets *err on expiry.
cudaError_t launch_wait_ready(const uint32_t* ready, int32_t n_groups, uint32_t epoch,
                              uint64_t timeout_ns, int32_t* err, cudaStream_t s);
cudaError_t launch_energy_total(const double* e_pair, const int32_t* status, int64_t n_pairs,
                                const int32_t* err, double* out3, cudaStream_t s);
int forward_blocks_per_sm(int precision, int variant);
// gather mode: adjoint scatter into per-orbital blocks (one CTA per orbital,
// pairs in list order)
cudaError_t launch_scatter(const double* dAgi, const double* dAgj, const double* dAfi,
                           const double* dAfj, const PairDesc* desc_by_pair, const GatherDesc* gdesc,
                           const int32_t* map_pao, const int32_t* map_aux, const int64_t* orb_ptr,
                           const int32_t* orb_list, const int64_t* off_orb, const int32_t* ld_orb,
                           int32_t n_orb, double* dBg, double* dBf, cudaStream_t s);
int backward_blocks_per_sm(int precision, int variant);

}  // namespace pf12
