/*
 * pairf12.h -- C ABI of the GB300 (sm_103a) pair-F12 library (libpairf12.so).
 *
 * What it computes (Kumar, Neese, Valeev, arXiv 2008.03237): for every F12
 * pair P = (i, j), i <= j, of localised occupied orbitals, the amplitude term
 * of the pair-specific F12 correction in the spin-independent PNO basis.
 *
 *   1. local DF with the pair's auxiliary metric (Sec. "F12 integral
 *      transformations": integrals of i and j are sieved onto the pair domain
 *      and recombined through local density fitting):
 *         J_g = L L^T (FP64 Cholesky),  C_x = A^g_x J_g^{-1},  x in {i, j}
 *   2. robust (Dunlap) fit of the F12 pair integral (Eq. V with the F12 kernel
 *      fitted from the Coulomb-metric coefficients):
 *         K = A^f_i C_j^T + C_i A^f_j^T - C_i J_f C_j^T       (p x p)
 *   3. PNO transform (Sec. "Pair-natural orbitals", "SOMO handling"):
 *         V = Q^T K Q                                          (k x k)
 *   4. amplitude contraction (term 1/2 V^{ij}_{ab} t^{ab}_{ij} of Eq. Vtilde):
 *         d = sum V_ab T_ab,  x = sum V_ab T_ba
 *   5. spin cases (Eqs. F12energy_sf*, ROHF rules after them):
 *         e_ab = n_ab (3d + x)/8, e_aa = n_aa (d - x)/4, e_bb = n_bb (d - x)/4
 *      with (n_ab, n_aa, n_bb) = DOMO-DOMO (2,1,1), (1,0,0) if i == j;
 *      SOMO-DOMO (1,1,0); SOMO-SOMO (0,1,0), (0,0,0) if i == j.
 *   6. E = sum of all pair energies, FP64, fixed order (deterministic).
 *
 * The device pipeline evaluates steps 1-3 in the exactly equivalent order
 * At = Q^T A (k x m), Ct = At^g J_g^{-1}, V = At^f_i Ct_j^T + Ct_i At^f_j^T -
 * (Ct_i J_f) Ct_j^T, so the FP64 solves run on k right-hand sides, not p.
 * The Cholesky factorisation, both triangular solves and all energy sums are
 * always FP64.  The projections and the J_f / V products follow `precision`.
 *
 * Conventions for every entry point
 *   - Return 0 on success or a negative PF12_ERR_* code; pf12_last_error()
 *     gives a message.  No call aborts the process.
 *   - Tensor arguments are caller-owned device buffers (float64, row-major)
 *     unless marked "host".  The library never frees them; they must stay
 *     valid until the next pf12_upload_pairs or pf12_destroy.
 *   - The library owns its workspace, pair metadata and CUDA graph.
 *   - Calls are ordered on the context's stream; only the calls that return
 *     host values (pf12_energy's E_host, pf12_pair_status, pf12_stats)
 *     synchronise that stream.
 */
#ifndef PAIRF12_H
#define PAIRF12_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PF12_OK 0
#define PF12_ERR_INVALID_ARG (-1) /* bad size, index, offset, null pointer, call order */
#define PF12_ERR_NOT_SPD (-2)     /* a pair's J_g has a pivot <= 0 (see pf12_pair_status) */
#define PF12_ERR_OOM (-3)         /* workspace allocation failed or exceeds workspace_bytes */
#define PF12_ERR_CUDA (-4)        /* a CUDA runtime call failed */
#define PF12_ERR_TIMEOUT (-5)     /* a bounded device wait ran out */
#define PF12_ERR_NONFINITE (-6)   /* a pair energy is NaN or Inf */
#define PF12_ERR_UNSUPPORTED (-7) /* option not built into this library */

/* per-pair status codes written by the device (pf12_pair_status) */
#define PF12_PAIR_OK 0
#define PF12_PAIR_NOT_SPD 1      /* Cholesky pivot <= 0 or not finite */
#define PF12_PAIR_NONFINITE 2    /* V or the pair energy is not finite */

/* Arithmetic of the projections (Q^T A) and of the J_f / V products.
 * FP64 Cholesky, solves and energy sums in every mode. */
typedef enum {
  PF12_FP64 = 0,       /* everything FP64 (plain mode) */
  PF12_MIXED_FP32 = 2  /* FP32-class products: FP32 FFMA summed in two levels (each
                          32-wide K chunk, then a running FP32 sum), widened to FP64
                          once per output; or, when the autotuner picks the
                          tensor-core variant, tcgen05 split-TF32 (hi + lo, 3 products)
                          for the projections and the J_f product, added into FP64
                          every 32 of K */
} pf12_precision;

typedef struct pf12_ctx pf12_ctx; /* opaque, library-owned */

typedef struct {
  int precision;           /* pf12_precision */
  void* cuda_stream;       /* cudaStream_t all work is ordered on; NULL = legacy stream */
  size_t workspace_bytes;  /* cap on library-owned device workspace; 0 = no cap */
  int deterministic;       /* reserved: energy sums are always fixed-order */
  const char* tuner_cache; /* path of the autotuner's cache file, or NULL (no cache) */
  int force_variant;       /* -1: autotune; else the forward variant to use (see
                              pf12_stats_t.tile_config); unavailable ones are refused */
  int sieve_plain;         /* gather mode: 1 = sieve with plain loads; 0 = TMA tile::gather4
                              loads when every orbital block starts and strides on 16 bytes */
  int debug_wait_timeout;  /* tests only, keep 0: the tensor-core and TMA paths issue no work
                              before their first barrier wait and poll it briefly, so the
                              bounded wait expires; the pair gets status 3 and pf12_energy
                              returns PF12_ERR_TIMEOUT with the context still usable */
  int augment_somo;        /* 1: SOMO-augmented PNO space (Sec. "SOMO handling"): every PAO
                              domain holds the n_s SOMOs of orb_kind and the PAO-to-PNO matrix
                              is blockdiag(Q, I_{n_s}).  Per pair, Ag/Af blocks are
                              (p + n_s) x m (SOMO rows last), Q stays p x k, T and V are
                              (k + n_s) x (k + n_s) (SOMO virtuals last).  Alpha virtuals are
                              the PNOs, beta virtuals the PNOs and SOMOs, and each spin case
                              sums over its own virtuals.  Packed mode only (gather mode:
                              PF12_ERR_UNSUPPORTED); k + n_s <= 256.  0: plain PNO space */
  int metric_packed;       /* 1: Jg and Jf blocks are packed lower triangles, m (m + 1) / 2
                              doubles at off_mm[P]: row r holds J[r][0..r] at r (r + 1) / 2.
                              The metrics are symmetric, so this halves their share of the
                              inputs (the bulk of them) in memory and in host-to-device
                              copies; the library unpacks J_f into its workspace (m x m per
                              CTA more).  0: full row-major m x m blocks */
} pf12_opts;

/* Packed ("plain mode") per-pair tensors.  Pair P's blocks start at element
 * offset off_xx[P] of the matching buffer:
 *   Ag_i, Ag_j, Af_i, Af_j : p x m   at off_pm[P]  (DF factors of orbital i / j,
 *                                                   Coulomb g and F12 f kernels)
 *   Jg, Jf                 : m x m   at off_mm[P]  (SPD auxiliary metrics; packed
 *                                                   lower triangles with metric_packed)
 *   Q                      : p x k   at off_pk[P]  (PAO -> PNO coefficients)
 *   T                      : k x k   at off_kk[P]  (PNO amplitudes t^{ab}_{ij})
 * Offsets are host arrays, element (not byte) offsets, multiples of 2 (16-byte
 * aligned), and each block must lie inside its buffer (len_xx elements).
 * Device pointers must be 16-byte aligned. */
typedef struct {
  const double* Ag_i;
  const double* Ag_j;
  const double* Af_i;
  const double* Af_j;
  const double* Jg;
  const double* Jf;
  const double* Q;
  const double* T;
  const int64_t* off_pm; /* host */
  const int64_t* off_mm; /* host */
  const int64_t* off_pk; /* host */
  const int64_t* off_kk; /* host */
  int64_t len_pm, len_mm, len_pk, len_kk;
} pf12_tensors;

typedef struct {
  double ms_fit;         /* device time of the last pf12_fit (CUDA events) */
  double ms_energy;      /* device time of the last pf12_energy reduction */
  double ms_backward;    /* device time of the last pf12_backward */
  double flops_fp64;     /* algorithmic FP64 flops of one forward pass: sum m^3/3 + 4 k m^2
                            (+ the mixable flops in PF12_FP64 mode) */
  double flops_mixed;    /* algorithmic flops of the mixable part: 8pkm + 2km^2 + 4k^2m */
  double bytes_in;       /* algorithmic input bytes of one forward pass */
  int64_t n_pairs;
  int32_t n_ctas;        /* persistent CTAs of the fused pair kernel */
  int32_t launches_fit;  /* kernels launched by one pf12_fit */
  int32_t tile_config;   /* autotuner choice: forward variant (0: SIMT, 2 CTAs/SM; 1: SIMT,
                            3 CTAs/SM; 2: tcgen05 tensor-core contractions, mixed mode only;
                            3: SIMT, 3 CTAs/SM, Cholesky look-ahead 16; full mode: 0 / 1 =
                            2 / 3 CTAs/SM); its tile shape is reported below */
  int32_t graph_used;    /* 1 when pf12_fit replays a captured CUDA graph */
  double tune_ms[4];     /* autotuner timings of the variants on its sample, median of three
                            launches (0 if not run or unavailable) */
  int32_t ctas_variant[4]; /* persistent CTAs each variant launches (0: unavailable) */
  int32_t bwd_variant;   /* adjoint variant (0: 2 CTAs/SM, 1: 3 CTAs/SM; -1 before tuning) */
  int32_t sieve_tma;     /* gather mode: 1 when the sieve uses TMA tile::gather4 loads */
  double tune_bwd_ms[2]; /* adjoint tuner timings */
  /* tile shape of the chosen forward variant */
  int32_t look_depth;    /* Cholesky panels per look-ahead group (deep update every 32 x this) */
  int32_t ctas_per_sm;   /* resident persistent CTAs per SM */
  int32_t tensor_cores;  /* 1: projections and the J_f product on tcgen05 */
  int32_t gemm_tile;     /* output tile edge of the CTA GEMM */
  int32_t gemm_k_chunk;  /* K chunk staged per step of the CTA GEMM */
  int32_t panel_width;   /* Cholesky / solve panel width */
} pf12_stats_t;

/* Create a context.  opts may be NULL (FP64, legacy stream, no cap). */
int pf12_create(pf12_ctx** ctx, const pf12_opts* opts);

/* Re-target the stream for subsequent calls (e.g. torch's current stream). */
int pf12_set_stream(pf12_ctx* ctx, void* cuda_stream);

/* Register the pair list and the packed tensors (Sec. "Pair-screenings": the
 * F12 pair list; Sec. "F12 integral transformations": the pair domains).
 *   n_orb, orb_kind (host, n_orb): 0 = DOMO, 1 = SOMO
 *   pi, pj (host, n_pairs): orbital indices, 0 <= pi <= pj < n_orb
 *   n_pao, n_pno, n_aux (host, n_pairs): p >= 1, 1 <= k <= p, m >= 1,
 *     m <= 4096, k <= 256
 *   t: packed tensors (see pf12_tensors)
 * Copies metadata to the device, orders pairs by cost for the persistent
 * kernel and sizes the workspace.  Invalidates any captured graph. */
int pf12_upload_pairs(pf12_ctx* ctx, int32_t n_orb, const int8_t* orb_kind, int64_t n_pairs,
                      const int32_t* pi, const int32_t* pj, const int32_t* n_pao,
                      const int32_t* n_pno, const int32_t* n_aux, const pf12_tensors* t);

/* Steps 1-4 for every pair in one persistent fused launch (replayed from a
 * captured CUDA graph after the first call): projections, FP64 Cholesky of
 * J_g, FP64 solves, robust fit to V (kept in the context), and the pair
 * contractions d, x.  A pair whose J_g is not SPD gets status NOT_SPD and NaN
 * energies; the call itself still returns 0 (query pf12_pair_status).
 * With streamed inputs (pf12_set_arrival) the launch is direct, not from the
 * graph. */
int pf12_fit(pf12_ctx* ctx);

/* Streamed inputs for the next pf12_fit calls: the fit may start before the
 * inputs have reached the device.  No counterpart in the paper, which streams
 * pair integrals from disk on the CPU; here the host-to-device copies of one
 * pair list overlap its single persistent launch, so copying and computing
 * run at the same time without a launch (and its tail) per batch.
 *   n_groups: number of arrival groups; 0 turns streaming off (the queue goes
 *     back to the plain cost order).
 *   group_end (host, n_groups): group g holds the pairs [group_end[g-1],
 *     group_end[g]) of the caller's list (group_end[-1] = 0); strictly
 *     increasing, last entry n_pairs.
 *   ready_dev (device, n_groups uint32, 4-byte aligned, caller-owned): the
 *     caller writes ready_dev[g] = epoch once every input block of group g's
 *     pairs is on the device, with a copy (cudaMemcpyAsync of 4 bytes) issued
 *     on the copy stream of that group's copies, after them (groups may use
 *     several streams and land in any order) -- not with a kernel, which
 *     could wait behind the persistent launch for a free SM.  Issue the copies
 *     before pf12_fit (or on a stream that runs concurrently with it), and
 *     after this call, which reorders the queue with small copies from
 *     pageable memory on the context's stream.
 *   epoch: the value that marks this call's data (change it every call, e.g.
 *     a counter; comparison is wrap-safe).
 * The queue is ordered group by group (longest pair first within a group);
 * a CTA waits for a group's flag before its first pair of that group, at most
 * 60 s (2 ms under pf12_opts.debug_wait_timeout); on expiry the pair gets
 * status 3, the launch stops taking pairs and pf12_energy returns
 * PF12_ERR_TIMEOUT (upload again before the next fit).  A context that still
 * has to time its variants first waits for every group (expiry: the same
 * error, with no pair evaluated).  Packed mode only
 * (gather mode: PF12_ERR_UNSUPPORTED).  A new pf12_upload_pairs clears the
 * setting; pf12_backward does not wait (call it after the fit). */
int pf12_set_arrival(pf12_ctx* ctx, int32_t n_groups, const int64_t* group_end,
                     const uint32_t* ready_dev, uint32_t epoch);

/* Copy V^{ij} of every pair (k x k, row-major) into V_dev at the pair's off_kk
 * offset (same layout as T).  Requires a previous pf12_fit. */
int pf12_build_v(pf12_ctx* ctx, double* V_dev);

/* Step 5-6: spin-case pair energies and the total.
 *   e_pair_dev (device, n_pairs x 3, may be NULL): (e_ab, e_aa, e_bb) per pair
 *   E_host (host, may be NULL): the FP64 total, summed in a fixed order
 * Returns PF12_ERR_NOT_SPD / PF12_ERR_NONFINITE when any pair failed (E_host
 * is then NaN).  Requires a previous pf12_fit. */
int pf12_energy(pf12_ctx* ctx, double* e_pair_dev, double* E_host);

/* Adjoint of dE * E with respect to the DF factors, PNO coefficients and
 * amplitudes (J_g, J_f are constants).  Recomputes the forward intermediates
 * pair by pair instead of storing them.  Outputs use the input layouts
 * (off_pm / off_pk / off_kk) and are overwritten (not accumulated); any output
 * pointer may be NULL to skip it.  A pair whose J_g is not SPD gets status
 * NOT_SPD (pf12_pair_status) and all-zero gradient blocks.  Formulas, with alpha, beta the weights of
 * E_P = alpha d + beta x:
 *   G_V = alpha T + beta T^T,   dT = alpha V + beta V^T
 *   dAf_i = Q G_V Ct_j,  dAf_j = Q G_V^T Ct_i
 *   dAg_i = Q G_V Z_j^T, dAg_j = Q G_V^T Z_i^T, Z_x^T = (At^f_x - Ct_x J_f) J_g^{-1}
 *   dQ = (Af_i Ct_j^T + Ag_i Z_j) G_V^T + (Af_j Ct_i^T + Ag_j Z_i) G_V */
int pf12_backward(pf12_ctx* ctx, double dE, double* dAg_i, double* dAg_j, double* dAf_i,
                  double* dAf_j, double* dQ, double* dT);

/* Per-pair status (host, n_pairs) of the last pf12_fit / pf12_backward. */
int pf12_pair_status(pf12_ctx* ctx, int32_t* status_host);

/* Timers, flop and byte counts of the last calls. */
int pf12_stats(pf12_ctx* ctx, pf12_stats_t* out);

/* Message of the last error on this context (never NULL). */
const char* pf12_last_error(const pf12_ctx* ctx);

/* Release the context's workspace, graph and metadata. */
void pf12_destroy(pf12_ctx* ctx);

/* Gather mode ("pair-extended SparseMaps", Sec. "F12 integral
 * transformations"): the three-index factors exist once per occupied orbital
 * o on its pair-extended domain (PAOs of all pairs of o x auxiliary functions
 * of all pairs of o), and every pair sieves its rows and columns out of the
 * blocks of i and j on the device.  J_g, J_f, Q, T stay packed per pair.
 *   Bg, Bf (device): per-orbital blocks, orbital o at element offset
 *     off_orb[o], P_o rows x ld_o columns (row-major, ld_o >= M_o), 16-byte
 *     aligned base; len_orb elements in each buffer
 *   off_orb, ext_pao (P_o), ext_aux (M_o), ext_ld (ld_o): host, n_orb
 *   map_pao (host): per pair 2p row indices, first into orbital i's block,
 *     then into j's, each run strictly increasing; pair P's at off_map_pao[P]
 *   map_aux (host): per pair 2m column indices, same convention
 * The library copies the maps to the device.  Gradients come back per orbital
 * block through pf12_backward_gather. */
typedef struct {
  const double* Bg;
  const double* Bf;
  const int64_t* off_orb;
  const int32_t* ext_pao;
  const int32_t* ext_aux;
  const int32_t* ext_ld;
  int64_t len_orb;
  const int32_t* map_pao;
  const int32_t* map_aux;
  const int64_t* off_map_pao;
  const int64_t* off_map_aux;
  int64_t len_map_pao, len_map_aux;
  const double* Jg;
  const double* Jf;
  const double* Q;
  const double* T;
  const int64_t* off_mm;
  const int64_t* off_pk;
  const int64_t* off_kk;
  int64_t len_mm, len_pk, len_kk;
} pf12_gather_tensors;

/* As pf12_upload_pairs, with the factors given in gather mode. */
int pf12_upload_pairs_gather(pf12_ctx* ctx, int32_t n_orb, const int8_t* orb_kind,
                             int64_t n_pairs, const int32_t* pi, const int32_t* pj,
                             const int32_t* n_pao, const int32_t* n_pno, const int32_t* n_aux,
                             const pf12_gather_tensors* g);

/* Adjoint in gather mode: per-pair factor gradients (computed as in
 * pf12_backward) are summed into the per-orbital blocks dBg, dBf (layout of
 * Bg, Bf; overwritten) in pair-list order, so the result is deterministic.
 * dQ, dT as in pf12_backward.  Any pointer may be NULL to skip it. */
int pf12_backward_gather(pf12_ctx* ctx, double dE, double* dBg, double* dBf, double* dQ,
                         double* dT);

/* ------------------------------------------------------------------------
 * Complete pair energy ("full mode"): every term of E_(2)F12 = sum_{i<j}
 * 2 Vt^{ij}_{ij} + B~^{ij}_{ij} (Eq. F12 energy), per pair:
 *   Vt (Eq. Vtilde)  occupied block V^{ij}_{ij}, amplitude term 1/2 V_ab t^ab,
 *                    Fock-coupling term 1/2 C_ab t^ab (Eq. C) and the singles
 *                    terms V^{ij}_{i a_j} t^{a_j}_j + V^{ij}_{a_i j} t^{a_i}_i
 *   V  (Eq. V)       robust fit of the V kernel with the Q_ij projector
 *                    (Eq. Qij): the part of the geminal on PNO pairs removed
 *                    through the PNO-pair factors
 *   B~ (Eqs. B, X, Btilde, XAppr)  B - X^{i j_F} - X^{i_F j} with the
 *                    Fock-transformed occupied orbitals (pair decoupling)
 * then the spin-adapted energies (Eqs. F12energy_sf*).  The pair's PAO
 * domain (orthonormal) stands in for the complete virtual space of the sums in
 * Eqs. C, B and X, so the fit runs in the PAO domain: FP64 solves on 4p + 4
 * right-hand sides (the PAOs and i, j for both orbitals, and the PAOs for i_F
 * and j_F).  In spatial terms, per pair,
 *   Vt_d = 1/2 (Vh[i,j] + <Vh,T> + Vh[i,s_j] + Vh[s_i,j]) + <C,T>
 *   Vt_x = 1/2 (Vh[j,i] + <Vh,T^T> + Vh[j,s_i] + Vh[s_j,i]) + <C,T^T>
 *   B~_dd = tr(R F R^T) + tr(R^T F R) - <K_jF, R> - <K_iF, R>
 *   B~_dx = 2 tr(R F R) - <K_jF, R^T> - <K_iF, R^T>
 *   e_ab = n_ab (3/4 Vt_d + 1/4 Vt_x + (10 B~_dd + 6 B~_dx)/64)
 *   e_aa = n_aa (1/2 (Vt_d - Vt_x) + (B~_dd - B~_dx)/16),  e_bb likewise
 * with R the projected geminal over the PAO domain, F the virtual Fock block,
 * Vh the projected V over the PNOs and i, j, and C = Ft^T K Q + Q^T K Ft,
 * Ft = (1 - Q Q^T) F Q.
 *
 * Per-pair tensors, pair P's blocks at element offset off_xx[P] (multiples of
 * 2) of the matching buffer, all float64 row-major:
 *   Ag_i .. ArF_j : (p + 2) x m at off_pm.  Rows 0..p-1 are the PAOs; rows p
 *        and p + 1 are the occupied orbitals i and j as bra functions, used
 *        by Ag_*, Af_* only (row p + 1 of the i blocks equals row p of the j
 *        blocks: (ij|X)).  Ag: Coulomb factors; Af: V-kernel factors; Ar:
 *        geminal factors; AgF_*, ArF_*: the same for the Fock-transformed
 *        occupied orbitals i_F, j_F
 *   Jg, Jf, Jr    : m x m at off_mm (SPD metrics of the three operators)
 *   Q : p x k at off_pk;  T : k x k at off_kk
 *   Fv : p x p at off_pp (Fock matrix over the PAO domain, symmetric)
 *   S  : 2 x k at off_s (singles amplitudes of i, then j, in the pair's PNOs)
 *   B  : k x m x (k + 2) at off_b: B[c][X][q] = (c q|X) contracted with the
 *        Coulomb metric's inverse square root, q over the PNOs, then i, then j
 * Limits: 1 <= k <= p, m <= 4096, k <= 256.
 * Gather mode, SOMO augmentation, packed metrics, streamed inputs, V output
 * and the adjoint are not offered in full mode (PF12_ERR_UNSUPPORTED). */
typedef struct {
  const double* Ag_i;
  const double* Ag_j;
  const double* Af_i;
  const double* Af_j;
  const double* Ar_i;
  const double* Ar_j;
  const double* AgF_i;
  const double* AgF_j;
  const double* ArF_i;
  const double* ArF_j;
  const double* Jg;
  const double* Jf;
  const double* Jr;
  const double* Q;
  const double* T;
  const double* Fv;
  const double* S;
  const double* B;
  const int64_t* off_pm; /* host */
  const int64_t* off_mm; /* host */
  const int64_t* off_pk; /* host */
  const int64_t* off_kk; /* host */
  const int64_t* off_pp; /* host */
  const int64_t* off_s;  /* host */
  const int64_t* off_b;  /* host */
  int64_t len_pm, len_mm, len_pk, len_kk, len_pp, len_s, len_b;
} pf12_full_tensors;

#define PF12_FULL_TERMS 14 /* per-pair spatial terms written by pf12_full_terms */

/* Register a pair list for the complete pair energy (arguments as
 * pf12_upload_pairs, tensors as above).  pf12_fit then evaluates every term
 * for every pair in one persistent launch and pf12_energy returns the
 * spin-case pair energies and the total as in the amplitude-only mode. */
int pf12_upload_full(pf12_ctx* ctx, int32_t n_orb, const int8_t* orb_kind, int64_t n_pairs,
                     const int32_t* pi, const int32_t* pj, const int32_t* n_pao,
                     const int32_t* n_pno, const int32_t* n_aux, const pf12_full_tensors* t);

/* Full mode: copy the per-pair spatial terms of the last pf12_fit into
 * terms_dev (device, n_pairs x PF12_FULL_TERMS, caller's pair order):
 *   0 Vh[i,j]  1 Vh[j,i]  2 <Vh,T>  3 <Vh,T^T>  4 singles (direct)
 *   5 singles (exchange)  6 <C,T>  7 <C,T^T>  8 B_dd  9 B_dx
 *   10 <K_jF,R>  11 <K_jF,R^T>  12 <K_iF,R>  13 <K_iF,R^T> */
int pf12_full_terms(pf12_ctx* ctx, double* terms_dev);

/* Allocation-free forward pass: steps 1-6 for every pair in one call, with
 * no cudaMalloc, cudaFree or other allocating call.  The paper has no
 * counterpart; this entry point exists for callers that cannot allocate
 * device memory themselves or through the library (code running inside a
 * memory pool or arena it does not own, plugins whose host program owns
 * every device allocation, callers just refused more memory).
 *   Scratch: a fixed 64 MiB file-scope device array inside the library,
 *     held by every GPU that loads it until the process exits.  One call
 *     needs 84 B per pair of metadata (+ 1 KiB) plus one Cholesky/solve slab of
 *     8 ((m + 2k) ld + 2k ld + 64) bytes (ld = m rounded up to 4) for the
 *     largest pair; sizes beyond that return PF12_ERR_INVALID_ARG.  The
 *     number of concurrent pairs is whatever number of slabs fits (at most
 *     2 per SM), pairs are taken in the caller's order.
 *   Set-up: the first call on each device looks up the array's device
 *     address (cudaGetSymbolAddress) with that device current.
 *   Not capturable: every call copies pair descriptors from host stack
 *     memory, synchronises the stream and reads the total back, none of
 *     which a stream capture can hold; on a capturing stream the call
 *     returns PF12_ERR_UNSUPPORTED before any other CUDA call, so the
 *     caller's capture stays valid.
 *   Sharing: every call uses the same array and leaves the last call's
 *     contents in it; calls whose GPU work overlaps (other streams or host
 *     threads) race on it and must be serialised by the caller.
 *   Arguments as pf12_upload_pairs plus: precision (pf12_precision), stream
 *   (cudaStream_t, NULL = legacy stream), V_dev (device, len_kk doubles, out:
 *   V in the T layout), e_pair_dev (device, n_pairs x 3, out), E_host (host,
 *   out, may be NULL).  Synchronises the stream.  Returns as pf12_energy. */
int pf12_energy_noalloc(int32_t n_orb, const int8_t* orb_kind, int64_t n_pairs, const int32_t* pi,
                        const int32_t* pj, const int32_t* n_pao, const int32_t* n_pno,
                        const int32_t* n_aux, const pf12_tensors* t, int32_t precision,
                        void* cuda_stream, double* V_dev, double* e_pair_dev, double* E_host);

#ifdef __cplusplus
}
#endif
#endif /* PAIRF12_H */
