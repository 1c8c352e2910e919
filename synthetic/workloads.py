"""Seeded synthetic workloads for the pair-F12 path: pair lists, per-pair domain
sizes and per-pair input tensors.

Nothing here computes any part of the F12 method; it only draws inputs.  The
oracle, the tests and the benchmark all take their inputs from this module (and
from its CUDA twin, synthetic/csrc/synth_gen.cu, for full-size device fills).

Shapes follow the paper's workloads as stand-ins (no molecule, basis set or
integral code is used):

* pairs (i <= j) of localised occupied orbitals, DOMOs first and SOMOs last
  (a chain-end radical, Sec. "SOMO handling"), kept by a distance cutoff like the
  F12 pair subset of Sec. "Pair-screenings";
* per pair a PAO domain of size p, an auxiliary (local DF) domain of size m and
  k PNOs (Sec. "Orbital domains", "Pair-natural orbitals");
* DF factors A^g_i, A^g_j, A^f_i, A^f_j (p x m), auxiliary metrics J_g, J_f
  (m x m, SPD, X X^T + 0.1 I), orthonormal PNO coefficients Q (p x k) and
  amplitudes T (k x k).

Every random number is a Philox4x32-10 word keyed by (seed, pair, tensor id,
element); Gaussians are Irwin-Hall sums of four uniform integers, so every
value is an exact integer times one FP64 constant and host and device produce
identical bits.  Q alone is orthonormalised on the host (numpy QR) and uploaded.
"""
from dataclasses import dataclass, field
import json
import math
import os

import numpy as np

from .philox import philox4x32

SEED_BASE = 20080323
KEY_HI = 0x50463132  # second Philox key word, fixed

# Philox counter word c3: which tensor of the pair is being drawn
TID_SIZES, TID_AGI, TID_AGJ, TID_AFI, TID_AFJ, TID_XG, TID_XF, TID_Q, TID_T = range(9)

# exp(-0.3) rounded to FP64, written as a literal so that every platform starts
# the decay powers from the same bits.
EXP_M03 = 0.7408182206817179

# Irwin-Hall constants.  Sum of four uniform 16-bit integers: mean 131070,
# variance 4 (2^32 - 1) / 12.  Sum of four uniform 4-bit integers: mean 30,
# variance 4 (16^2 - 1) / 12 = 85.
IH16_MEAN = 131070
IH16_VAR = 4.0 * (65536.0 * 65536.0 - 1.0) / 12.0
IH16_INV_STD = 1.0 / math.sqrt(IH16_VAR)
IH4_MEAN = 30
IH4_VAR = 85.0

METRIC_SHIFT = 0.1      # J = X X^T + 0.1 I
T_STD = 1e-2            # amplitudes ~ N(0, (1e-2)^2)
ALIGN = 32              # every packed block starts on a multiple of 32 doubles (256 B)


@dataclass
class Workload:
    name: str
    seed: int
    n_domo: int
    n_somo: int
    orb_kind: np.ndarray      # int8, 0 = DOMO, 1 = SOMO, per orbital
    pi: np.ndarray            # int32, pair list, pi <= pj
    pj: np.ndarray
    n_pao: np.ndarray         # int32 per pair (p)
    n_pno: np.ndarray         # int32 per pair (k)
    n_aux: np.ndarray         # int32 per pair (m)
    decay: np.ndarray         # float64 per pair, s_P scaling all four DF factors
    metric_shift: float = METRIC_SHIFT
    meta: dict = field(default_factory=dict)
    somo_aug: int = 0         # SOMO-augmented PNO space: SOMO rows / virtuals per pair

    @property
    def n_orb(self):
        return self.n_domo + self.n_somo

    @property
    def n_pairs(self):
        return int(self.pi.shape[0])

    def subset(self, idx, name=None):
        """Workload restricted to the pairs in idx (keeps each pair's seed keys)."""
        idx = np.asarray(idx, dtype=np.int64)
        w = Workload(name or self.name + "[sub]", self.seed, self.n_domo, self.n_somo,
                     self.orb_kind, self.pi[idx], self.pj[idx], self.n_pao[idx],
                     self.n_pno[idx], self.n_aux[idx], self.decay[idx],
                     self.metric_shift, dict(self.meta), self.somo_aug)
        base = self.meta.get("pair_key", np.arange(self.n_pairs, dtype=np.int64))
        w.meta["pair_key"] = np.asarray(base)[idx]
        return w

    def augmented(self):
        """The same pair list in the SOMO-augmented PNO space (Sec. "SOMO
        handling"): every pair's factors gain the n_somo SOMO rows (drawn as
        rows p .. p + n_s - 1 of the same Philox stream, so rows 0 .. p - 1 are
        unchanged) and its amplitudes become (k + n_s) square."""
        return Workload(self.name + "[somo-aug]", self.seed, self.n_domo, self.n_somo,
                        self.orb_kind, self.pi, self.pj, self.n_pao, self.n_pno, self.n_aux,
                        self.decay, self.metric_shift, dict(self.meta), int(self.n_somo))

    @property
    def n_rows(self):
        """Rows of each pair's factor blocks: p, plus the SOMOs when augmented."""
        return self.n_pao.astype(np.int64) + self.somo_aug

    @property
    def n_virt(self):
        """Virtual dimension of V and T per pair: k, plus the SOMOs when augmented."""
        return self.n_pno.astype(np.int64) + self.somo_aug

    def pair_key(self, P):
        """Philox counter word that identifies pair P (its index in the full list)."""
        keys = self.meta.get("pair_key")
        return int(P) if keys is None else int(keys[P])


# --------------------------------------------------------------------------
# scalar draws


def _uniform_int(word, lo, hi):
    """Map a uint32 word onto [lo, hi] (multiply-shift)."""
    span = np.uint64(hi - lo + 1)
    return lo + int((np.uint64(word) * span) >> np.uint64(32))


def _ih16(w_a, w_b):
    """Irwin-Hall integer from two uint32 words (four 16-bit uniforms), centred."""
    w_a = np.asarray(w_a, dtype=np.int64)
    w_b = np.asarray(w_b, dtype=np.int64)
    s = (w_a & 0xFFFF) + (w_a >> 16) + (w_b & 0xFFFF) + (w_b >> 16)
    return s - IH16_MEAN


def _decay_power(d):
    s = 1.0
    for _ in range(int(d)):
        s = s * EXP_M03
    return s


# --------------------------------------------------------------------------
# workloads


def _chain_pairs(n_orb, cutoff):
    pi, pj = [], []
    for i in range(n_orb):
        for j in range(i, n_orb):
            if cutoff is None or j - i <= cutoff:
                pi.append(i)
                pj.append(j)
    return np.array(pi, np.int32), np.array(pj, np.int32)


def _lattice_points(n_points, side):
    c = (side - 1) / 2.0
    pts = [(x, y, z) for x in range(side) for y in range(side) for z in range(side)]
    pts.sort(key=lambda q: ((q[0] - c) ** 2 + (q[1] - c) ** 2 + (q[2] - c) ** 2, q))
    return pts[:n_points]


def _draw_sizes(seed, n_pairs, pao, pno, aux, keys=None):
    """Per-pair (p, k, m).  pao/aux: (lo, hi) uniform; pno: ("uniform", lo, hi) or
    ("lognormal", median, sigma, lo, hi)."""
    keys = np.arange(n_pairs, dtype=np.int64) if keys is None else keys
    w0, w1, w2, w3 = philox4x32(0, 0, keys, TID_SIZES, seed, KEY_HI)
    p = np.empty(n_pairs, np.int32)
    k = np.empty(n_pairs, np.int32)
    m = np.empty(n_pairs, np.int32)
    for P in range(n_pairs):
        m[P] = _uniform_int(w0[P], aux[0], aux[1])
        p[P] = _uniform_int(w1[P], pao[0], pao[1])
        if pno[0] == "uniform":
            kk = _uniform_int(w2[P], pno[1], pno[2])
        else:
            _, med, sig, lo, hi = pno
            z = float(_ih16(w2[P], w3[P])) * IH16_INV_STD
            kk = int(round(math.exp(math.log(med) + sig * z)))
            kk = max(lo, min(hi, kk))
        k[P] = min(kk, p[P])
    return p, k, m


def make_chain(name, n_domo, n_somo, cutoff, pao, pno, aux, seed):
    n_orb = n_domo + n_somo
    kind = np.zeros(n_orb, np.int8)
    kind[n_domo:] = 1                     # SOMOs are the last orbitals (chain end)
    pi, pj = _chain_pairs(n_orb, cutoff)
    p, k, m = _draw_sizes(seed, len(pi), pao, pno, aux)
    decay = np.array([_decay_power(j - i) for i, j in zip(pi, pj)], np.float64)
    return Workload(name, seed, n_domo, n_somo, kind, pi, pj, p, k, m, decay)


def make_lattice(name, n_domo, n_somo, side, r_cut, pao, pno, aux, seed):
    n_orb = n_domo + n_somo
    pts = np.array(_lattice_points(n_orb, side), np.float64)
    # SOMOs: the points closest to the centre are the first entries; move them last
    order = list(range(n_somo, n_orb)) + list(range(n_somo))
    pts = pts[order]
    kind = np.zeros(n_orb, np.int8)
    kind[n_domo:] = 1
    pi, pj, dist = [], [], []
    for i in range(n_orb):
        d = np.sqrt(((pts[i:] - pts[i]) ** 2).sum(axis=1))
        for jj in np.nonzero(d <= r_cut + 1e-12)[0]:
            pi.append(i)
            pj.append(i + int(jj))
            dist.append(float(d[jj]))
    pi = np.array(pi, np.int32)
    pj = np.array(pj, np.int32)
    p, k, m = _draw_sizes(seed, len(pi), pao, pno, aux)
    decay = np.array([math.exp(-0.3 * r) for r in dist], np.float64)
    return Workload(name, seed, n_domo, n_somo, kind, pi, pj, p, k, m, decay)


CONFIG_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "configs")


def from_config(name_or_path):
    """Workload described by a JSON file of configs/ (by name) or at a path:
    kind "chain" (n_domo, n_somo, cutoff) or "lattice" (n_domo, n_somo, side,
    r_cut), size ranges pao, pno, aux, and seed SEED_BASE + seed_offset."""
    path = name_or_path
    if os.path.sep not in path and not path.endswith(".json"):
        path = os.path.join(CONFIG_DIR, path + ".json")
    with open(path) as fh:
        c = json.load(fh)
    pno = tuple(c["pno"])
    seed = SEED_BASE + int(c["seed_offset"])
    if c["kind"] == "chain":
        return make_chain(c["label"], c["n_domo"], c["n_somo"], c["cutoff"], tuple(c["pao"]), pno,
                          tuple(c["aux"]), seed)
    if c["kind"] == "lattice":
        return make_lattice(c["label"], c["n_domo"], c["n_somo"], c["side"], c["r_cut"],
                            tuple(c["pao"]), pno, tuple(c["aux"]), seed)
    raise ValueError(f"unknown workload kind {c['kind']!r} in {path}")


def tiny():
    """7 DOMO + 1 SOMO, all 36 pairs, p = 30, k ~ U[8,16], m ~ U[60,120] (configs/tiny.json)."""
    return from_config("tiny")


def c40h81():
    """C40H81-radical chain: 120 DOMO + 1 SOMO, |i-j| <= 25 (2,821 unique pairs; configs/c40h81.json)."""
    return from_config("c40h81")


def c160h321():
    """C160H321-radical chain: 480 DOMO + 1 SOMO, |i-j| <= 30 (14,446 unique pairs;
    configs/c160h321.json)."""
    return from_config("c160h321")


def lattice_quartet():
    """700 DOMO + 3 SOMO on a 9x9x9 lattice, distance cutoff 3.0 (29,226 unique pairs;
    configs/lattice703.json)."""
    return from_config("lattice703")


def custom(n_domo, n_somo, cutoff, pao, pno, aux, seed=SEED_BASE + 100, name="custom"):
    """Chain workload with caller-chosen size ranges (tests: several tiles + ragged tails)."""
    return make_chain(name, n_domo, n_somo, cutoff, pao, pno, aux, seed)


WORKLOADS = {"tiny": tiny, "c40h81": c40h81, "c160h321": c160h321,
             "lattice703": lattice_quartet}


# --------------------------------------------------------------------------
# per-pair tensors


def _gauss16(seed, key, tid, n, c):
    """n Gaussian-like draws, value = fl(z * c) with z an Irwin-Hall integer.

    Element e uses words (2 (e % 2), 2 (e % 2) + 1) of Philox call e // 2."""
    e = np.arange(n, dtype=np.int64)
    w = philox4x32(e >> 1, 0, key, tid, seed, KEY_HI)
    lo = np.where((e & 1) == 0, w[0], w[2])
    hi = np.where((e & 1) == 0, w[1], w[3])
    z = _ih16(lo, hi).astype(np.float64)
    return z * c


def _ih4_matrix(seed, key, tid, m):
    """m x m integer matrix Z with entries in [-30, 30] (four 4-bit uniforms each).

    Element e uses nibbles 4 (e % 2) .. 4 (e % 2) + 3 of word (e // 2) % 4 of
    Philox call e // 8."""
    n = m * m
    e = np.arange(n, dtype=np.int64)
    w = philox4x32(e >> 3, 0, key, tid, seed, KEY_HI)
    word_sel = (e >> 1) & 3
    word = np.choose(word_sel, [x.astype(np.int64) for x in w])
    sh = (e & 1) * 16
    v = word >> sh
    z = (v & 15) + ((v >> 4) & 15) + ((v >> 8) & 15) + ((v >> 12) & 15) - IH4_MEAN
    return z.reshape(m, m)


def factor_scale(decay):
    """FP64 constant c with A = fl(z * c): unit-variance Gaussian times s_P."""
    return IH16_INV_STD * float(decay)


def amplitude_scale():
    return IH16_INV_STD * T_STD


def metric_scale(m):
    """c2 = fl(1 / (85 m)) so that c2 * Z Z^T = X X^T with X ~ N(0, 1/m)."""
    return 1.0 / (IH4_VAR * float(m))


def metric_from_int(Z, m, shift):
    S = Z.astype(np.float64) @ Z.T.astype(np.float64)   # exact: |S| < 2^53
    J = S * metric_scale(m)
    J[np.diag_indices(m)] += shift
    return J


def pair_inputs(wl, P):
    """Host tensors of pair P: dict Agi, Agj, Afi, Afj (p x m), Jg, Jf (m x m),
    Q (p x k), T (k x k), all float64 row-major.  Augmented workloads: the
    factors are (p + n_s) x m and T is (k + n_s) square."""
    key = wl.pair_key(P)
    p, k, m = int(wl.n_rows[P]), int(wl.n_pno[P]), int(wl.n_aux[P])
    diag = int(wl.pi[P]) == int(wl.pj[P])
    c = factor_scale(wl.decay[P])
    out = {}
    out["Agi"] = _gauss16(wl.seed, key, TID_AGI, p * m, c).reshape(p, m)
    out["Afi"] = _gauss16(wl.seed, key, TID_AFI, p * m, c).reshape(p, m)
    if diag:   # (ii) pair: both sides are the same orbital's block
        out["Agj"] = out["Agi"].copy()
        out["Afj"] = out["Afi"].copy()
    else:
        out["Agj"] = _gauss16(wl.seed, key, TID_AGJ, p * m, c).reshape(p, m)
        out["Afj"] = _gauss16(wl.seed, key, TID_AFJ, p * m, c).reshape(p, m)
    out["Jg"] = metric_from_int(_ih4_matrix(wl.seed, key, TID_XG, m), m, wl.metric_shift)
    out["Jf"] = metric_from_int(_ih4_matrix(wl.seed, key, TID_XF, m), m, wl.metric_shift)
    out["Q"] = pno_coefficients(wl, P)
    out["T"] = amplitudes(wl, P)
    return out


def pno_coefficients(wl, P):
    """Orthonormal p x k Q: QR of a Gaussian matrix, columns signed so diag(R) > 0."""
    key = wl.pair_key(P)
    p, k = int(wl.n_pao[P]), int(wl.n_pno[P])
    G = _gauss16(wl.seed, key, TID_Q, p * k, IH16_INV_STD).reshape(p, k)
    Qm, R = np.linalg.qr(G, mode="reduced")
    sgn = np.where(np.diag(R) < 0, -1.0, 1.0)
    return np.ascontiguousarray(Qm * sgn[None, :])


def amplitudes(wl, P):
    """k x k amplitudes, std 1e-2; symmetrised for diagonal pairs (t^{ab}_{ii} = t^{ba}_{ii})."""
    key = wl.pair_key(P)
    k = int(wl.n_virt[P])
    T = _gauss16(wl.seed, key, TID_T, k * k, amplitude_scale()).reshape(k, k)
    if int(wl.pi[P]) == int(wl.pj[P]):
        T = (T + T.T) * 0.5
    return np.ascontiguousarray(T)


# --------------------------------------------------------------------------
# packed (ragged) layout


def _round_up(x, a=ALIGN):
    return (x + a - 1) // a * a


def packed_offsets(wl, metric_packed=False):
    """Element offsets of each pair's blocks in the packed buffers.

    Returns dict with off_pm, off_mm, off_pk, off_kk (int64, n_pairs) and the
    buffer lengths len_pm, len_mm, len_pk, len_kk.  Blocks start on multiples of
    ALIGN doubles.  metric_packed: J blocks hold lower triangles, m (m + 1) / 2."""
    p = wl.n_pao.astype(np.int64)
    k = wl.n_pno.astype(np.int64)
    m = wl.n_aux.astype(np.int64)
    r, v = wl.n_rows, wl.n_virt       # factor rows and virtual dimension (augmented)
    mm = m * (m + 1) // 2 if metric_packed else m * m
    out = {}
    for name, sz in (("pm", r * m), ("mm", mm), ("pk", p * k), ("kk", v * v)):
        padded = _round_up(sz)
        off = np.zeros(len(sz), np.int64)
        if len(sz) > 1:
            off[1:] = np.cumsum(padded)[:-1]
        out["off_" + name] = off
        out["len_" + name] = int(padded.sum()) if len(sz) else 0
    return out


def pack_lower(J):
    """Lower triangle of a square matrix, row by row (row r: J[r, 0..r])."""
    return J[np.tril_indices(J.shape[0])]


def packed_inputs(wl, with_metrics=True, metric_packed=False):
    """Host packed buffers (float64) of every pair, plus the offsets.
    metric_packed: J blocks stored as lower triangles (pack_lower)."""
    lay = packed_offsets(wl, metric_packed)
    buf = {n: np.zeros(lay["len_pm"]) for n in ("Agi", "Agj", "Afi", "Afj")}
    if with_metrics:
        buf["Jg"] = np.zeros(lay["len_mm"])
        buf["Jf"] = np.zeros(lay["len_mm"])
    buf["Q"] = np.zeros(lay["len_pk"])
    buf["T"] = np.zeros(lay["len_kk"])
    for P in range(wl.n_pairs):
        t = pair_inputs(wl, P)
        for n in ("Agi", "Agj", "Afi", "Afj"):
            o = lay["off_pm"][P]
            buf[n][o:o + t[n].size] = t[n].ravel()
        if with_metrics:
            for n in ("Jg", "Jf"):
                o = lay["off_mm"][P]
                v = pack_lower(t[n]) if metric_packed else t[n].ravel()
                buf[n][o:o + v.size] = v
        o = lay["off_pk"][P]
        buf["Q"][o:o + t["Q"].size] = t["Q"].ravel()
        o = lay["off_kk"][P]
        buf["T"][o:o + t["T"].size] = t["T"].ravel()
    return buf, lay


def unpack(buf, off, P, rows, cols):
    o = int(off[P])
    return buf[o:o + rows * cols].reshape(rows, cols)
