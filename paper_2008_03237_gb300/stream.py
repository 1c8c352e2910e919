"""Pair-streamed execution for pair lists whose inputs exceed device memory.

The pair list is cut into contiguous batches whose packed inputs fit a byte
budget.  For each batch a caller-supplied producer fills reused device buffers
(integral code in an application, the synthetic generator in the tests and the
benchmark); the library then runs the fused forward launch, the pair energies
and optionally the adjoint on that batch.  Pair energies land in one device
array in pair-list order; the total is the FP64 sum of the batch totals in
batch order, so it is deterministic for a given budget.
"""
import numpy as np
import torch

from . import PairF12

ALIGN = 32  # packed blocks start on multiples of 32 doubles (256 B)


def packed_layout(n_pao, n_pno, n_aux, align=ALIGN):
    """Element offsets of the library's packed layout (see pf12_tensors)."""
    p, k, m = (np.asarray(a, np.int64) for a in (n_pao, n_pno, n_aux))
    out = {}
    for name, sz in (("pm", p * m), ("mm", m * m), ("pk", p * k), ("kk", k * k)):
        padded = (sz + align - 1) // align * align
        off = np.zeros(len(sz), np.int64)
        if len(sz) > 1:
            off[1:] = np.cumsum(padded)[:-1]
        out["off_" + name] = off
        out["len_" + name] = int(padded.sum()) if len(sz) else 0
    return out


def full_packed_layout(n_pao, n_pno, n_aux, align=ALIGN):
    """Element offsets of the complete-pair-energy layout (see pf12_full_tensors):
    off_pm ((p + 2) x m), off_mm, off_pk, off_kk, off_pp (p x p), off_s (2 x k),
    off_b (k x m x (k + 2))."""
    p, k, m = (np.asarray(a, np.int64) for a in (n_pao, n_pno, n_aux))
    out = {}
    for name, sz in (("pm", (p + 2) * m), ("mm", m * m), ("pk", p * k), ("kk", k * k),
                     ("pp", p * p), ("s", 2 * k), ("b", k * m * (k + 2))):
        padded = (sz + align - 1) // align * align
        off = np.zeros(len(sz), np.int64)
        if len(sz) > 1:
            off[1:] = np.cumsum(padded)[:-1]
        out["off_" + name] = off
        out["len_" + name] = int(padded.sum()) if len(sz) else 0
    return out


def input_bytes(n_pao, n_pno, n_aux):
    p, k, m = (np.asarray(a, np.float64) for a in (n_pao, n_pno, n_aux))
    return 8.0 * (4 * p * m + 2 * m * m + p * k + k * k)


def full_input_bytes(n_pao, n_pno, n_aux):
    p, k, m = (np.asarray(a, np.float64) for a in (n_pao, n_pno, n_aux))
    return 8.0 * (10 * (p + 2) * m + 3 * m * m + p * k + k * k + p * p + 2 * k + k * m * (k + 2))


# full-mode tensors and the layout key of each
FULL_KEYS = {**{n: "pm" for n in ("Agi", "Agj", "Afi", "Afj", "Ari", "Arj", "AgiF", "AgjF", "AriF",
                                  "ArjF")},
             "Jg": "mm", "Jf": "mm", "Jr": "mm", "Q": "pk", "T": "kk", "Fv": "pp", "S": "s", "B": "b"}
PLAIN_KEYS = {"Agi": "pm", "Agj": "pm", "Afi": "pm", "Afj": "pm", "Jg": "mm", "Jf": "mm",
              "Q": "pk", "T": "kk"}


def plan_batches(n_pao, n_pno, n_aux, budget_bytes, per=None):
    """Contiguous [begin, end) ranges of pairs with inputs <= budget_bytes each
    (per: bytes of each pair, default the amplitude-term inputs)."""
    per = input_bytes(n_pao, n_pno, n_aux) if per is None else np.asarray(per, np.float64)
    if len(per) and per.max() > budget_bytes:
        raise ValueError("one pair alone exceeds the batch budget")
    out, beg, acc = [], 0, 0.0
    for P, b in enumerate(per):
        if acc + b > budget_bytes and P > beg:
            out.append((beg, P))
            beg, acc = P, 0.0
        acc += b
    if beg < len(per):
        out.append((beg, len(per)))
    return out


class ResumeRecord:
    """Batch-level resume record of a streamed run: which batches are done,
    their totals, pair energies and statuses.  Written atomically (temporary
    file + rename) after every batch, so a run that stops (an exception in a
    producer, a lost process) restarts at the first unfinished batch and
    reproduces the uninterrupted result bit for bit."""

    def __init__(self, path, batches, n_pairs):
        self.path = path
        self.batches = np.asarray(batches, np.int64).reshape(-1, 2)
        self.n = int(n_pairs)
        self.done = np.zeros(len(self.batches), bool)
        self.totals = np.zeros(len(self.batches))
        self.e_pair = np.zeros((self.n, 3))
        self.status = np.zeros(self.n, np.int32)

    @classmethod
    def open(cls, path, batches, n_pairs):
        """The record at path if it belongs to the same batch plan, else a new one."""
        import os
        rec = cls(path, batches, n_pairs)
        if path and os.path.exists(path):
            with np.load(path) as z:
                if (int(z["n"]) == rec.n and z["batches"].shape == rec.batches.shape
                        and np.array_equal(z["batches"], rec.batches)):
                    rec.done = z["done"].astype(bool)
                    rec.totals = z["totals"].copy()
                    rec.e_pair = z["e_pair"].copy()
                    rec.status = z["status"].copy()
        return rec

    def commit(self, q, total, e_pair, status):
        import os
        b, e = self.batches[q]
        self.e_pair[b:e] = e_pair
        self.status[b:e] = status
        self.totals[q] = total
        self.done[q] = True
        if self.path:
            tmp = self.path + ".tmp.npz"
            np.savez(tmp, n=self.n, batches=self.batches, done=self.done, totals=self.totals,
                     e_pair=self.e_pair, status=self.status)
            os.replace(tmp, self.path)


class StreamedPairF12:
    """Runs the pair-F12 path batch by batch.

    producer(begin, end, tensors, layout) must fill the packed device tensors
    (keys Agi, Agj, Afi, Afj, Jg, Jf, Q, T) for pairs [begin, end) in the given
    layout.  grad_consumer(begin, end, grads, layout), when given, receives the
    batch's gradients (same packed layout) before the buffers are reused.
    checkpoint (a file path), when given, keeps a ResumeRecord: batches it
    lists as done are not produced or evaluated again (nor handed to the
    gradient consumer, which received them in the earlier run)."""

    def __init__(self, precision="mixed_fp32", budget_bytes=48e9, tuner_cache=None, full=False):
        """full: the complete pair energy (pf12_upload_full; tensors FULL_KEYS,
        layout full_packed_layout); no adjoint in that mode."""
        self.precision = precision
        self.budget = float(budget_bytes)
        self.tuner_cache = tuner_cache
        self.full = bool(full)

    def run(self, n_orb, orb_kind, pi, pj, n_pao, n_pno, n_aux, producer, backward=False,
            grad_consumer=None, dE=1.0, checkpoint=None):
        """Evaluates every batch; returns (E, e_pair (device, n x 3), status).

        Two sets of input buffers alternate: while batch q is evaluated on the
        current stream, the producer fills batch q + 1 on a side stream (torch's
        current stream while it runs; it must order its device work on that
        stream, not synchronise the device).  Its host work (for the synthetic
        generator, the PNO coefficients and amplitudes) overlaps the GPU's."""
        n = len(pi)
        if self.full and backward:
            raise ValueError("the complete pair energy has no adjoint")
        keys = FULL_KEYS if self.full else PLAIN_KEYS
        layout = full_packed_layout if self.full else packed_layout
        per = (full_input_bytes if self.full else input_bytes)(n_pao, n_pno, n_aux)
        batches = plan_batches(n_pao, n_pno, n_aux, self.budget, per)
        rec = ResumeRecord.open(checkpoint, batches, n)
        lays = [layout(n_pao[b:e], n_pno[b:e], n_aux[b:e]) for b, e in batches]
        cap = {key: max([L["len_" + key] for L in lays] + [2]) for key in set(keys.values())}
        dev = "cuda"
        todo = [q for q in range(len(batches)) if not rec.done[q]]
        n_sets = 2 if len(todo) > 1 else 1
        sets = [{x: torch.zeros(cap[key], dtype=torch.float64, device=dev) for x, key in keys.items()}
                for _ in range(n_sets)]
        g = None
        if backward:
            g = {x: torch.zeros_like(sets[0][x]) for x in ("Agi", "Agj", "Afi", "Afj", "Q", "T")}
        e_pair = torch.empty((max(n, 1), 3), dtype=torch.float64, device=dev)
        eng = PairF12(self.precision, tuner_cache=self.tuner_cache)
        compute = torch.cuda.current_stream()
        side = torch.cuda.Stream()
        produced = {}

        def produce(i):
            q = todo[i]
            b, e = batches[q]
            # the buffer set's previous batch (i - 1 of the same parity is i - 2)
            # is complete: the host synchronised on its results before this call
            with torch.cuda.stream(side):
                producer(b, e, sets[i % n_sets], lays[q])
                ev = torch.cuda.Event()
                ev.record(side)
            produced[i] = ev

        self.resumed = int(rec.done.sum())
        if todo:
            produce(0)
        for i, q in enumerate(todo):
            b, e = batches[q]
            t, lay = sets[i % n_sets], lays[q]
            compute.wait_event(produced.pop(i))
            upload = eng.upload_full if self.full else eng.upload_pairs
            upload(n_orb, orb_kind, pi[b:e], pj[b:e], n_pao[b:e], n_pno[b:e], n_aux[b:e], t, lay)
            eng.fit()
            failure = None
            if i + 1 < len(todo) and n_sets == 2:
                try:
                    produce(i + 1)                 # overlaps this batch's evaluation
                except Exception as exc:           # finish and record this batch first
                    failure = exc
            Eb, _ = eng.energy(e_pair[b:e], check=False)
            st_b = eng.pair_status()
            if backward:
                eng.backward(dE, g)
                if grad_consumer is not None:
                    grad_consumer(b, e, g, lay)
            rec.commit(q, Eb, e_pair[b:e].cpu().numpy(), st_b)
            if failure is not None:
                eng.close()
                raise failure
            if i + 1 < len(todo) and n_sets == 1:
                produce(i + 1)
        torch.cuda.synchronize()
        e_pair[:n].copy_(torch.from_numpy(rec.e_pair))
        status = rec.status.copy()
        E = 0.0
        for x in rec.totals:
            E += x
        self.stats = eng.stats()
        eng.close()
        self.batches = batches
        return E, e_pair[:n], status


def run_from_host(eng, n_orb, orb_kind, pi, pj, n_pao, n_pno, n_aux, host, layout,
                  budget_bytes):
    """End-to-end run from packed inputs in (pinned) host memory.

    The pair list is cut into batches under budget_bytes; batch b + 1's slices
    are copied host -> device on a separate stream into the other of two device
    slots while batch b is fitted on the current stream, so copies overlap the
    compute.  Batch b + 1's copies are issued after batch b's upload: the
    upload copies its small descriptor arrays from pageable memory on the
    compute stream, and queued behind a batch-sized copy that small copy
    would hold the fit back until the next batch had arrived.  eng is a PairF12 context, reused across calls (its device
    buffers and tuned variant carry over).  Returns (E, e_pair (device,
    n x 3), status, number of batches)."""
    n = len(pi)
    batches = plan_batches(n_pao, n_pno, n_aux, budget_bytes)
    kinds = {"Agi": "pm", "Agj": "pm", "Afi": "pm", "Afj": "pm", "Jg": "mm", "Jf": "mm",
             "Q": "pk", "T": "kk"}
    sizes = {"pm": np.asarray(n_pao, np.int64) * n_aux, "mm": np.asarray(n_aux, np.int64) ** 2,
             "pk": np.asarray(n_pao, np.int64) * n_pno, "kk": np.asarray(n_pno, np.int64) ** 2}
    ranges = []
    for b, e in batches:
        r = {}
        for key in ("pm", "mm", "pk", "kk"):
            off = layout["off_" + key]
            r[key] = (int(off[b]), int(off[e - 1] + sizes[key][e - 1]))
        ranges.append(r)
    cap = {key: max(r[key][1] - r[key][0] for r in ranges) + 2 for key in ("pm", "mm", "pk", "kk")}
    slots = [{x: torch.empty(cap[kinds[x]], dtype=torch.float64, device="cuda") for x in kinds}
             for _ in range(2)]
    copy_stream = torch.cuda.Stream()
    compute = torch.cuda.current_stream()
    copied = [torch.cuda.Event() for _ in batches]
    done = [torch.cuda.Event() for _ in batches]

    def issue(q):
        slot = slots[q % 2]
        with torch.cuda.stream(copy_stream):
            if q >= 2:
                copy_stream.wait_event(done[q - 2])
            for x, key in kinds.items():
                s0, s1 = ranges[q][key]
                slot[x][:s1 - s0].copy_(host[x][s0:s1], non_blocking=True)
            copied[q].record(copy_stream)

    e_pair = torch.empty((max(n, 1), 3), dtype=torch.float64, device="cuda")
    status = np.zeros(n, np.int32)
    totals = []
    issue(0)
    for q, (b, e) in enumerate(batches):
        compute.wait_event(copied[q])
        lay_b = {"off_" + key: np.asarray(layout["off_" + key][b:e]) - ranges[q][key][0]
                 for key in ("pm", "mm", "pk", "kk")}
        eng.upload_pairs(n_orb, orb_kind, pi[b:e], pj[b:e], n_pao[b:e], n_pno[b:e], n_aux[b:e],
                         slots[q % 2], lay_b)
        if q + 1 < len(batches):
            issue(q + 1)
        eng.fit()
        Eb, _ = eng.energy(e_pair[b:e], check=False)
        totals.append(Eb)
        status[b:e] = eng.pair_status()
        done[q].record(compute)
    torch.cuda.synchronize()
    E = 0.0
    for x in totals:
        E += x
    return E, e_pair[:n], status, len(batches)


def arrival_groups(n_pao, n_pno, n_aux, first_bytes=0.5e9, max_bytes=4e9, n_somo_aug=0,
                   metric_packed=False):
    """Contiguous pair groups for streamed inputs: the first group holds about
    first_bytes of inputs and each next one twice the previous, up to
    max_bytes, so the launch starts early and the copies stay ahead of it.
    Returns the group ends (int64, last = n_pairs)."""
    p = np.asarray(n_pao, np.float64) + n_somo_aug
    k = np.asarray(n_pno, np.float64)
    m = np.asarray(n_aux, np.float64)
    v = k + n_somo_aug
    mm = m * (m + 1) / 2 if metric_packed else m * m
    per = 8.0 * (4 * p * m + 2 * mm + (p - n_somo_aug) * k + v * v)
    ends, acc, cap = [], 0.0, float(first_bytes)
    for P, b in enumerate(per):
        if acc > 0 and acc + b > cap:
            ends.append(P)
            acc, cap = 0.0, min(2 * cap, float(max_bytes))
        acc += b
    if len(per):
        ends.append(len(per))
    return np.asarray(ends, np.int64)


class HostStreamer:
    """End-to-end evaluation of a pair list whose packed inputs sit in pinned
    host memory, with one persistent launch per call.

    Every call copies the inputs group by group (arrival_groups) on a copy
    stream into device buffers owned by this object and, after each group,
    writes that group's arrival flag with a 4-byte copy; the fit is launched
    at once and its CTAs wait for a group's flag before its first pair
    (pf12_set_arrival).  Copies and compute overlap without a launch, and a
    queue tail, per batch.  eng is a PairF12 context, reused across calls."""

    def __init__(self, eng, first_bytes=0.5e9, max_group_bytes=4e9, copy_streams=1):
        self.eng = eng
        self.first_bytes = float(first_bytes)
        self.max_group_bytes = float(max_group_bytes)
        self.dev = {}
        # groups may alternate between copy streams: each group's flag follows
        # its own copies on its stream and a CTA polls the flag of its pair's
        # group, so groups may land in any order.  One stream is the faster
        # choice: the queue consumes groups in order, and two streams share
        # the link between the group needed now and the next one (C160H321,
        # 3,895 pairs: 804 ms per step with one stream, 976 ms with two)
        self.copy_streams = [torch.cuda.Stream() for _ in range(max(1, int(copy_streams)))]
        self.epoch = 0
        self.epoch_host = torch.zeros(1, dtype=torch.int32, pin_memory=True)
        self.ready = None

    def _buffers(self, host):
        for x, h in host.items():
            if x not in self.dev or self.dev[x].numel() < h.numel():
                self.dev[x] = torch.empty(h.numel(), dtype=torch.float64, device="cuda")
        return self.dev

    def run(self, n_orb, orb_kind, pi, pj, n_pao, n_pno, n_aux, host, layout):
        """host: dict of pinned packed float64 tensors (Agi ... T) in the
        layout of `layout` (off_pm/off_mm/off_pk/off_kk).  Returns (E,
        e_pair (device, n x 3), status, number of groups)."""
        eng = self.eng
        n = len(pi)
        s_aug = int(np.sum(np.asarray(orb_kind) == 1)) if getattr(eng, "augment_somo", False) else 0
        tri = bool(getattr(eng, "metric_packed", False))
        ends = arrival_groups(n_pao, n_pno, n_aux, self.first_bytes, self.max_group_bytes, s_aug,
                              tri)
        dev = self._buffers(host)
        if self.ready is None or self.ready.numel() < max(len(ends), 1):
            self.ready = torch.zeros(max(len(ends), 1), dtype=torch.int32, device="cuda")
        # block ends per tensor kind: pair P's blocks end at off + size
        rows = np.asarray(n_pao, np.int64) + s_aug
        virt = np.asarray(n_pno, np.int64) + s_aug
        m = np.asarray(n_aux, np.int64)
        sizes = {"pm": rows * m, "mm": m * (m + 1) // 2 if tri else m * m,
                 "pk": np.asarray(n_pao, np.int64) * np.asarray(n_pno, np.int64), "kk": virt * virt}
        kinds = {"Agi": "pm", "Agj": "pm", "Afi": "pm", "Afj": "pm", "Jg": "mm", "Jf": "mm",
                 "Q": "pk", "T": "kk"}
        block_end = {key: np.asarray(layout["off_" + key], np.int64) + sizes[key] for key in sizes}
        for key, be in block_end.items():   # groups are copied as contiguous ranges
            if len(be) > 1 and (np.diff(np.asarray(layout["off_" + key], np.int64)) < 0).any():
                raise ValueError("HostStreamer needs blocks laid out in pair order")
        compute = torch.cuda.current_stream()
        # metadata first (small copies from pageable memory on the compute stream)
        eng.upload_pairs(n_orb, orb_kind, pi, pj, n_pao, n_pno, n_aux, dev, layout)
        if n == 0:
            eng.fit()
            E, e_pair = eng.energy(check=False)
            return E, e_pair, np.zeros(0, np.int32), 0
        self.epoch = (self.epoch + 1) & 0x7FFFFFFF
        eng.set_arrival(ends, self.ready, self.epoch)
        self.epoch_host[0] = self.epoch
        for cs in self.copy_streams:
            cs.wait_stream(compute)              # device buffers free (previous fit done)
        beg = {key: 0 for key in sizes}
        for g, e in enumerate(ends):
            cs = self.copy_streams[g % len(self.copy_streams)]
            with torch.cuda.stream(cs):
                for x, key in kinds.items():
                    s0, s1 = beg[key], int(block_end[key][e - 1])
                    if s1 > s0:
                        dev[x][s0:s1].copy_(host[x][s0:s1], non_blocking=True)
                self.ready[g:g + 1].copy_(self.epoch_host, non_blocking=True)
            for key in sizes:
                beg[key] = int(block_end[key][e - 1])
        eng.fit()
        E, e_pair = eng.energy(check=False)
        status = eng.pair_status()
        for cs in self.copy_streams:
            compute.wait_stream(cs)
        return E, e_pair, status, len(ends)
