"""Throughput of the pair-F12 path on GB300 (one JSON line on rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload c160h321] [--precision mixed_fp32] [--max-pairs N]

A step is one pass of the whole path over the workload's pair list: the fused
persistent forward launch (projections, FP64 Cholesky + solves, robust-fit V,
pair contractions) and the fixed-order FP64 energy total.  Inputs are drawn on
the device before timing (synthetic, seeded) and stay resident in HBM; they
total ~177 GB for the C160H321-shaped chain, far above the 129 MB L2, so no
L2 flush is needed between steps.

Also reported: the same step in plain FP64 mode, the error of the mixed-precision
energies against it, an end-to-end figure through the public API from pinned
host buffers, the roofline of the fused kernel, SM clocks sampled during the
timed region, and the FP64 CPU oracle timed on a bounded sample on the host
cores (--impl reference times that oracle as the reference arm).

Multi-GPU (torchrun): every rank runs an independent copy of the workload
(its own seed), so per-GPU work is fixed (weak scaling) and there is no
data-path collective; value = all ranks' pairs / the slowest rank's time.
With --shard the ranks instead split one pair list (LPT shards) and gather the
pair energies in list order every step (strong scaling).
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "F12 pairs/s & TFLOP/s, mixed-prec vs plain FP64 on 1 GB300 at ≤1 µEh error"
# FP64 peak of the pipe the fused kernels are bound by, derived from unit counts
# and clock: 152 SMs x 2 DFMA/clk/SM (4 flop/clk) x 2.07 GHz maximum SM clock
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12


def measured_peaks():
    """The generated MEASURED_PEAKS.json (BF16 tensor TFLOP/s, HBM GB/s), if present."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}
CHEM_SCALE_PER_ORB = 4.8e-3  # Eh per orbital (C160H322 F12 correction / valence orbitals)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c160h321")
    ap.add_argument("--precision", default="mixed_fp32", choices=["mixed_fp32", "fp64"])
    ap.add_argument("--max-pairs", type=int, default=0, help="deterministic subset (profiling)")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint figure (C40H81)")
    ap.add_argument("--no-full", action="store_true",
                    help="skip the complete-pair-energy figure (C40H81)")
    ap.add_argument("--shard", action="store_true",
                    help="torchrun: split ONE pair list over the ranks (LPT) and gather the pair "
                         "energies in list order every step (strong scaling); default: every "
                         "rank evaluates its own copy of the workload (weak scaling)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--stream-gb", type=float, default=0.0,
                    help="pair-streamed run: inputs drawn on the device batch by batch "
                         "(workloads larger than HBM); 0 = inputs resident")
    ap.add_argument("--backward", action="store_true", help="streamed run: adjoint per batch too")
    ap.add_argument("--augment-somo", action="store_true",
                    help="SOMO-augmented PNO space (no e2e or CPU legs)")
    ap.add_argument("--variant", type=int, default=None,
                    help="force a forward kernel variant instead of autotuning (profiling)")
    ap.add_argument("--full", action="store_true",
                    help="the complete pair energy E_(2)F12 (every term of Eqs. Vtilde, Btilde "
                         "with the PNO projector) instead of the amplitude term alone")
    return ap.parse_args()


def fp64_probe(iters=40000):
    """Measured FP64 FMA rate of this GPU (libpf12probe.so, CUDA events), TFLOP/s."""
    import ctypes
    from paper_2008_03237_gb300 import build as b
    lib = ctypes.CDLL(b.build_probe())
    fn = lib.pf12probe_fp64_fma
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    tf, ms = ctypes.c_double(0), ctypes.c_double(0)
    best = None
    for _ in range(3):
        rc = fn(iters, ctypes.byref(tf), ctypes.byref(ms))
        if rc != 0:
            return None
        best = tf.value if best is None else max(best, tf.value)
    return {"tflops": best, "kernel": "dfma_chains (16 independent FMA chains per thread, "
            "8 CTAs x 256 threads per SM)", "ms_per_launch": ms.value, "best_of": 3}


def make_workload(name, max_pairs, rank=0):
    import synthetic as S
    wl = S.WORKLOADS[name]()
    if rank:
        wl.seed += 1000 * rank
    if max_pairs and max_pairs < wl.n_pairs:
        idx = np.linspace(0, wl.n_pairs - 1, max_pairs).round().astype(np.int64)
        wl = wl.subset(np.unique(idx), name=f"{wl.name}[{max_pairs} pairs]")
    return wl


# DRAM bytes (read + write) of one launch of the forward kernel, measured by
# ncu (dram__bytes_read.sum + dram__bytes_write.sum) on a deterministic subset
# of the C160H321 chain and scaled to other lists by algorithmic input bytes.
# Only the variant whose current code was captured is listed: variant 3 (SIMT,
# 3 CTAs/SM, look-ahead 16, FP32 tile with cp.async staging), 400 pairs,
# 5.01 GB of algorithmic input bytes.
TRAFFIC_CAPTURE = {
    3: {"bytes": 17.657836e9 + 4.410247e9, "alg_bytes": 5011263536.0,
        "precision": "mixed_fp32"},
}


def traffic_bytes(args, wl, byts, variant):
    """Per-launch DRAM traffic of the dominant kernel, from the ncu capture of
    the same kernel variant scaled by algorithmic bytes; None when the timed
    kernel is not a captured one."""
    cap = TRAFFIC_CAPTURE.get(variant)
    if (cap is None or args.precision != cap["precision"] or args.stream_gb
            or args.augment_somo):
        return None
    return cap["bytes"] * byts / cap["alg_bytes"]


def flops_bytes(wl):
    """Algorithmic FP64 flops, mixable flops and input bytes of one forward
    pass.  SOMO-augmented lists: the solves and V act on k + n_s virtuals, the
    factors have p + n_s rows, Q stays p x k."""
    p, k, m = (wl.n_pao.astype(float), wl.n_pno.astype(float), wl.n_aux.astype(float))
    v, r = wl.n_virt.astype(float), wl.n_rows.astype(float)
    f64 = float((m ** 3 / 3 + 4 * v * m * m).sum())
    fmix = float((8 * p * k * m + 2 * v * m * m + 4 * v * v * m).sum())
    byts = float((8 * (4 * r * m + 2 * m * m + p * k + v * v)).sum())
    return f64, fmix, byts


# --------------------------------------------------------------------------- clocks


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = np.array([num(r[1]) for r in rows])
        mx = np.nanmax([num(r[2]) for r in rows])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i]
                          and "Not" not in r[5 + i]})
        return {"sm_mhz": float(np.nanmedian(sm)), "sm_max_mhz": float(mx), "reasons": reasons,
                "samples": len(rows), "power_w_max": float(np.nanmax([num(r[3]) for r in rows]))}


# --------------------------------------------------------------------------- CPU oracle


_ORACLE_WORKER = """
import sys, os, time, json
sys.path.insert(0, {root!r})
import numpy as np
import oracle, synthetic as S
from bench import make_workload
wl = make_workload({name!r}, {max_pairs})
rank, nproc, budget, n_pairs, steps, go = {rank}, {nproc}, {budget}, {n_pairs}, {steps}, {go!r}
order = np.random.default_rng(12345).permutation(wl.n_pairs)[rank::nproc][:n_pairs]
cache = [(int(P), S.pair_inputs(wl, int(P))) for P in order]   # drawn before any timing
open(go + ".ready%d" % rank, "w").close()
res = []
for s in range(steps):
    while not os.path.exists(go + ".%d" % s):
        time.sleep(0.01)
    done, t_used = 0, 0.0
    for P, t in cache:
        t0 = time.perf_counter()
        oracle.run(wl, pairs=[P], inputs=lambda q: t)
        t_used += time.perf_counter() - t0
        done += 1
        if t_used >= budget:
            break
    res.append((done, t_used))
    open(go + ".done%d.%d" % (s, rank), "w").close()
print(json.dumps(res))
"""


def cpu_model():
    """Host CPU model name (lscpu, else /proc/cpuinfo), for the baseline record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cpu_oracle_rate(wl, budget_s, threads=None, steps=1):
    """FP64 CPU oracle (as it stands) on a deterministic sample of wl's pairs,
    parallel over pairs: `threads` worker processes with one BLAS thread each
    (default: every host core).  Each worker draws the inputs of its share of
    the sample once, before any timing; then, `steps` times, all workers are
    released together and each evaluates its pairs in order until its oracle
    time reaches budget_s.  A step's rate is all pairs evaluated in it / the
    slowest worker's oracle time.  Returns (per-step pairs/s list, workers,
    sample description)."""
    import shutil
    import tempfile
    nproc = threads or os.cpu_count() or 1
    # pairs each worker draws: the oracle runs tens of pairs/s per core on the
    # bench workload, drawing the inputs about ten times slower
    n_pairs = 12 + int(6 * budget_s)
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    tmp = tempfile.mkdtemp(prefix="pf12_oracle_")
    go = os.path.join(tmp, "go")
    procs = []
    for r in range(nproc):
        code = _ORACLE_WORKER.format(root=ROOT, name=wl.meta.get("bench_name", "c160h321"),
                                     max_pairs=int(wl.meta.get("bench_max", 0)), rank=r,
                                     nproc=nproc, budget=float(budget_s), n_pairs=n_pairs,
                                     steps=int(steps), go=go)
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))

    def wait_files(names):
        while not all(os.path.exists(x) for x in names):
            if any(p.poll() not in (None, 0) for p in procs):
                _, err = next(p for p in procs if p.poll() not in (None, 0)).communicate()
                raise RuntimeError("cpu oracle worker failed: " + err[-2000:])
            time.sleep(0.02)
    wait_files([go + ".ready%d" % r for r in range(nproc)])
    for s in range(steps):       # one step at a time: all workers start together
        open(go + ".%d" % s, "w").close()
        wait_files([go + ".done%d.%d" % (s, r) for r in range(nproc)])
    per = []
    for p in procs:
        out, err = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("cpu oracle worker failed: " + err[-2000:])
        per.append(json.loads(out.strip().splitlines()[-1]))
    shutil.rmtree(tmp, ignore_errors=True)
    rates, done_last, slow_last = [], 0, 0.0
    for s in range(steps):
        done = sum(w[s][0] for w in per)
        slowest = max(w[s][1] for w in per)
        rates.append(done / slowest)
        done_last, slow_last = done, slowest
    return rates, nproc, (f"{done_last} pairs of {wl.name} per step (fixed permutation, seed "
                          f"12345; inputs drawn before timing) over {nproc} worker process(es) x "
                          f"1 BLAS thread, {slow_last:.1f} s of oracle time in the slowest worker")


# --------------------------------------------------------------------------- our arm


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    import __graft_entry__
    import paper_2008_03237_gb300 as pf
    from synthetic import device

    torch.cuda.set_device(local_rank)
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
        __graft_entry__.build()
    wl = make_workload(args.workload, args.max_pairs, rank)
    wl.meta["bench_name"] = args.workload
    wl.meta["bench_max"] = args.max_pairs
    if args.augment_somo:
        wl = wl.augmented()
        args.no_e2e = args.no_cpu = True
    f64, fmix, byts = flops_bytes(wl)
    t, lay = device.allocate(wl)
    device.fill(wl, t, lay)

    def make(prec):
        var = args.variant if (args.variant is not None and (prec != "fp64" or args.variant < 2)) else None
        eng = pf.PairF12(prec, variant=var, augment_somo=args.augment_somo)
        eng.upload_pairs(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux, t, lay)
        return eng

    def timed(eng, steps, warmup, sampler=None):
        stream = torch.cuda.current_stream()
        for _ in range(warmup):
            eng.fit()
            eng.energy(want_host=False)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        fit_ms = []
        ev0.record(stream)
        ctx = sampler if sampler is not None else _Null()
        with ctx:
            for _ in range(steps):
                eng.fit()
                eng.energy(want_host=False)
                fit_ms.append(None)
            ev1.record(stream)
            torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ms = ev0.elapsed_time(ev1) / steps
        return ms

    out = {}
    if args.backward:
        # differentiation workload: every step is forward + energy + adjoint
        # (gradients w.r.t. A^g, A^f, Q, T into resident buffers)
        eng = make(args.precision)
        grads = {x: torch.zeros_like(t[x]) for x in ("Agi", "Agj", "Afi", "Afj", "Q", "T")}
        for _ in range(args.warmup):
            eng.fit()
            eng.energy(want_host=False)
            eng.backward(1.0, grads)
        torch.cuda.synchronize()
        sampler = ClockSampler(local_rank)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        bwd_ms = []
        with sampler:
            ev0.record()
            for _ in range(args.steps):
                eng.fit()
                eng.energy(want_host=False)
                eng.backward(1.0, grads)
            ev1.record()
            torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / args.steps
        st = eng.stats()
        E, _ = eng.energy()
        out.update(ms=ms, ms_fit=st["ms_fit"], ms_backward=st["ms_backward"], E=E,
                   status_bad=int((eng.pair_status() != 0).sum()), stats=st,
                   clocks=sampler.summary())
        eng.close()
        del grads
        return wl, f64, fmix, byts, out
    # headline: requested precision
    eng = make(args.precision)
    sampler = ClockSampler(local_rank)
    ms = timed(eng, args.steps, args.warmup, sampler)
    # per-launch duration of the fused kernel, measured on its own stream with events
    fit_ms = []
    for _ in range(max(2, min(args.steps, 5))):
        eng.fit()
        fit_ms.append(eng.stats()["ms_fit"])
    ms_fit = float(np.mean(fit_ms))
    E, e_pair = eng.energy()
    e_main = e_pair.cpu().numpy()
    status_bad = int((eng.pair_status() != 0).sum())
    st = eng.stats()
    eng.close()
    del eng
    torch.cuda.empty_cache()
    out.update(ms=ms, ms_fit=ms_fit, E=E, status_bad=status_bad, stats=st, clocks=sampler.summary())

    # plain FP64 mode of the same step, and the error of the headline energies against it
    if not args.no_fp64_compare and args.precision != "fp64":
        eng = make("fp64")
        ms64 = timed(eng, min(4, max(2, args.steps // 2)), 1)
        E64, e64 = eng.energy()
        e64 = e64.cpu().numpy()
        eng.close()
        del eng
        torch.cuda.empty_cache()
        sum_abs = float(np.abs(e64.sum(axis=1)).sum())
        kappa = CHEM_SCALE_PER_ORB * wl.n_orb / sum_abs
        out["fp64_mode"] = {"value": wl.n_pairs / ms64 * 1e3, "ms_per_step": ms64,
                            "fp64_tflops": (f64 + fmix) / ms64 / 1e9}
        out["error_vs_fp64"] = {
            "total_Eh_normalised": abs(E - E64) * kappa,
            "max_pair_Eh_normalised": float(np.abs(e_main - e64).max() * kappa),
            "total_rel_to_sum_abs": abs(E - E64) / sum_abs, "kappa": kappa,
            "E_mixed_raw": E, "E_fp64_raw": E64}

    # end to end through the public API from pinned host buffers
    if not args.no_e2e:
        out["e2e"] = run_e2e(args, wl, t, lay, pf, torch)
    del t
    torch.cuda.empty_cache()
    if not args.no_adjoint and world == 1:
        out["adjoint"] = run_adjoint(args, pf, torch, device)
    if not args.no_full and world == 1:
        out["full_energy"] = full_energy_figure(args, pf, torch, device, "c40h81", steps=3, warmup=1)
    out["fp64_probe"] = fp64_probe()
    return wl, f64, fmix, byts, out


def run_adjoint(args, pf, torch, device, name="c40h81"):
    """Device time of the adjoint kernel (pf12_backward) on the C40H81 chain:
    gradients with respect to A^g, A^f, Q and T of all 2,821 pairs into
    resident buffers, three launches after the tuning one, CUDA events on the
    launching stream.  Algorithmic FP64 work per pair: m^3/3 + 8 k m^2 (the
    factorisation, the two solves of the forward fit and the two of
    Z^T = R J_g^{-1})."""
    wl = make_workload(name, 0)
    t, lay = device.allocate(wl)
    device.fill(wl, t, lay)
    eng = pf.PairF12(args.precision)
    eng.upload_pairs(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux, t, lay)
    eng.fit()
    eng.energy(want_host=False)
    grads = {x: torch.zeros_like(t[x]) for x in ("Agi", "Agj", "Afi", "Afj", "Q", "T")}
    eng.backward(1.0, grads)
    ms = []
    for _ in range(3):
        eng.backward(1.0, grads)
        ms.append(eng.stats()["ms_backward"])
    st = eng.stats()
    bad = int((eng.pair_status() != 0).sum())
    eng.close()
    del grads, t
    torch.cuda.empty_cache()
    k, m = wl.n_pno.astype(float), wl.n_aux.astype(float)
    f64_b = float((m ** 3 / 3 + 8 * k * m * m).sum())
    ms_mean = float(np.mean(ms))
    return {"workload": wl.name, "pairs": wl.n_pairs, "precision": args.precision,
            "kernel": "pair_backward_kernel (fused persistent adjoint)",
            "ms_per_launch": ms_mean, "ms_launches": ms, "fp64_tflops": f64_b / ms_mean / 1e9,
            "frac_of_fp64_peak": f64_b / ms_mean / 1e9 / FP64_PEAK_TFLOPS,
            "variant": st["bwd_variant"], "tune_ms": st["tune_bwd_ms"], "pairs_failed": bad}


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def host_memory_available():
    """Bytes the host can still give (MemAvailable of /proc/meminfo), or 0."""
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def run_e2e(args, wl_full, t_full, lay_full, pf, torch):
    """Pairs/s of the workload end to end from pinned host memory: every step
    uploads the pair list, copies the inputs host->device group by group on a
    copy stream while one persistent fit (launched at once) waits for each
    group's arrival flag, and reads the total and the pair statuses back to
    the host.  The whole list is used when its packed inputs fit in 70 % of
    the host's available memory, else the longest prefix that does (recorded
    in the result).  The resident device inputs are released once the host
    copies exist (t_full is emptied)."""
    import synthetic as S
    from synthetic import workloads as W
    budget = 0.7 * host_memory_available()
    n = 0
    acc = 0.0
    p, k, m = wl_full.n_pao, wl_full.n_pno, wl_full.n_aux
    per = 8.0 * (4 * p * m + m * (m + 1) + p * k + k * k)      # packed metric triangles
    while n < wl_full.n_pairs and acc + per[n] <= budget:
        acc += per[n]
        n += 1
    if n == 0:
        raise RuntimeError("no host memory for the end-to-end inputs")
    prefix = wl_full.subset(np.arange(n))
    lay_src = W.packed_offsets(prefix)        # where the prefix blocks sit in t_full
    # the host keeps its pair list longest first (the library's cost model), so
    # that arrival groups follow the persistent queue's order and the launch
    # ends on the smallest pairs
    pp, kk, mm_ = (prefix.n_pao.astype(float), prefix.n_pno.astype(float), prefix.n_aux.astype(float))
    cost = mm_ ** 3 / 3 + 4 * kk * mm_ ** 2 + (8 * pp * kk * mm_ + 2 * kk * mm_ ** 2 + 4 * kk * kk * mm_) / 8
    order = np.argsort(-cost, kind="stable")
    label = "all" if n == wl_full.n_pairs else f"first {n}"
    wl = prefix.subset(order, name=f"{wl_full.name}[{label} pairs, longest first]")
    # and the metrics as packed lower triangles (pf12_opts.metric_packed): they
    # are symmetric, and that cuts the bytes each step copies by a third
    lay = W.packed_offsets(wl, metric_packed=True)
    lens = {"Agi": lay["len_pm"], "Agj": lay["len_pm"], "Afi": lay["len_pm"], "Afj": lay["len_pm"],
            "Jg": lay["len_mm"], "Jf": lay["len_mm"], "Q": lay["len_pk"], "T": lay["len_kk"]}
    key = {"Agi": "pm", "Agj": "pm", "Afi": "pm", "Afj": "pm", "Jg": "mm", "Jf": "mm", "Q": "pk",
           "T": "kk"}
    size = {"pm": wl.n_pao.astype(np.int64) * wl.n_aux, "pk": wl.n_pao.astype(np.int64) * wl.n_pno,
            "kk": wl.n_pno.astype(np.int64) ** 2}
    tril = {}
    host = {}
    for x, L in lens.items():       # pinned buffers written by the host, as an application's
        src = torch.zeros(max(L, 2), dtype=torch.float64, device="cuda")
        kx = key[x]
        for P in range(n):          # gathered on the device in the new order
            o_s, o_d = int(lay_src["off_" + kx][order[P]]), int(lay["off_" + kx][P])
            if kx == "mm":          # lower triangle of the full block
                m = int(wl.n_aux[P])
                if m not in tril:
                    r, c = np.tril_indices(m)
                    tril[m] = torch.from_numpy(r * m + c).cuda()
                src[o_d:o_d + tril[m].numel()] = t_full[x][o_s:o_s + m * m][tril[m]]
            else:
                z = int(size[kx][P])
                src[o_d:o_d + z] = t_full[x][o_s:o_s + z]
        host[x] = torch.empty(max(L, 2), dtype=torch.float64, pin_memory=True)
        host[x].copy_(src)
        del src
    del tril
    t_full.clear()                  # the resident inputs are not needed any more
    torch.cuda.empty_cache()
    h2d = sum(v.numel() * 8 for v in host.values())
    from paper_2008_03237_gb300.stream import HostStreamer
    # raw pinned host -> device bandwidth of this machine (one large copy)
    big = host["Jg"]
    dst = torch.empty_like(big, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dst.copy_(big, non_blocking=True)
    torch.cuda.synchronize()
    h2d_gbs = big.numel() * 8 / (time.perf_counter() - t0) / 1e9
    del dst
    eng = pf.PairF12(args.precision, variant=args.variant, metric_packed=True)
    streamer = HostStreamer(eng)

    def step():
        E, _, st, ng = streamer.run(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno,
                                    wl.n_aux, host, lay)
        if (st != 0).any():
            raise RuntimeError("e2e step: pairs failed")
        return E, ng
    for _ in range(2):
        step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps = min(5, max(2, args.steps))
    for _ in range(steps):
        E_e2e, nb = step()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    eng.close()
    del host, streamer
    torch.cuda.empty_cache()
    return {"value": n / dt, "unit": "pairs/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": 32 + 4 * n, "pairs": n, "ms_per_step": dt * 1e3, "steps": steps,
            "host_budget_gb": budget / 1e9,
            "workload": wl.name, "arrival_groups": nb, "h2d_gbs_raw": h2d_gbs,
            "metric_layout": "packed lower triangles",
            "note": "pinned host inputs copied in growing groups (0.5 GB doubling to 4 GB) on a "
                    "copy stream; one persistent fit per step waits for each group's arrival flag"}


# --------------------------------------------------------------------------- main


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if args.stream_gb:
        return run_streamed(args, rank, world, local_rank)
    if args.shard and world > 1:
        return run_sharded(args, rank, world, local_rank)
    if args.full and not args.stream_gb:
        return run_full(args, rank, world, local_rank)
    wl, f64, fmix, byts, o = run_ours(args, rank, world, local_rank)
    ms = o["ms"]
    if world > 1:
        import torch
        import torch.distributed as dist
        x = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        ms = float(x.item())
    if rank != 0:
        return
    n_pairs = wl.n_pairs
    value = world * n_pairs / ms * 1e3
    flops_dom = f64 + (fmix if args.precision == "fp64" else 0.0)
    achieved = flops_dom / o["ms_fit"] / 1e9
    probe = o.get("fp64_probe")
    line = {
        "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32" if args.precision != "fp64" else "f64",
        "data": "synthetic (seeded Philox4x32-10 draws, device-resident)",
        "config": {"workload": wl.name, "pairs": n_pairs, "orbitals": wl.n_orb,
                   "somos": wl.n_somo, "somo_augmented": bool(wl.somo_aug),
                   "precision": args.precision,
                   "p_range": [int(wl.n_pao.min()), int(wl.n_pao.max())],
                   "k_range": [int(wl.n_pno.min()), int(wl.n_pno.max())],
                   "m_range": [int(wl.n_aux.min()), int(wl.n_aux.max())],
                   "l2": f"inputs {byts / 1e9:.0f} GB >> 129 MB L2, no flush"},
        "tflops": {"fp64": f64 / ms / 1e9, "mixed_part": fmix / ms / 1e9,
                   "total": (f64 + fmix) / ms / 1e9,
                   "fp64_frac_of_peak": f64 / ms / 1e9 / FP64_PEAK_TFLOPS,
                   "mixed_part_frac_of_bf16_tensor_peak":
                       (fmix / ms / 1e9 / measured_peaks()["bf16_tflops"])
                       if measured_peaks().get("bf16_tflops") else None},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                     "traffic": traffic_bytes(args, wl, byts, o["stats"]["tile_config"]),
                     "kernel": "pair_forward_kernel (fused persistent)",
                     "peak_kind": "FP64 DFMA pipe, derived: 152 SMs x 4 flop/clk x 2.07 GHz",
                     "peak_measured": probe["tflops"] if probe else None,
                     "frac_of_measured": achieved / probe["tflops"] if probe else None,
                     "ms_per_launch": o["ms_fit"]},
        "fp64_probe": probe,
        "clocks": o["clocks"],
        "gpu_launches": 2 * args.steps,
        "E_total_raw": o["E"], "pairs_failed": o["status_bad"],
        "autotuner": {"variant": o["stats"]["tile_config"],
                      "variants": ["SIMT 2 CTAs/SM look-ahead 8", "SIMT 3 CTAs/SM look-ahead 8",
                                   "tcgen05 3 CTAs/SM look-ahead 8", "SIMT 3 CTAs/SM look-ahead 16"],
                      "sample_ms_median_of_3": o["stats"]["tune_ms"],
                      "ctas": o["stats"]["ctas_variant"],
                      "tile_shape": {n: o["stats"][n] for n in ("look_depth", "ctas_per_sm",
                                                                 "tensor_cores", "gemm_tile",
                                                                 "gemm_k_chunk", "panel_width")}},
    }
    for key in ("fp64_mode", "error_vs_fp64", "e2e", "adjoint", "full_energy"):
        if key in o:
            line[key] = o[key]
    if args.backward:
        # adjoint FP64 work per pair: m^3/3 + 8 k m^2 (factorisation + four solves)
        p_, k_, m_ = (wl.n_pao.astype(float), wl.n_pno.astype(float), wl.n_aux.astype(float))
        f64_b = float((m_ ** 3 / 3 + 8 * k_ * m_ * m_).sum())
        line["config"]["step"] = "forward + energy + adjoint"
        line["backward"] = {"ms_per_launch": o["ms_backward"],
                            "fp64_tflops": f64_b / o["ms_backward"] / 1e9,
                            "frac_of_fp64_peak": f64_b / o["ms_backward"] / 1e9 / FP64_PEAK_TFLOPS}
        line["gpu_launches"] = 3 * args.steps
    if "e2e" not in line:
        line["e2e"] = None
    if not args.no_cpu and world == 1:
        (rate,), cores, sample = cpu_oracle_rate(wl, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                                "cpu_model": cpu_model(),
                                "sample": sample}
        (rate1,), _, sample1 = cpu_oracle_rate(wl, max(3.0, args.cpu_seconds / 3), threads=1)
        line["cpu_baseline_1thread"] = {"value": rate1, "unit": "pairs/s", "cores": 1,
                                        "kind": "oracle", "sample": sample1}
    print(json.dumps(line), flush=True)


def full_flops(wl):
    """Algorithmic FP64 flops (factorisation + solves on 4p + 4 right-hand
    sides), mixable flops and input bytes of one full-energy pass."""
    p, k, m = (wl.n_pao.astype(float), wl.n_pno.astype(float), wl.n_aux.astype(float))
    k2 = k + 2
    f64 = float((m ** 3 / 3 + 2 * (4 * p + 4) * m * m).sum())
    fmix = float((8 * p * k * m + 2 * k2 * m * m + 4 * k2 * k2 * m + 4 * p * m * m
                  + 12 * p * p * m + 8 * p * p * k + 12 * p * k * k + 2 * k * k * k2 * m
                  + 2 * k * k2 * k2 * m + 4 * p ** 3).sum())
    byts = float((8 * (10 * (p + 2) * m + 3 * m * m + p * k + k * k + p * p + 2 * k
                       + k * m * k2)).sum())
    return f64, fmix, byts


def full_energy_figure(args, pf, torch, device, name, max_pairs=0, local_rank=0, steps=None,
                       warmup=None, sample_clocks=False):
    """The complete pair energy on one workload with resident inputs: the
    requested precision timed (CUDA events around fit + energy), the FP64
    mode beside it, and the error of the mixed energies against FP64 on the
    chemical scale."""
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    wl = make_workload(name, max_pairs)
    f64, fmix, byts = full_flops(wl)
    t, lay = device.allocate_full(wl)
    device.fill_full(wl, t, lay)
    res = {}
    for prec in (args.precision, "fp64") if args.precision != "fp64" else ("fp64",):
        eng = pf.PairF12(prec, variant=args.variant if args.full else None)
        eng.upload_full(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno, wl.n_aux, t, lay)
        n_steps = steps if prec == args.precision else max(2, steps // 2)
        for _ in range(warmup if prec == args.precision else 1):
            eng.fit()
            eng.energy(want_host=False)
        torch.cuda.synchronize()
        sampler = ClockSampler(local_rank) if (sample_clocks and prec == args.precision) else _Null()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        with sampler:
            ev0.record()
            for _ in range(n_steps):
                eng.fit()
                eng.energy(want_host=False)
            ev1.record()
            torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / n_steps
        E, e = eng.energy()
        st = eng.stats()
        res[prec] = {"ms": ms, "ms_fit": st["ms_fit"], "E": E, "e": e.cpu().numpy(),
                     "bad": int((eng.pair_status() != 0).sum()), "variant": st["tile_config"],
                     "tune_ms": st["tune_ms"][:2],
                     "clocks": sampler.summary() if isinstance(sampler, ClockSampler) else None}
        eng.close()
    del t
    torch.cuda.empty_cache()
    head = res[args.precision]
    achieved = (f64 + (fmix if args.precision == "fp64" else 0)) / head["ms_fit"] / 1e9
    out = {"workload": wl.name, "pairs": wl.n_pairs, "precision": args.precision,
           "energy": "complete E_(2)F12 per pair (occupied, amplitude, C and singles terms of "
                     "Vtilde; B~ with i_F, j_F; PNO projector term)",
           "value": wl.n_pairs / head["ms"] * 1e3, "unit": "pairs/s", "ms_per_step": head["ms"],
           "kernel": "pair_full_kernel (fused persistent)", "ms_per_launch": head["ms_fit"],
           "fp64_tflops": f64 / head["ms_fit"] / 1e9, "mixed_part_tflops": fmix / head["ms_fit"] / 1e9,
           "achieved_tflops": achieved, "frac_of_fp64_peak": achieved / FP64_PEAK_TFLOPS,
           "inputs_gb": byts / 1e9, "E_total_raw": head["E"], "pairs_failed": head["bad"],
           "variant": head["variant"], "tune_ms": head["tune_ms"], "clocks": head["clocks"]}
    if "fp64" in res and args.precision != "fp64":
        r64 = res["fp64"]
        sum_abs = float(np.abs(r64["e"].sum(axis=1)).sum())
        kappa = CHEM_SCALE_PER_ORB * wl.n_orb / sum_abs
        out["fp64_mode"] = {"value": wl.n_pairs / r64["ms"] * 1e3, "ms_per_step": r64["ms"],
                            "fp64_tflops": (f64 + fmix) / r64["ms_fit"] / 1e9,
                            "frac_of_fp64_peak": (f64 + fmix) / r64["ms_fit"] / 1e9 / FP64_PEAK_TFLOPS}
        out["error_vs_fp64"] = {"total_Eh_normalised": abs(head["E"] - r64["E"]) * kappa,
                                "max_pair_Eh_normalised": float(np.abs(head["e"] - r64["e"]).max() * kappa),
                                "kappa": kappa}
    return out


def run_full(args, rank, world, local_rank):
    """bench.py --full: the complete pair energy as the headline line (default
    workload C40H81, whose inputs stay resident)."""
    import torch

    import __graft_entry__
    import paper_2008_03237_gb300 as pf
    from synthetic import device
    torch.cuda.set_device(local_rank)
    __graft_entry__.build()
    name = args.workload if args.workload != "c160h321" or args.max_pairs else "c40h81"
    fig = full_energy_figure(args, pf, torch, device, name, args.max_pairs, local_rank,
                             sample_clocks=True)
    line = {"metric": METRIC, "value": fig["value"], "unit": "pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": fig["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64+f32" if args.precision != "fp64" else "f64",
            "data": "synthetic (seeded Philox4x32-10 draws, device-resident)",
            "config": {"workload": fig["workload"], "pairs": fig["pairs"],
                       "precision": args.precision, "energy": fig["energy"],
                       "l2": f"inputs {fig['inputs_gb']:.0f} GB >> 129 MB L2, no flush"},
            "tflops": {"fp64": fig["fp64_tflops"], "mixed_part": fig["mixed_part_tflops"]},
            "roofline": {"bound": "alu", "achieved": fig["achieved_tflops"],
                         "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": fig["frac_of_fp64_peak"], "kernel": fig["kernel"],
                         "ms_per_launch": fig["ms_per_launch"], "traffic": None},
            "clocks": fig["clocks"], "gpu_launches": 2 * args.steps, "e2e": None,
            "E_total_raw": fig["E_total_raw"], "pairs_failed": fig["pairs_failed"],
            "autotuner": {"variant": fig["variant"], "sample_ms": fig["tune_ms"],
                          "variants": ["2 CTAs/SM", "3 CTAs/SM"]}}
    for key in ("fp64_mode", "error_vs_fp64"):
        if key in fig:
            line[key] = fig[key]
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_sharded(args, rank, world, local_rank):
    """One pair list split over the ranks: longest-processing-time shards by
    the kernel's cost model, every rank holding and evaluating its shard only;
    each step ends with the pair energies gathered over NCCL in pair-list
    order and summed on the host (shard.gather_pair_energies).  value = the
    list's pairs / the slowest rank's step time (strong scaling)."""
    import torch
    import torch.distributed as dist

    import __graft_entry__
    import paper_2008_03237_gb300 as pf
    from paper_2008_03237_gb300.shard import gather_pair_energies, lpt_partition, pair_costs
    from synthetic import device
    torch.cuda.set_device(local_rank)
    if rank == 0:
        __graft_entry__.build()
    dist.barrier()
    __graft_entry__.build()
    wl = make_workload(args.workload, args.max_pairs)          # the same list on every rank
    mine = lpt_partition(pair_costs(wl.n_pao, wl.n_pno, wl.n_aux), world)[rank]
    sub = wl.subset(mine)
    f64, fmix, byts = flops_bytes(wl)
    t, lay = device.allocate(sub)
    device.fill(sub, t, lay)
    eng = pf.PairF12(args.precision, variant=args.variant)
    eng.upload_pairs(sub.n_orb, sub.orb_kind, sub.pi, sub.pj, sub.n_pao, sub.n_pno, sub.n_aux, t, lay)
    e_loc = torch.empty((sub.n_pairs, 3), dtype=torch.float64, device="cuda")

    def step():
        eng.fit()
        eng.energy(e_pair=e_loc, want_host=False)
        return gather_pair_energies(e_loc.cpu().numpy(), mine, wl.n_pairs)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with sampler:
        ev0.record()
        for _ in range(args.steps):
            full, total = step()
        ev1.record()
        torch.cuda.synchronize()
    dist.barrier()
    ms = ev0.elapsed_time(ev1) / args.steps
    x = torch.tensor([ms], device="cuda", dtype=torch.float64)
    dist.all_reduce(x, op=dist.ReduceOp.MAX)
    ms = float(x.item())
    bad = int((eng.pair_status() != 0).sum())
    eng.close()
    if rank != 0:
        return
    line = {"metric": METRIC, "value": wl.n_pairs / ms * 1e3, "unit": "pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "f64+f32" if args.precision != "fp64" else "f64",
            "data": "synthetic (seeded Philox4x32-10 draws, device-resident, each rank its shard)",
            "config": {"workload": wl.name, "pairs": wl.n_pairs, "precision": args.precision,
                       "sharding": "LPT over ranks, pair energies all-gathered in list order",
                       "pairs_rank0": int(len(mine)),
                       "l2": f"inputs {byts / 1e9:.0f} GB >> 129 MB L2, no flush"},
            "tflops": {"fp64": f64 / ms / 1e9, "mixed_part": fmix / ms / 1e9},
            "E_total_raw": total, "pairs_failed_rank0": bad, "clocks": sampler.summary(),
            "gpu_launches": 2 * args.steps, "e2e": None}
    print(json.dumps(line), flush=True)


def run_streamed(args, rank, world, local_rank):
    """Workloads larger than HBM: every step draws each batch's inputs on the
    device and runs the path (and with --backward the adjoint) batch by batch;
    value = pairs/s including the input production."""
    import tempfile

    import torch

    import __graft_entry__
    from paper_2008_03237_gb300.stream import StreamedPairF12
    from synthetic import device
    torch.cuda.set_device(local_rank)
    __graft_entry__.build()
    wl = make_workload(args.workload, args.max_pairs, rank)
    f64, fmix, byts = full_flops(wl) if args.full else flops_bytes(wl)
    fill = device.fill_full if args.full else device.fill

    def produce(b, e, t, lay):
        fill(wl.subset(np.arange(b, e)), t, lay)
    cache = os.path.join(tempfile.gettempdir(), f"pf12_tune_{os.getpid()}.txt")
    sp = StreamedPairF12(args.precision, budget_bytes=args.stream_gb * 1e9, tuner_cache=cache,
                         full=args.full)
    peak = [0]
    total_mem = torch.cuda.mem_get_info()[1]

    def consume(b, e, g, lay):
        peak[0] = max(peak[0], total_mem - torch.cuda.mem_get_info()[0])
    times = []
    sampler = ClockSampler(local_rank)
    for it in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx = sampler if it == args.warmup else _Null()
        with ctx:
            E, e_pair, st = sp.run(wl.n_orb, wl.orb_kind, wl.pi, wl.pj, wl.n_pao, wl.n_pno,
                                   wl.n_aux, produce, backward=args.backward,
                                   grad_consumer=consume if args.backward else None)
            torch.cuda.synchronize()
        peak[0] = max(peak[0], total_mem - torch.cuda.mem_get_info()[0])
        if it >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = float(np.mean(times)) * 1e3
    if rank != 0:
        return
    line = {"metric": METRIC, "value": world * wl.n_pairs / ms * 1e3, "unit": "pairs/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64+f32" if args.precision != "fp64" else "f64",
            "data": "synthetic, drawn on the device batch by batch inside every step",
            "config": {"workload": wl.name, "pairs": wl.n_pairs, "precision": args.precision,
                       "energy": ("complete E_(2)F12 per pair" if args.full
                                  else "amplitude term (1/2 V t of Eq. Vtilde)"),
                       "streamed": True, "batch_budget_gb": args.stream_gb,
                       "batches": len(sp.batches), "backward": bool(args.backward),
                       "inputs_gb": byts / 1e9, "peak_device_gb": peak[0] / 1e9},
            "tflops": {"fp64_forward": f64 / ms / 1e9,
                       "frac_of_fp64_peak": f64 / ms / 1e9 / FP64_PEAK_TFLOPS},
            "overlap": "the next batch is drawn on a side stream while the current one is evaluated",
            "E_total_raw": E, "pairs_failed": int((st != 0).sum()),
            "clocks": sampler.summary(), "e2e": None}
    print(json.dumps(line), flush=True)


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle as it stands, on the host cores."""
    if rank != 0:
        return
    wl = make_workload(args.workload, args.max_pairs)
    wl.meta["bench_name"] = args.workload
    wl.meta["bench_max"] = args.max_pairs
    # the sample's inputs are drawn once; every step times the oracle on it
    budget = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    rates, cores, sample = cpu_oracle_rate(wl, budget, steps=args.warmup + args.steps)
    value = float(np.mean(rates[args.warmup:]))
    line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Philox4x32-10 draws)", "impl": "reference",
            "config": {"workload": wl.name, "pairs": wl.n_pairs, "precision": "fp64"},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                             "cpu_model": cpu_model(),
                             "sample": sample},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
