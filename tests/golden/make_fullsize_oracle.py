"""Writes <workload>_oracle.npz in this directory: the FP64 oracle's pair
energies (e_pair, n_pairs x 3), contractions d, x and the pair-order total E
for every pair of a workload.  Calls only oracle/ and synthetic/; pairs are
spread over a spawn process pool with one BLAS thread per process.

    python tests/golden/make_fullsize_oracle.py c40h81 c160h321 [--procs N]
"""
import argparse
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))


def _chunk(args):
    name, pairs = args
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle
    import synthetic as S
    wl = S.WORKLOADS[name]()
    out = np.zeros((len(pairs), 5))
    for n, P in enumerate(pairs):
        i, j = int(wl.pi[P]), int(wl.pj[P])
        f = oracle.pair_forward(S.pair_inputs(wl, P), int(wl.orb_kind[i]), int(wl.orb_kind[j]), i == j)
        out[n, :3] = f["e"]
        out[n, 3], out[n, 4] = f["d"], f["x"]
    return pairs, out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workloads", nargs="+")
    ap.add_argument("--procs", type=int, default=os.cpu_count())
    a = ap.parse_args()
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    os.environ["OMP_NUM_THREADS"] = "1"
    import multiprocessing as mp
    import numpy as np
    sys.path.insert(0, ROOT)
    import oracle
    import synthetic as S
    ctx = mp.get_context("spawn")
    for name in a.workloads:
        t0 = time.time()
        n = S.WORKLOADS[name]().n_pairs
        chunks = [(name, list(range(s, min(n, s + 16)))) for s in range(0, n, 16)]
        res = np.zeros((n, 5))
        with ctx.Pool(a.procs) as pool:
            for pairs, out in pool.imap_unordered(_chunk, chunks):
                res[pairs] = out
        e_pair = res[:, :3]
        E = 0.0
        for P in range(n):
            E += e_pair[P, 0] + e_pair[P, 1] + e_pair[P, 2]
        np.savez_compressed(os.path.join(HERE, f"{name}_oracle.npz"), e_pair=e_pair, d=res[:, 3],
                            x=res[:, 4], E=E, E_kahan=oracle.kahan_total(e_pair),
                            sum_abs=float(np.abs(e_pair.sum(axis=1)).sum()))
        print(f"{name}: {n} pairs, E = {E!r}, {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
