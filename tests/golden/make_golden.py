"""Writes tiny_oracle.json: oracle pair energies of the tiny 7 DOMO + 1 SOMO
workload (36 pairs, p = 30, k ~ U[8,16], m ~ U[60,120]), and
tiny_aug_oracle.json: the same list in the SOMO-augmented PNO space.  Calls
only oracle/ and synthetic/.  Run from the repository root:
python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O          # noqa: E402
import synthetic as S       # noqa: E402


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    for wl, name in ((S.tiny(), "tiny_oracle.json"), (S.tiny().augmented(), "tiny_aug_oracle.json")):
        r = O.run(wl)
        out = {"workload": wl.name, "n_pairs": wl.n_pairs, "E": r["E"],
               "e_pair": r["e_pair"].tolist(), "d": r["d"].tolist(), "x": r["x"].tolist(),
               "sum_abs": r["sum_abs"]}
        with open(os.path.join(here, name), "w") as fh:
            json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
