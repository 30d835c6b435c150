"""Writes oracle_regression.json from the CPU oracle only.

    python tests/golden/make_oracle_golden.py

The stored digests pin the oracle against unintended changes; a change of its
arithmetic must regenerate this file in the same commit and name the passage
of the paper (or the reading of it) that justifies the change.
"""
import hashlib
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2103_14737_gb300 import synth  # noqa: E402

CASES = {
    "single_e65_4ev_seed1": dict(parts=lambda: synth.single_particle(4), seed=1, first_event=0),
    "ttbar400_seed1": dict(parts=lambda: synth.ttbar_like(1, 1), seed=1, first_event=0),
}


def digest(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()[:32]


def compute():
    geo = synth.geometry()
    prm = synth.params(geo)
    og, op = O.OracleGeometry(geo), O.OracleParams(prm)
    out = {}
    for name, c in CASES.items():
        r = O.simulate(og, op, c["parts"](), seed=c["seed"], first_event=c["first_event"])
        out[name] = dict(
            n_tasks=r.n_tasks, n_hits=r.n_hits,
            task_n=digest(r.task_n.astype(np.int32)),
            task_Ehit=digest(r.task_Ehit.astype(np.float32)),
            cells_canon=digest(r.cells_canon.astype(np.float32)),
            nnz=int(np.count_nonzero(r.cells64)),
            sum_cells64=float(r.cells64.sum()),
        )
    return out


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_regression.json")
    with open(path, "w") as f:
        json.dump(compute(), f, indent=1, sort_keys=True)
    print("wrote", path)
