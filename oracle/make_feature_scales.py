"""Write the per-column descriptor RMS used to scale the random first layers.

Trained potentials store an input normalisation; these random-init models do
the same with the RMS of each descriptor column over the workload's initial
configuration, computed here with the FP64 oracle (descriptors only, before any
network).  Output: paper_2310_08439_gb300/data/feature_scales.json, a model
statistic read by ``inputs.random_model``.  Run from the repository root:

    python oracle/make_feature_scales.py
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, _ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2310_08439_gb300 import inputs as I  # noqa: E402


def column_rms(model, systems):
    S, Dd = model.n_species, model.n_desc
    om = O.OracleModel(model)
    acc = np.zeros((S, Dd))
    cnt = np.zeros(S)
    for s in systems:
        out = O.evaluate(om, s.pos, s.types, s.box, s.pbc, want_G=True)
        for t in range(S):
            sel = s.types == t
            acc[t] += (out["G"][sel] ** 2).sum(axis=0)
            cnt[t] += sel.sum()
    rms = np.sqrt(acc / np.maximum(cnt, 1)[:, None])
    return rms


def main():
    table = {}
    w = I.tiny(feature_scale=False)
    table["tiny"] = column_rms(w.model, w.systems).ravel().tolist()
    w = I.medium(feature_scale=False)
    table["medium"] = column_rms(w.model, w.systems).ravel().tolist()
    # the 1,048,576-atom cell is too large for the O(N^2) search; an 8^3 cell
    # of the same lattice, spacing and jitter has the same column statistics
    w = I.large(feature_scale=False, reps=8)
    table["large"] = column_rms(w.model, w.systems).ravel().tolist()
    w = I.batch(feature_scale=False)
    table["batch"] = column_rms(w.model, [s for s in w.systems[:64] if s.n <= 3000]).ravel().tolist()
    w = I.serve(feature_scale=False)
    table["serve"] = column_rms(w.model, [s for s in w.systems[:64] if s.n <= 3000]).ravel().tolist()
    out_dir = os.path.join(_ROOT, "paper_2310_08439_gb300", "data")
    os.makedirs(out_dir, exist_ok=True)
    with open(os.path.join(out_dir, "feature_scales.json"), "w") as f:
        json.dump({k: [float(f"{x:.9g}") for x in v] for k, v in table.items()}, f, indent=0)
    print({k: (min(v), max(v)) for k, v in table.items()})


if __name__ == "__main__":
    main()
