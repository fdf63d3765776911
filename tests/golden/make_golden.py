"""Writes tests/golden/oracle_regression.json from the CPU oracle only.

The paper (arXiv:0712.0813) prints no numerical example, so the stored values
are regression anchors for the oracle itself: they change only if the oracle's
arithmetic changes, and such a change must cite the passage that justifies it.
Inputs come from the shared seeded generator.  Run: python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_0712_0813_gb300.icgen import lattice_ics  # noqa: E402

CASES = [
    # 32^3, 2 fields, no expansion, L=20, dt=0.05, phi0=1, q=1.2 (the plain FP64 case)
    dict(name="32cube_plain", dims=3, N=32, L=20.0, dt=0.05, nf=2, q=[1.2], expansion=False, steps=100, seed=1),
    # the same lattice with expansion on
    dict(name="32cube_expanding", dims=3, N=32, L=20.0, dt=0.05, nf=2, q=[1.2], expansion=True, steps=100, seed=1),
    # 2D, 4 fields, expansion
    dict(name="2d_4field", dims=2, N=48, L=20.0, dt=0.02, nf=4, q=[0.8, 5.0, 40.0], expansion=True, steps=200, seed=2),
]
SAMPLE_SITES = [0, 1, 7, 1000, 2303]


def run_case(c):
    p = oracle.Params(dims=c["dims"], N=c["N"], L=c["L"], dt=c["dt"], nf=c["nf"],
                      q=tuple(c["q"]), expansion=c["expansion"])
    f0, u0 = lattice_ics(c["dims"], c["N"], c["L"], c["nf"], phi0=1.0, q=c["q"], seed=c["seed"])
    st = oracle.init(p, f0, u0)
    oracle.step(st, c["steps"])
    en = oracle.energy(st)
    mean, var = oracle.means_variances(p, st.f)
    S = p.S
    f = st.f.reshape(c["nf"], S)
    v = st.v.reshape(c["nf"], S)
    return {
        "K": list(en["K"]), "G": list(en["G"]), "V": en["V"], "E": en["E"],
        "a": en["a"], "ap": en["ap"], "friedmann_resid": en["friedmann_resid"],
        "mean": list(mean), "var": list(var),
        "f_samples": [[float(f[i, s]) for s in SAMPLE_SITES] for i in range(c["nf"])],
        "v_samples": [[float(v[i, s]) for s in SAMPLE_SITES] for i in range(c["nf"])],
    }


def main():
    out = {"note": "oracle regression anchors; written by make_golden.py (oracle only)",
           "sample_sites": SAMPLE_SITES, "cases": []}
    for c in CASES:
        out["cases"].append({"config": c, "result": run_case(c)})
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
