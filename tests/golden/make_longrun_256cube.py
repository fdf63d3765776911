"""Writes tests/golden/longrun_256cube.json from the CPU oracle only.

The configuration is the expanding 256^3 lattice: 2 fields with
V = phi^4/4 + (q/2) phi^2 chi^2, q = 1.2, L = 20, dt = 0.02, expansion on,
phi0 = 1, inputs from the shared seeded generator (numpy backend, seed 1),
5000 leapfrog steps of the serial FP64 oracle (arXiv:0712.0813 Sec. III
scheme, with the readings of the oracle's header).

Stored:
  - at step 100: f(t) and f'(t+dt/2) at a fixed, seeded sample of sites, and
    the maximum of |f_i| and |f'_i| over the whole lattice (the denominators of
    the relative max error);
  - at steps 0, 100, 500, 1000, ..., 5000: per-field means and variances, the
    energies K_i, G_i, V, E, the scale factor a(t), a'(t) and the Friedmann
    residual.

The paper prints no values for this run; the file is what the GPU tests and the
benchmark compare the library's long runs against (statistics within 1e-3, the
tolerance stated for chaotic runs).  It takes about two hours on one core.
Run: python tests/golden/make_longrun_256cube.py [--steps 5000] [--out PATH]
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_0712_0813_gb300.icgen import lattice_ics  # noqa: E402

CONFIG = dict(dims=3, N=256, L=20.0, dt=0.02, nf=2, q=[1.2], expansion=True, phi0=1.0, seed=1,
              steps=5000, ic_backend="numpy")
CHECKPOINTS = [0, 100] + list(range(500, 5001, 500))
SAMPLE_STEP = 100


def sample_sites(N: int, n_random: int = 4096, seed: int = 20240) -> list:
    """Seeded random sites plus every combination of the edge coordinates
    {0, 1, N/2 - 1, N/2, N - 2, N - 1} in x, y and z (lattice faces, corners and
    the middle planes, where tiles and z-chunks meet)."""
    rng = np.random.default_rng(seed)
    s = set(int(v) for v in rng.integers(0, N ** 3, size=n_random))
    edges = [0, 1, N // 2 - 1, N // 2, N - 2, N - 1]
    for z in edges:
        for y in edges:
            for x in edges:
                s.add(int(x + N * (y + N * z)))
    return sorted(s)


def statistics(p, st) -> dict:
    en = oracle.energy(st)
    mean, var = oracle.means_variances(p, st.f)
    return {"step": int(st.scale.step), "t": float(st.scale.t), "mean": [float(x) for x in mean],
            "var": [float(x) for x in var], "K": [float(x) for x in en["K"]],
            "G": [float(x) for x in en["G"]], "V": float(en["V"]), "E": float(en["E"]),
            "a": float(en["a"]), "ap": float(en["ap"]), "friedmann_resid": float(en["friedmann_resid"])}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=CONFIG["steps"])
    ap.add_argument("--out", default=os.path.join(HERE, "longrun_256cube.json"))
    args = ap.parse_args()
    c = dict(CONFIG, steps=args.steps)
    p = oracle.Params(dims=c["dims"], N=c["N"], L=c["L"], dt=c["dt"], nf=c["nf"], q=tuple(c["q"]),
                      expansion=c["expansion"])
    f0, u0 = lattice_ics(c["dims"], c["N"], c["L"], c["nf"], phi0=c["phi0"], q=c["q"], seed=c["seed"],
                         backend=c["ic_backend"])
    sites = sample_sites(c["N"])
    t_start = time.time()
    st = oracle.init(p, f0, u0)
    del f0, u0
    out = {"note": "oracle reference values of the expanding 256^3 run; written by "
                   "make_longrun_256cube.py (oracle only)",
           "config": c, "sample_step": SAMPLE_STEP, "sample_sites": sites, "checkpoints": []}

    def dump(done: bool):
        out["complete"] = done
        out["oracle_seconds"] = time.time() - t_start
        tmp = args.out + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(out, fh)
        os.replace(tmp, args.out)

    S = p.S
    cps = [k for k in CHECKPOINTS if k <= c["steps"]]
    for k in cps:
        oracle.step(st, k - st.scale.step)
        out["checkpoints"].append(statistics(p, st))
        if k == SAMPLE_STEP:
            f = st.f.reshape(c["nf"], S)
            v = st.v.reshape(c["nf"], S)
            idx = np.asarray(sites)
            out["samples"] = {"f": [[float(x) for x in f[i, idx]] for i in range(c["nf"])],
                              "v_staggered": [[float(x) for x in v[i, idx]] for i in range(c["nf"])],
                              "f_absmax": [float(np.abs(f[i]).max()) for i in range(c["nf"])],
                              "v_absmax": [float(np.abs(v[i]).max()) for i in range(c["nf"])]}
        dump(False)
        print(f"step {k} done after {time.time() - t_start:.0f} s", flush=True)
    dump(True)


if __name__ == "__main__":
    main()
