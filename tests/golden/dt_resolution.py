"""Is the filtered estimator resolved at the prescribed RK4 step dt = 0.05?

Writes tests/golden/dt_resolution.json from the FP64 oracle alone (and the
seeded input generator): for H2 (800 nm, axis along the field) and N2
(1200 nm, cos^2-weighted axis), 2e4 trajectories drawn as R = 10 independent
replicas of 2000, each propagated twice from the same initial points: on the
workloads' grid (dt = 0.05) and on the grid of half the step (the births at
the same times, grid index doubled), the finer dipole read at the coarser
grid's times.  With the workloads' filters (prefactor |C| <= 1e4, stability
taper from max|M| = 1e3 to 2e3) and with the prefactor filter only.

Reported per target and filter setting, all relative L2 against the dt/2
estimate over all 2e4 trajectories:
  change      || v(dt) - v(dt/2) ||, the discretisation change of the estimate;
  change_noise  the replica spread of that paired difference, / sqrt(R): how
                well `change` is resolved;
  sample_noise  the replica spread of the estimate itself, / sqrt(R): the
                Monte Carlo noise of a 2e4-trajectory estimate;
  c_noise, c_change  the same times sqrt(N): noise ~ c / sqrt(N).

    python tests/golden/dt_resolution.py        (a few minutes on 8 cores)
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2608_13686_b300 import workloads as W  # noqa: E402

R, N_REP, SEED = 10, 2000, 31
CASES = [("H2", W.PULSE_800, W.fixed(0.0), "H2, 800 nm 3 cycles 1.5e14 W/cm^2, axis along z"),
         ("N2", W.PULSE_1200, W.COS2, "N2, 1200 nm 3 cycles 1.2e14 W/cm^2, cos^2 axis")]
FILTERS = {"workloads": dict(cutoff=W.CUTOFF, stab_cutoff=W.STAB_CUTOFF, stab_taper=W.STAB_TAPER),
           "prefactor_only": dict(cutoff=W.CUTOFF, stab_cutoff=0.0, stab_taper=0.0)}


def replica_dipoles(t, p, al, filt):
    p2 = dict(p, dt=0.5 * p["dt"])
    coarse, fine = [], []
    for r in range(R):
        soa, _, _ = O.sample(t, p, al, seed=SEED, j_begin=r * N_REP, n=N_REP)
        soa2 = soa.copy()
        soa2[0] = 2 * soa[0]                   # the same birth times on the finer grid
        v1, _, _ = O.propagate(t, p, soa, W.GAMMA, **filt)
        v2, _, _ = O.propagate(t, p2, soa2, W.GAMMA, **filt)
        coarse.append(v1)
        fine.append(v2[::2][: len(v1)])
    return np.array(coarse), np.array(fine)


def main():
    out = {"_about": __doc__.split("\n\n")[0] + " (tests/golden/dt_resolution.py)",
           "replicas": R, "per_replica": N_REP, "seed": SEED, "cases": {}}
    n_all = R * N_REP
    for name, p, al, label in CASES:
        t = W.TARGETS[name]
        case = {"workload": label}
        for fname, filt in FILTERS.items():
            c, f = replica_dipoles(t, p, al, filt)
            ref = np.linalg.norm(f.mean(0))
            d = c - f
            change = np.linalg.norm(d.mean(0)) / ref
            change_noise = np.sqrt(np.sum(d.var(0, ddof=1)) / R) / ref
            noise = np.sqrt(np.sum(f.var(0, ddof=1)) / R) / ref
            case[fname] = {"change": float(change), "change_noise": float(change_noise),
                           "sample_noise": float(noise),
                           "c_noise": float(noise * np.sqrt(n_all)),
                           "c_change": float(change * np.sqrt(n_all)),
                           "change_over_noise": float(change / noise)}
            print(name, fname, json.dumps(case[fname]), flush=True)
        out["cases"][name] = case
    with open(os.path.join(HERE, "dt_resolution.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
