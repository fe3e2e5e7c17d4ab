"""Shared helpers of the GPU parity tests: run the same seeded problem through
the CUDA library (via the C-ABI binding) and through the FP64 oracle, and
compare element by element."""
from __future__ import annotations

import numpy as np

# Bar of the FP32 path: max-abs distribution difference after 1000 steps.
TOL_POPS = 1e-5
TOL_AUX = 1e-5


def gpu_run(params_list, fields, steps, storage=0):
    from paper_2403_16122_gb300 import lbm

    lat = lbm.Lattice(params_list, storage=storage)
    for k, (phi0, T0) in enumerate(fields):
        lat.init(phi0, T0, inst=k)
    if steps:
        lat.step(steps)
    return lat


def oracle_run(oracle_mod, p, phi0, T0, steps):
    o = oracle_mod.Oracle(p).init(phi0, T0)
    if steps:
        o.step(steps)
    return o


def max_abs(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max())


def compare_state(gpu_state, oracle_state, tol_pops=TOL_POPS, tol_aux=TOL_AUX):
    gp, ga = gpu_state
    op, oa = oracle_state
    assert np.isfinite(gp).all() and np.isfinite(ga).all()
    d = {
        "g": max_abs(gp[0:9], op[0:9]),
        "h": max_abs(gp[9:18], op[9:18]),
        "f": max_abs(gp[18:27], op[18:27]),
        "fs": max_abs(ga[0], oa[0]),
        "phiu": max_abs(ga[1:3], oa[1:3]),
        "p": max_abs(ga[3], oa[3]),
        "S": max_abs(ga[4], oa[4]),
    }
    worst_pop = max(d["g"], d["h"], d["f"])
    worst_aux = max(d["fs"], d["phiu"], d["p"], d["S"])
    assert worst_pop <= tol_pops, d
    assert worst_aux <= tol_aux, d
    return d
