"""Comparison of library outputs with the FP64 oracle.

Tolerance: post-contingency loadings within TOL of each branch's thermal limit,
TOL = 1e-4 for the FP32 sweep and 1e-3 when the low-rank term runs in BF16 on
the tensor cores, plus FLOW_ULPS = 2^-20 (16 FP32 ulps) of the flow itself:
|fmax_gpu - fmax_oracle| <= TOL * limit + FLOW_ULPS * |fmax_oracle|.  The flows
are FP32 by design; for a post-contingency flow far above its limit (hundreds
of times it, as in the 2000-bus batch) one FP32 ulp of the flow is already tens
of millionths of the limit, so the absolute bar alone would test FP32's
representation, not the method.  Near the limit, where overloads are decided,
the second term is below 1e-6 of the limit.  Islanding flags, descriptors and
cells must match bit for bit.  Critical-branch counts may differ only where the
oracle's loading sits within the tolerance band of the limit.
"""
import os

import numpy as np

from oracle import dcflow

TOL_FP32 = 1e-4
TOL_BF16 = 1e-3
FLOW_ULPS = 2.0 ** -20


def n_procs():
    return max(1, min(16, os.cpu_count() or 1))


def oracle_eval(grid, topo, idx, timesteps=None, d_split=8, d_moved=8, d_disc=1):
    return dcflow.evaluate_many(grid, [topo[i] for i in idx], processes=min(n_procs(), len(idx)),
                                timesteps=timesteps, d_split=d_split, d_moved=d_moved, d_disc=d_disc)


def split_report(split, tol):
    return (f"near the limit (|F| <= 2 limit, {split['n_near']} entries) {split['near']:.2e} of limit "
            f"(plain bar {tol:.0e}); beyond ({split['n_far']} entries) {split['far']:.2e}, "
            f"{split['far_over_plain']} above the plain bar")


def compare(grid, out, idx, refs, tol=TOL_FP32, fitness_kind=0, split=None):
    """Assert parity for sampled batch indices; returns the largest loading
    error in units of the thermal limit.  ``split`` (a dict) collects the error
    in two parts: loadings within twice the limit (where overloads are
    decided; there the flow-scaled term is below 2^-19 of the limit, so the
    bar is the plain tol * limit) and the flows beyond that, with the number
    of entries that pass only thanks to the flow-scaled term."""
    lim = grid.limit[grid.monitored.astype(np.int64)]
    worst = 0.0
    if split is not None:
        split.setdefault("near", 0.0)
        split.setdefault("far", 0.0)
        split.setdefault("n_near", 0)
        split.setdefault("n_far", 0)
        split.setdefault("far_over_plain", 0)
    for i, r in zip(idx, refs):
        isl = int(out["island"][i])
        assert (isl & 1) == (1 if r["island_base"] else 0), f"base islanding differs at {i}"
        assert int(out["cell"][i]) == r["cell"], f"cell differs at {i}"
        assert tuple(int(x) for x in out["desc"][i]) == (r["ns"], r["nm"])
        if r["island_base"]:
            assert out["fitness"][i] == -np.inf
            continue
        assert ((isl >> 1) & 1) == (1 if r["island_any"] else 0), f"outage islanding differs at {i}"
        fm = out["fmax"][i].astype(np.float64)
        err = np.abs(fm - r["fmax"]) / lim[None, :]
        worst = max(worst, float(err.max()))
        allowed = tol + FLOW_ULPS * np.abs(r["fmax"]) / lim[None, :]
        assert np.all(err <= allowed), (f"topology {i}: fmax error {err.max():.3e} of limit, "
                                        f"{float((err / allowed).max()):.2f} of the allowed")
        if split is not None:
            near = np.abs(r["fmax"]) <= 2.0 * lim[None, :]
            split["near"] = max(split["near"], float(err[near].max(initial=0.0)))
            split["far"] = max(split["far"], float(err[~near].max(initial=0.0)))
            split["n_near"] += int(near.sum())
            split["n_far"] += int((~near).sum())
            split["far_over_plain"] += int((err[~near] > tol).sum())
        lam_o = r["lambda_o"]
        n = r["fmax"].size
        m = out["metrics"][i]
        band = tol * lim[None, :] + FLOW_ULPS * np.abs(r["fmax"])
        assert abs(m[0] - lam_o) <= (band.sum() + 1e-5 * abs(lam_o) + 1e-6), (i, m[0], lam_o)
        assert abs(m[1] - r["maxload"]) <= tol + 1e-6 * r["maxload"], (i, m[1], r["maxload"])
        near = int((np.abs(r["fmax"] - lim[None, :]) <= band).sum())
        assert abs(int(m[2]) - r["lambda_c"]) <= near, (i, m[2], r["lambda_c"], near)
        band0 = tol * lim[None, :] + FLOW_ULPS * np.abs(r["fprime"])
        near0 = int((np.abs(np.abs(r["fprime"]) - lim[None, :]) <= band0).sum())
        assert abs(int(m[3]) - r["lambda_c0"]) <= near0, (i, m[3], r["lambda_c0"])
        if fitness_kind == 0:
            ref = r["fitness"]
            bound = band.sum() + tol + 1e-5 * abs(ref) + 1e-6
        else:
            ref = r["lambda_f1"]
            bound = band.sum() + 50.0 * near + 200.0 * near0 + 1e-5 * abs(ref) + 1e-6
        assert abs(float(out["fitness"][i]) - ref) <= bound, (i, out["fitness"][i], ref)
        del n
    return worst
