"""Small grids shared by the tests (inputs only; no method arithmetic)."""
import json
import os

import numpy as np

from synth.grids import SynthGrid, make_grid, INJECTION

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def three_bus():
    with open(os.path.join(GOLDEN, "three_bus.json")) as fh:
        d = json.load(fh)
    gd = d["grid"]
    st = d["station"]
    assets = st["assets"]
    m = len(assets)
    masks = []
    for mm in range(1, 1 << (m - 1)):
        mask = mm << 1
        if any((mask >> i) & 1 and assets[i] >= 0 for i in range(m)):
            masks.append(mask)
    g = SynthGrid(
        name="three_bus", n_bus=gd["n_bus"], from_bus=np.array(gd["from"], dtype=np.int32),
        to_bus=np.array(gd["to"], dtype=np.int32), b=np.array(gd["b"], dtype=np.float64),
        slack=gd["slack"], p=np.array(gd["p"], dtype=np.float64),
        limit=np.array(gd["limit"], dtype=np.float64),
        monitored=np.arange(3, dtype=np.int32), outages=np.arange(3, dtype=np.int32),
        station_bus=np.array([st["bus"]], dtype=np.int32),
        asset_offset=np.array([0, m], dtype=np.int32),
        asset_branch=np.array(assets, dtype=np.int32),
        action_offset=np.array([0, len(masks)], dtype=np.int32),
        action_station=np.zeros(len(masks), dtype=np.int32),
        action_mask=np.array(masks, dtype=np.uint32), k_max=1)
    return g, d


def small_grid(seed, n_bus=12, n_branch=22, n_station=4, T=2, k_max=3, assets=(4, 7)):
    g = make_grid(n_bus, n_branch, n_station, assets=assets, T=T,
                  b_dist=("uniform", 5.0, 50.0), noise=0.1 if T > 1 else 0.0, seed=seed,
                  k_max=k_max, name=f"small{seed}", knn=5)
    return g


def action_of(grid, station, mask):
    lo, hi = grid.action_offset[station], grid.action_offset[station + 1]
    for a in range(lo, hi):
        if int(grid.action_mask[a]) == mask:
            return a
    raise KeyError(mask)


__all__ = ["three_bus", "small_grid", "action_of", "INJECTION"]
