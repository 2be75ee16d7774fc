"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports
every entry point that include/tto.h declares, and rejects invalid grid
descriptions with TTO_E_ARG before it touches a device."""
import os
import re

import numpy as np
import pytest

from paper_2605_10128_b300 import _lib
from synth import config_grid
from tests.gridcases import three_bus

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    syms = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            syms |= set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(tto_[a-z_0-9]+)\s*\(", txt, re.M))
    return syms


def test_library_exports_every_declared_symbol():
    h = _lib.lib()
    syms = declared_symbols()
    assert len(syms) >= 16
    for s in syms:
        assert hasattr(h, s), s
    assert syms <= set(_lib.exported_symbols()) | {"tto_last_error"}


def _create_rc(grid):
    try:
        h = _lib.tto_grid_create(grid)
    except _lib.TTOError as e:
        return e.code, str(e)
    _lib.tto_grid_destroy(h)
    return 0, ""


def test_invalid_grids_rejected_before_device_use():
    g, _ = three_bus()
    bad = []
    x = g.with_limits(g.limit.copy())
    x.b = np.array([1.0, -1.0, 1.0])
    bad.append(x)
    x = g.with_limits(g.limit.copy())
    x.limit = np.array([1.0, 0.0, 1.0])
    bad.append(x)
    x = g.with_limits(g.limit.copy())
    x.from_bus = np.array([0, 1, 1], dtype=np.int32)
    x.to_bus = np.array([1, 2, 1], dtype=np.int32)
    bad.append(x)
    x = g.with_limits(g.limit.copy())
    x.station_bus = np.array([0], dtype=np.int32)  # slack bus
    bad.append(x)
    x = g.with_limits(g.limit.copy())
    x.action_mask = np.array([1] * g.n_action, dtype=np.uint32)  # asset 0 moved
    bad.append(x)
    x = g.with_limits(g.limit.copy())
    x.outages = np.array([0, 0], dtype=np.int32)
    bad.append(x)
    x = g.with_limits(g.limit.copy())
    x.k_max = 9
    bad.append(x)
    for y in bad:
        code, msg = _create_rc(y)
        assert code == _lib.TTO_E_ARG, msg


def test_action_without_branch_on_a_busbar_rejected():
    g = config_grid("tto30")
    g = g.with_limits(np.ones(g.n_branch))
    s = 0
    assets = g.station_assets(s)
    inj = int(np.flatnonzero(assets < 0)[0])
    g.action_mask = g.action_mask.copy()
    g.action_mask[0] = np.uint32(1 << inj)  # busbar B = injection only
    code, msg = _create_rc(g)
    assert code == _lib.TTO_E_ARG and "busbar" in msg
