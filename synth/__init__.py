"""Seeded synthetic inputs for DC N-1 topology evaluation.

This package holds input generation only: grid graphs, susceptances, injections,
splittable stations and their action tables, random evaluation batches, and the
recipe that turns already-computed base-case flows into thermal limits.  It
performs no loadflow, no contingency analysis and no fitness arithmetic; those
belong to the method (and to its independent test oracle).
"""
from .grids import (  # noqa: F401
    SynthGrid,
    make_grid,
    limits_from_flows,
    random_topologies,
    CONFIGS,
    config_grid,
)
