"""Frozen-phonon average of the EELS map.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Thermal vibration enters the paper's simulations as frozen phonon passes (Sec. IV A
switches them off for the comparison; Sec. IV D quotes the cost of one pass): each
pass is a full simulation of one configuration of thermally displaced atoms, and the
thermal map is the mean of the passes.  The displaced configurations are inputs
(drawn by the input generator); the average itself is the plain mean.
"""
from __future__ import annotations

import numpy as np

from . import linear as lin


def average_map(configs, scheme: str = "stream"):
    """Mean over configurations of the FP64 map, float64 [n_types][n_sy][n_sx]."""
    acc = None
    for wl in configs:
        m = lin.linear_map(wl, scheme=scheme)
        acc = m if acc is None else acc + m
    return acc / len(configs)
