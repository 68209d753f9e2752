"""Shared helpers of the GPU tests: seeded inputs, oracle targets, error report."""

from __future__ import annotations

import json
import os

import numpy as np

from phantom import Geometry, Volume

# Tolerances (relative L2 unless stated), as stated for the method's results:
# projections and gradients 1e-4, recovered w 1e-3, tumor position 0.1 mm.
TOL_PROJ = 1e-4
TOL_GRAD = 1e-4
TOL_W = 1e-3
TOL_TUMOR_MM = 0.1


def rel(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def report(name: str, **values):
    """Print the FP64-reference error of a result and append it to the JSON
    report named by PR_PARITY_REPORT (if set)."""
    line = {"case": name}
    for k, v in values.items():
        line[k] = float(v) if np.ndim(v) == 0 else [float(x) for x in np.ravel(v)]
    print("PARITY", json.dumps(line))
    path = os.environ.get("PR_PARITY_REPORT")
    if path:
        with open(path, "a") as fh:
            fh.write(json.dumps(line) + "\n")


def noisy(p: np.ndarray, seed: int, level: float = 0.01) -> np.ndarray:
    """Measured projection: p + level * p * N(0, 1) draws of the given seed."""
    from phantom import standard_normal

    return p + level * p * standard_normal(seed, p.shape)


def random_volume(vol: Volume, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).random(vol.shape)


RAGGED_VOL = Volume(13, 11, 9, 3.0, 3.5, 4.0)
RAGGED_GEOM = Geometry(1000.0, 1500.0, 37, 21, 2.1, 2.7, 1.3)
