import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU case")


@pytest.fixture(scope="session")
def small_case():
    """The 64^3 / 128x128 workload: phantom, K=3 PCA model, 1.5x test field at t = 1 s."""
    import numpy as np

    from phantom import (build_pca, dvf_analytic, phantom_volume, training_dvfs, tumor_centre,
                         workload_small)

    w = workload_small()
    vol = w["vol"]
    f0 = phantom_volume(vol)
    pca = build_pca(training_dvfs(vol), w["K"])
    x_test = dvf_analytic(vol, w["t"], w["scale"])
    return dict(w, f0=f0, pca=pca, x_test=x_test, c0=tumor_centre(vol),
                angle=np.deg2rad(w["angle_deg"]))
