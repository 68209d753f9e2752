"""Checks of the seeded input generator (phantom, breathing DVFs, PCA model)."""

import numpy as np

from phantom import (MU_BODY, MU_LUNG, MU_SPINE, MU_TUMOR, Volume, breathing_phase, build_pca,
                     dvf_analytic, phantom_volume, standard_normal, training_dvfs, tumor_centre,
                     tumor_truth, workload_small)


def test_breathing_phase_endpoints():
    assert breathing_phase(0.0) == 0.0
    assert abs(breathing_phase(2.0) - 1.0) < 1e-15
    assert abs(breathing_phase(1.0) - 0.25) < 1e-15
    assert abs(breathing_phase(4.0)) < 1e-15


def test_reference_phase_has_zero_dvf():
    vol = Volume(16, 16, 16, 4.0, 4.0, 4.0)
    assert np.all(dvf_analytic(vol, 0.0) == 0.0)


def test_phantom_values_and_tumor_site():
    vol = workload_small()["vol"]
    f0 = phantom_volume(vol)
    assert f0.min() == 0.0 and abs(f0.max() - MU_SPINE) < 1e-15
    c0 = tumor_centre(vol)
    idx = np.round((c0 - vol.origin) / vol.spacing).astype(int)
    assert abs(f0[idx[2], idx[1], idx[0]] - MU_TUMOR) < 1e-3  # tumor centre voxel
    assert c0[0] < 0  # patient right is -x
    # lung tissue surrounds the tumor
    assert abs(f0[idx[2], idx[1], idx[0] + 5] - MU_LUNG) < 1e-12
    assert abs(f0[vol.nz // 2, vol.ny // 2, vol.nx // 2] - MU_BODY) < 1e-12


def test_pca_model_normalisation_rank_and_sign():
    vol = Volume(32, 32, 24, 8.0, 8.0, 10.0)
    train = training_dvfs(vol)
    assert train.shape == (9, 3) + vol.shape
    m = build_pca(train, 3)
    n = vol.n
    G = np.array([[np.sum(m.U[a] * m.U[b]) for b in range(3)] for a in range(3)])
    assert np.allclose(G, n * np.eye(3), rtol=1e-10, atol=1e-6 * n)
    assert m.eigvals[2] / m.eigvals[0] > 1e-4  # rank >= 3
    for k in range(3):
        assert m.U[k, 2].sum() >= 0
    # training fields are reproduced to the discarded-eigenvalue level
    recon = m.mean + np.tensordot(m.coeffs, m.U, axes=(1, 0))
    resid = np.sum((recon - train) ** 2)
    assert resid <= 1.0001 * m.eigvals[3:].sum() + 1e-9
    assert np.allclose(m.project(train[4]), m.coeffs[4], atol=1e-10)


def test_tumor_truth_satisfies_pullback_relation():
    vol = workload_small()["vol"]
    p = tumor_truth(vol, 1.0, 1.5)
    d = dvf_analytic(vol, 1.0, 1.5, x=np.array(p[0]), y=np.array(p[1]), z=np.array(p[2])).reshape(3)
    assert np.max(np.abs(p + d - tumor_centre(vol))) < 1e-10


def test_noise_is_seeded():
    a = standard_normal(3, (4, 5))
    assert np.array_equal(a, standard_normal(3, (4, 5)))
    assert not np.array_equal(a, standard_normal(4, (4, 5)))
