"""The seeded generators produce the workload shapes they claim."""
import numpy as np
import pytest

import synth


def _site_changes(s):
    d = (s["qB"].astype(np.float64) - s["qA"].astype(np.float64))
    K = len(s["lam"])
    return np.array([d[s["site"] == k].sum() for k in range(K)])


def test_small_open():
    s = synth.small_open()
    assert s["x"].shape == (1000, 3) and s["x"].dtype == np.float32
    assert not s["periodic"] and s["L"] == 4.0 and (s["p"], s["depth"]) == (8, 2)
    assert s["qA"].sum() == 0 and set(np.unique(s["qA"])) == {-1.0, 1.0}
    assert (s["x"] >= 0).all() and (s["x"] < 4).all()
    assert len(s["lam"]) == 10 and np.bincount(s["site"][s["site"] >= 0]).tolist() == [4] * 10
    np.testing.assert_allclose(_site_changes(s), -1.0, atol=1e-6)
    # non-site atoms have identical forms
    assert (s["qA"][s["site"] < 0] == s["qB"][s["site"] < 0]).all()


def test_solvated_30k():
    s = synth.solvated_30k()
    assert s["x"].shape == (29000, 3) and s["periodic"] and s["L"] == 6.5
    assert abs(float(s["qA"].astype(np.float64).sum())) < 1e-4
    np.testing.assert_allclose(_site_changes(s), -1.0, atol=1e-5)
    assert len(s["lam"]) == 20
    assert synth.oxygen_min_distance(s) >= synth.OO_MIN
    # water geometry
    O = s["x"][2000::3].astype(np.float64); H1 = s["x"][2001::3].astype(np.float64)
    d = H1 - O
    d -= s["L"] * np.round(d / s["L"])
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), synth.OH_BOND, atol=2e-6)


def test_deterministic():
    a = synth.small_open(seed=0)
    b = synth.small_open(seed=0)
    for k in ("x", "qA", "qB", "site", "lam"):
        np.testing.assert_array_equal(a[k], b[k])


@pytest.mark.slow
def test_solvated_500k_shape():
    s = synth.solvated_500k()
    assert s["x"].shape == (500000, 3) and s["L"] == 17.0 and (s["p"], s["depth"]) == (10, 5)
    assert len(s["lam"]) == 200
    np.testing.assert_allclose(_site_changes(s), -1.0, atol=1e-5)


def test_tautomer_sites_forms():
    s = synth.tautomer_sites(synth.periodic_uniform(seed=5, n=500, L=2.0, n_sites=6, site_size=4), seed=2,
                             tautomer_fraction=0.5)
    K = 6
    assert s["forms"] == 4 and s["lam"].shape == (2 * K,) and s["lam"].dtype == np.float32
    assert np.array_equal(s["qC"], s["qD"])
    for k in range(K):
        g = s["site"] == k
        assert abs(float(s["qA"][g].astype(np.float64).sum() - s["qB"][g].astype(np.float64).sum())) < 1e-5
        assert abs(float(s["qC"][g].astype(np.float64).sum() - s["qA"][g].astype(np.float64).sum()) + 1.0) < 1e-5
    out = ~(s["site"] >= 0)
    assert np.array_equal(s["qA"][out], s["qB"][out])
