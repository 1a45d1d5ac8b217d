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


def test_charge_buffer_variant():
    """Sec. 2.5's charge buffers: every site owns one water oxygen whose charge goes from
    -0.834 to +0.166 e with the site's lambda, so each site's net change is 0 and the box is
    neutral at every lambda; the buffer is 2 nm or more from every cluster atom and about 3 nm
    from its site (minimum image)."""
    s = synth.solvated_30k_buf()
    base = synth.solvated_30k()
    assert s["x"].shape == base["x"].shape and np.array_equal(s["x"], base["x"])
    np.testing.assert_allclose(_site_changes(s), 0.0, atol=1e-5)
    K = len(s["lam"])
    for lam in (np.zeros(K), np.ones(K), np.random.default_rng(3).uniform(-0.1, 1.1, K)):
        w = np.where(s["site"] >= 0, lam[np.maximum(s["site"], 0)], 0.0)
        q = s["qA"].astype(np.float64) + w * (s["qB"].astype(np.float64) - s["qA"].astype(np.float64))
        assert abs(q.sum()) < 1e-4
    L, ns = s["L"], s["n_solute"]
    x = s["x"].astype(np.float64)
    new = np.nonzero((s["site"] >= 0) & (base["site"] < 0))[0]
    assert len(new) == K and len(np.unique(s["site"][new])) == K
    assert (new >= ns).all() and ((new - ns) % 3 == 0).all()  # water oxygens
    assert np.allclose(s["qA"][new], synth.BUFFER_QA) and np.allclose(s["qB"][new], synth.BUFFER_QB)
    for i in new:
        d = x[:ns] - x[i]
        d -= L * np.round(d / L)
        assert np.sqrt((d * d).sum(1)).min() >= 2.0
        g = np.nonzero(base["site"] == s["site"][i])[0]
        r = x[g] - x[g[0]]
        r -= L * np.round(r / L)
        c = x[g[0]] + r.mean(0) - x[i]
        c -= L * np.round(c / L)
        assert abs(np.linalg.norm(c) - 3.0) < 0.2
