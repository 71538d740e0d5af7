"""The seeded generators produce what their recipes state (shape, symmetry, spectrum, determinism)."""
import numpy as np

from paper_1703_02283_gb300 import workloads as W


def test_spd_recipe():
    c = W.spd_from_spectrum(200, 1e-3, 7)
    assert c.A.shape == (200, 200) and c.A.dtype == np.float64 and c.A.flags.c_contiguous
    assert np.array_equal(c.A, c.A.T)
    assert np.linalg.norm(c.Q.T @ c.Q - np.eye(200)) < 1e-12
    assert c.lam[0] == 1.0 and c.lam[-1] == 1e-3 and c.kappa == 1e3
    assert np.all(c.lam >= 1e-3) and np.all(c.lam <= 1.0)
    w = np.linalg.eigvalsh(c.A)
    np.testing.assert_allclose(np.sort(w), np.sort(c.lam), rtol=1e-10, atol=1e-14)
    d = W.spd_from_spectrum(200, 1e-3, 7)
    assert np.array_equal(c.A, d.A)
    assert not np.array_equal(c.A, W.spd_from_spectrum(200, 1e-3, 8).A)


def test_overlap_recipe():
    r = W.overlap_points(100, 20.0, 5000)
    assert r.shape == (100, 3) and r.min() >= 0 and r.max() <= 20.0
    S = W.overlap_matrix(r)
    assert np.array_equal(S, S.T) and np.all(np.diag(S) == 1.0)
    assert np.all(S > 0) and np.all(S <= 1.0)
    assert np.linalg.eigvalsh(S).min() > 0
    r2 = W.jitter_points(r, 0.01, np.random.default_rng(1))
    assert 0 < np.abs(r2 - r).max() < 0.1


def test_batched_specs():
    b = W.batched_specs(512)
    assert len(b.n) == 512 and b.n.min() >= 64 and b.n.max() <= 1024
    assert set(np.unique(b.p)) <= {1, 2, 3}
    assert np.all(b.lam_min <= 0.1 + 1e-12) and np.all(b.lam_min >= 1e-4 - 1e-18)
    assert b.seeds[0] == 1000 and b.seeds[-1] == 1511
