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


def test_sparse_overlap_recipe():
    # The densities of Sec. 4.1's overlap matrices, symmetric positive definite, unit diagonal, entries in
    # [0, 1], non-zeros in a band of columns for every block of 128 rows (points ordered by x).
    S, c = W.sparse_overlap(768, W.PAPER_OVERLAP_DENSITY[768], 3)
    assert S.shape == (768, 768) and S.flags.c_contiguous and np.array_equal(S, S.T)
    assert abs(np.count_nonzero(S) / S.size - 0.25) < 1e-3
    assert np.all(np.diag(S) == 1.0) and S.min() >= 0.0 and S.max() <= 1.0
    w = np.linalg.eigvalsh(S)
    assert w.min() > 0 and w.max() / w.min() < 1e3
    S2, c2 = W.sparse_overlap(768, W.PAPER_OVERLAP_DENSITY[768], 3)
    assert np.array_equal(S, S2) and c == c2
    S3, c3 = W.sparse_overlap(1536, W.PAPER_OVERLAP_DENSITY[1536], 3)
    assert abs(np.count_nonzero(S3) / S3.size - 0.124) < 1e-3 and c3 < c + 1.0
    for M, n in ((S, 768), (S3, 1536)):
        nz = M != 0
        spans = [np.ptp(np.nonzero(nz[b:b + 128].any(axis=0))[0]) + 1 for b in range(0, n, 128)]
        assert np.mean(spans) < (0.85 if n == 768 else 0.7) * n
