"""The seeded input recipes: deterministic per seed, inside the ranges their
docstrings state, and of the workloads' shapes."""
import numpy as np

from paper_2510_02639_gb300 import inputs as I


def test_binary_batch_recipe():
    params, t = I.binary_batch()
    params2, t2 = I.binary_batch()
    assert t.shape == (64, 10_000)
    np.testing.assert_array_equal(t, t2)
    assert params == params2
    p3, t3 = I.binary_batch(seed=3)
    assert not np.array_equal(t, t3) and p3[0]["q"] != params[0]["q"]
    q = np.array([p["q"] for p in params])
    s = np.array([p["s"] for p in params])
    rho = np.array([p["rho"] for p in params])
    assert np.all((q >= 1e-5) & (q <= 1e-1)) and np.all((s >= 0.3) & (s <= 3.0))
    assert np.all((rho >= 1e-4) & (rho <= 1e-2))
    assert np.all([abs(p["u0"]) <= 0.1 and 0.3 <= p["u1"] <= 0.8 and 0 <= p["alpha"] < 2 * np.pi
                   and p["tE"] == 20.0 and p["t0"] == 0.0 and p["n_lens"] == 2 for p in params])
    assert np.all(np.diff(t, axis=1) >= 0) and t.min() >= -40.0 and t.max() <= 40.0
    # log-uniform draws spread over the decades, not bunched at one end
    assert np.log10(q).std() > 0.8 and np.log10(rho).std() > 0.4


def test_other_recipes():
    ps, t = I.caustic_crossing_binary()
    assert len(ps) == 1 and t.shape == (1, 500) and ps[0]["q"] == 1e-3 and ps[0]["s"] == 1.0
    pt, tt = I.triple_curve()
    assert tt.shape == (1, 2000) and pt[0]["n_lens"] == 3 and pt[0]["q2"] == 1e-3 and pt[0]["q3"] == 3e-4
    pa, ta, centre, draws = I.adjoint_batch()
    assert ta.shape == (256, 5000) and draws.shape == (256, 5000) and len(pa) == 256
    for k in ("tE", "u0", "alpha", "rho", "u1", "s", "q"):
        rel = np.array([p[k] / centre[k] - 1.0 for p in pa])
        assert np.abs(rel).max() < 0.06 and 0.005 < rel.std() < 0.015, k
    assert abs(draws.std() - 0.01) < 1e-3
    m = I.param_matrix(pa)
    assert m.shape == (256, 8) and m[0, 4] == pa[0]["s"] and m[0, 7] == pa[0]["u1"]


def test_default_grid_is_a_fresh_copy():
    g = I.grid(n_r=128)
    assert g["n_r"] == 128 and I.DEFAULT_GRID["n_r"] == 64
    g["n_theta"] = 1
    assert I.grid()["n_theta"] == 256
