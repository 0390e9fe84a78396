"""The library's native local search (pp_al_search, host code, no GPU) against
the optimiser oracle (oracle/localsearch.py) on analytic objectives: both run
the same algorithm with the same constants and the same order of every
floating-point operation, so they take the same iterates bit for bit, and
running the starts in lockstep changes nothing."""
import math

import numpy as np
import pytest

from oracle import localsearch as LS

pp = pytest.importorskip("paper_1704_08919_gb300")


@pytest.fixture(scope="module")
def lib():
    from paper_1704_08919_gb300 import build
    build.build()
    return pp.lib()


def rosen_obj(X):
    x, y = X[:, 0], X[:, 1]
    f = 100.0 * (y - x ** 2) ** 2 + (1.0 - x) ** 2
    g = np.stack([-400.0 * x * (y - x ** 2) - 2.0 * (1.0 - x), 200.0 * (y - x ** 2)], axis=1)
    return -f, -g, np.zeros(len(X)), np.zeros_like(X)


# Objectives are written elementwise so that a row's value does not depend on
# how many rows are evaluated together.
def sphere_obj(c, U):
    def obj(X):
        J = X[:, 0] * c[0] + X[:, 1] * c[1] + X[:, 2] * c[2]
        C = U - (X[:, 0] * X[:, 0] + X[:, 1] * X[:, 1] + X[:, 2] * X[:, 2])
        return J, np.tile(c, (len(X), 1)), C, -2.0 * X
    return obj


def circle_obj(X):
    return (X[:, 0] ** 3 - 0.5 * X[:, 1], np.stack([3 * X[:, 0] ** 2, -0.5 + 0 * X[:, 0]], axis=1),
            1.0 - (X[:, 0] * X[:, 0] + X[:, 1] * X[:, 1]), -2.0 * X)


def oracle_run(obj, x0, **kw):
    return LS.augmented_lagrangian(lambda z: tuple(np.asarray(v)[0] for v in obj(z[None, :])), x0, **kw)


def test_rosenbrock_matches_oracle(lib):
    kw = dict(mu0=1.0, xi=0.5, outer=5, max_iter=200, gtol=1e-9, ctol=1e-8)
    r = pp.al_search(np.array([[-1.2, 1.0]]), rosen_obj, **kw)
    o = oracle_run(rosen_obj, np.array([-1.2, 1.0]), **kw)
    assert r["status"][0] == 0 and r["outer"][0] == 1 == o["outer"]
    assert r["evals"][0] == o["evals"]
    assert np.array_equal(r["x"][0], o["x"]) and r["J"][0] == o["J"]
    assert np.abs(r["x"][0] - 1.0).max() < 1e-8


@pytest.mark.parametrize("x0", [[0.3, 0.1, 0.2], [-1.0, 0.5, 2.0]])
def test_sphere_matches_oracle_and_closed_form(lib, x0):
    c, U = np.array([1.0, 2.0, -0.5]), 3.0
    kw = dict(mu0=1.0, xi=0.5, outer=30, max_iter=200, gtol=1e-10, ctol=1e-10)
    r = pp.al_search(np.array([x0]), sphere_obj(c, U), **kw)
    o = oracle_run(sphere_obj(c, U), np.array(x0), **kw)
    assert r["evals"][0] == o["evals"] and r["outer"][0] == o["outer"]
    assert r["lam"][0] == o["lam"] and np.array_equal(r["x"][0], o["x"])
    xs = math.sqrt(U) * c / np.linalg.norm(c)
    assert np.abs(r["x"][0] - xs).max() < 1e-9 and abs(r["C"][0]) <= 1e-10


def test_lockstep_multistart_equals_single_runs(lib):
    starts = np.array([[0.1, -0.95], [-0.2, 0.95], [0.95, -0.2], [0.5, 0.5]])
    kw = dict(mu0=0.1, xi=0.5, outer=30, max_iter=200, gtol=1e-9, ctol=1e-9)
    calls = []

    def counted(X):
        calls.append(len(X))
        return circle_obj(X)
    together = pp.al_search(starts, counted, **kw)
    assert max(calls) == len(starts) and len(calls) < sum(together["evals"])
    for i, x0 in enumerate(starts):
        alone = pp.al_search(x0[None, :], circle_obj, **kw)
        for k in ("x", "J", "C", "lam", "evals", "outer", "status"):
            assert np.array_equal(alone[k][0], together[k][i]), k
        o = oracle_run(circle_obj, x0, **kw)
        assert alone["evals"][0] == o["evals"]
        assert np.array_equal(alone["x"][0], o["x"]) and alone["J"][0] == o["J"]


def test_objective_error_is_reported(lib):
    def bad(X):
        raise ValueError("objective failed")
    with pytest.raises(ValueError):
        pp.al_search(np.zeros((1, 2)), bad)


def test_rejects_bad_options(lib):
    with pytest.raises(pp.PPError):
        pp.al_search(np.zeros((1, 2)), rosen_obj, xi=1.5)
    with pytest.raises(pp.PPError):
        pp.al_search(np.zeros((1, 2)), rosen_obj, mu0=0.0)


def test_native_optimizer_on_the_oracle_qke_objective(lib):
    """On the real objective (the oracle's QKE augmented Lagrangian pieces, evaluated
    row by row) the native optimiser and the oracle's take identical iterates."""
    import oracle
    from paper_1704_08919_gb300 import inputs
    K = 4
    sp = dict(K=K, order=3, w_min=0.0, w_max=2.0, T=20.0, fluence=1.0, n_steps=400)
    grid = inputs.small_grid(3, 3, 2)
    lo, hi, _ = inputs.param_bounds(K)
    X = lo + np.random.default_rng(4).random((2, 4 * K)) * (hi - lo)
    for x in X:
        U0, _ = oracle.fluence_raw(x, K, 3, 0.0, 2.0, 20.0)
        x[:K] *= math.sqrt(1.5 / U0)
        x[2 * K:3 * K] *= math.sqrt(1.5 / U0)

    def row(z):
        o = oracle.al_objective(z, sp, grid, 2.0, 0.0, 1.0, nthreads=1)
        return o["J"], o["gJ"], o["C"], o["gC"]

    def batch(Z):
        rs = [row(z) for z in Z]
        return (np.array([r[0] for r in rs]), np.stack([r[1] for r in rs]),
                np.array([r[2] for r in rs]), np.stack([r[3] for r in rs]))
    kw = dict(mu0=0.1, xi=0.5, outer=2, max_iter=8, gtol=1e-8, ctol=1e-10)
    r = pp.al_search(X, batch, **kw)
    for i in range(2):
        o = LS.augmented_lagrangian(row, X[i], **kw)
        assert r["evals"][i] == o["evals"] and r["outer"][i] == o["outer"]
        assert np.array_equal(r["x"][i], o["x"]) and r["J"][i] == o["J"] and r["lam"][i] == o["lam"]
