"""Pins of the local-search oracle (Sec. IV.A): the un-normalised field and its
time derivative, the fluence and its gradient, the adjoint gradient of the QKE
objective, the chain rule to the B-spline parameters, and the BFGS /
strong-Wolfe / augmented-Lagrangian optimiser -- each against something other
than itself: finite differences, closed forms, exact quadrature, known minimisers."""
import math

import numpy as np
import pytest

import oracle
from oracle import localsearch as LS
from paper_1704_08919_gb300 import inputs

K = 4
SPEC = dict(K=K, order=3, w_min=0.0, w_max=2.0, T=20.0, n_steps=200)
ARGS = (K, 3, 0.0, 2.0, 20.0)


def params(seed, U=2.0):
    """Random parameters with the amplitude weights scaled to fluence U."""
    lo, hi, _ = inputs.param_bounds(K)
    x = lo + np.random.default_rng(seed).random(4 * K) * (hi - lo)
    U0, _ = oracle.fluence_raw(x, *ARGS)
    s = math.sqrt(U / U0)
    x[:K] *= s
    x[2 * K:3 * K] *= s
    return x


def test_raw_field_is_the_normalised_field_unscaled():
    x = params(1)
    A, E, Ed, U = oracle.synth_raw(x, *ARGS, 200)
    An, En, s, rc = oracle.synth_field(x, *ARGS, 7.0, 200)
    assert rc == 0
    assert np.allclose(A * s[:, None, None], An, rtol=0, atol=1e-13 * np.abs(An).max())
    assert np.allclose(E * s[:, None, None], En, rtol=0, atol=1e-13 * np.abs(En).max())


def test_time_derivatives_by_central_differences():
    n = 4000
    x = params(2)
    A, E, Ed, _ = oracle.synth_raw(x, *ARGS, n)
    h = SPEC["T"] / (2 * n)
    dE = (E[0, :, 2:] - E[0, :, :-2]) / (2 * h)
    dA = (A[0, :, 2:] - A[0, :, :-2]) / (2 * h)
    # central differences are second order: error ~ h^2 w^3 |E| / 6
    assert np.abs(dE - Ed[0, :, 1:-1]).max() < 1e-5 * np.abs(Ed).max()
    assert np.abs(dA + E[0, :, 1:-1]).max() < 1e-5 * np.abs(E).max()
    assert np.abs(A[0, :, 0]).max() < 1e-15 and np.abs(A[0, :, -1]).max() < 1e-12


def test_fluence_is_the_exact_period_quadrature():
    """A trigonometric polynomial of degree < N is integrated exactly over its
    period by the N-point rectangle rule, so U = h sum_k |E(t_k)|^2."""
    x = params(3, U=5.0)
    n = 200
    _, E, _, U = oracle.synth_raw(x, *ARGS, n)
    h = SPEC["T"] / (2 * n)
    Uq = h * float(np.sum(E[0, :, :-1] ** 2))
    assert abs(U[0] - 5.0) < 1e-12 * 5
    assert abs(Uq - U[0]) < 1e-11 * U[0]


def test_fluence_gradient_by_finite_differences():
    x = params(4)
    U, dU = oracle.fluence_raw(x, *ARGS)
    for i in range(4 * K):
        e = np.zeros_like(x)
        e[i] = 1e-6
        fd = (oracle.fluence_raw(x + e, *ARGS)[0] - oracle.fluence_raw(x - e, *ARGS)[0]) / 2e-6
        assert abs(fd - dU[i]) < 1e-7 * max(1.0, abs(dU).max())
    assert np.all(dU[K:2 * K] == 0) and np.all(dU[3 * K:] == 0)


def test_rk4_growth_is_rejected():
    """RK4's amplification |1 + z + z^2/2 + z^3/6 + z^4/24| at z = i theta exceeds one
    for theta > 2 sqrt(2): a field far too strong for the step makes chi grow and the
    density is reported as NaN; the same field at a fine step gives a finite density."""
    x = params(5, U=2.0)
    p = np.array([[0.3, -0.2, 0.4]])
    A, E, Ed, _ = oracle.synth_raw(x, *ARGS, 40)
    coarse = oracle.qke6_modes(A[0] * 30, E[0] * 30, Ed[0] * 30, 40, 20.0 / 40, p)
    A, E, Ed, _ = oracle.synth_raw(x, *ARGS, 4000)
    fine = oracle.qke6_modes(A[0], E[0], Ed[0], 4000, 20.0 / 4000, p)
    assert np.isnan(coarse[0]) and 0.0 <= fine[0] <= 2.0


def test_adjoint_mode_matches_forward_solver():
    x = params(5)
    n = 2000
    A, E, Ed, _ = oracle.synth_raw(x, *ARGS, n)
    p = np.array([[0.3, -0.2, 0.4], [0.0, 0.0, 0.0], [-0.7, 0.5, 1.1]])
    fwd = oracle.qke6_modes(A[0], E[0], Ed[0], n, SPEC["T"] / n, p, nthreads=1)
    for m in range(3):
        f, *_ = oracle.qke6_adjoint_mode(A[0], E[0], Ed[0], n, SPEC["T"] / n, p[m])
        assert f == fwd[m]


def test_sample_gradient_by_finite_differences():
    """dJ/d(sample) from the adjoint against central differences of J in single samples."""
    n = 1500
    x = params(6, U=4.0)
    A, E, Ed, _ = oracle.synth_raw(x, *ARGS, n)
    A, E, Ed = A[0], E[0], Ed[0]
    p, w = oracle.grid_modes(inputs.small_grid(3, 2, 2))
    dt = SPEC["T"] / n
    J, _, gA, gE, gEd = oracle.qke6_grad(A, E, Ed, n, dt, p, w, nthreads=2)
    rng = np.random.default_rng(0)
    for arr, g in ((A, gA), (E, gE), (Ed, gEd)):
        for l, k in [(0, 0), (1, 2 * n), (0, 57), (1, 1101), (0, int(rng.integers(0, 2 * n + 1)))]:
            a0 = arr[l, k]

            def cd(h):
                arr[l, k] = a0 + h
                Jp = oracle.qke6_grad(A, E, Ed, n, dt, p, w, nthreads=2)[0]
                arr[l, k] = a0 - h
                Jm = oracle.qke6_grad(A, E, Ed, n, dt, p, w, nthreads=2)[0]
                arr[l, k] = a0
                return (Jp - Jm) / (2 * h)
            fd = (4 * cd(1e-4) - cd(2e-4)) / 3  # Richardson: the h^2 term cancels
            scale = np.abs(g).max()
            assert abs(fd - g[l, k]) < 2e-7 * scale, (l, k, fd, g[l, k])


def test_chain_rule_by_finite_differences():
    """synth_vjp is the transpose of the synthesis Jacobian: for random sample
    weights it equals the gradient of sum(wA A + wE E + wEd Ed)."""
    n = 60
    x = params(7)
    rng = np.random.default_rng(1)
    wA, wE, wD = (rng.normal(size=(2, 2 * n + 1)) for _ in range(3))
    g = oracle.synth_vjp(x, *ARGS, n, wA, wE, wD)

    def F(z):
        A, E, Ed, _ = oracle.synth_raw(z, *ARGS, n)
        return float(np.sum(wA * A[0]) + np.sum(wE * E[0]) + np.sum(wD * Ed[0]))
    for i in range(4 * K):
        e = np.zeros_like(x)
        e[i] = 1e-6
        fd = (F(x + e) - F(x - e)) / 2e-6
        assert abs(fd - g[i]) < 1e-7 * np.abs(g).max(), i


def test_lagrangian_gradient_by_finite_differences():
    x = params(8)
    SPEC = dict(globals()["SPEC"], n_steps=2000)
    grid = inputs.small_grid(3, 3, 2)
    lam, mu, U0 = 0.3, 0.5, 2.5

    def L(z):
        return oracle.al_objective(z, SPEC, grid, U0, lam, mu)
    r = L(x)
    assert abs(r["C"] - 0.5) < 1e-12
    assert abs(r["L"] - (-r["J"] - lam * r["C"] + r["C"] ** 2 / (2 * mu))) < 1e-15
    for i in range(4 * K):
        e = np.zeros_like(x)
        e[i] = 1e-6
        fd = (L(x + e)["L"] - L(x - e)["L"]) / 2e-6
        assert abs(fd - r["grad"][i]) < 1e-7 * np.abs(r["grad"]).max(), i


# ----------------------------------------------------------------------------- optimiser


def rosenbrock(x):
    f = 100.0 * (x[1] - x[0] ** 2) ** 2 + (1.0 - x[0]) ** 2
    g = np.array([-400.0 * x[0] * (x[1] - x[0] ** 2) - 2.0 * (1.0 - x[0]),
                  200.0 * (x[1] - x[0] ** 2)])
    return f, g, None


def test_bfgs_rosenbrock_minimiser():
    r = LS.bfgs(rosenbrock, [-1.2, 1.0], gtol=1e-9)
    assert r["status"] == "converged"
    assert np.abs(r["x"] - 1.0).max() < 1e-8


def test_bfgs_quadratic_solves_the_linear_system():
    rng = np.random.default_rng(2)
    M = rng.normal(size=(8, 8))
    A = M @ M.T + 8 * np.eye(8)
    b = rng.normal(size=8)
    r = LS.bfgs(lambda x: (0.5 * x @ A @ x - b @ x, A @ x - b, None), np.zeros(8), gtol=1e-10)
    assert np.abs(r["x"] - np.linalg.solve(A, b)).max() < 1e-8  # stops near rounding level


@pytest.mark.parametrize("seed", range(5))
def test_line_search_meets_strong_wolfe(seed):
    rng = np.random.default_rng(seed)
    c = np.array([rng.uniform(0.5, 3.0), rng.uniform(1.0, 3.0), rng.uniform(0.1, 0.9)])

    def f1(a):  # a smooth 1-D function with a minimum at positive alpha
        return (c[0] * (a - c[1]) ** 2 + np.sin(c[2] * a), 2 * c[0] * (a - c[1]) + c[2] * np.cos(c[2] * a))
    f0, g0 = f1(0.0)
    assert g0 < 0  # -2 c0 c1 + c2 < 0
    a, fa, _, _, ok = LS.line_search(lambda a: (*f1(a), None), f0, g0, 1.0)
    assert ok
    assert fa <= f0 + LS.C1 * a * g0
    assert abs(f1(a)[1]) <= -LS.C2 * g0


def test_augmented_lagrangian_on_the_sphere():
    """max c.x subject to |x|^2 = U: x* = sqrt(U) c/|c| with multiplier |c| / (2 sqrt(U))."""
    c = np.array([1.0, 2.0, -0.5])
    U = 3.0
    r = LS.augmented_lagrangian(lambda x: (c @ x, c, U - x @ x, -2 * x), np.array([0.3, 0.1, 0.2]),
                                mu0=1.0, xi=0.5, outer=30, gtol=1e-10, ctol=1e-10)
    xs = math.sqrt(U) * c / np.linalg.norm(c)
    assert abs(r["C"]) <= 1e-10
    assert np.abs(r["x"] - xs).max() < 1e-9
    assert abs(r["lam"] / (np.linalg.norm(c) / (2 * math.sqrt(U))) - 1) < 1e-4


def test_multistart_picks_the_best_feasible_run():
    """J = x1^3 - x2/2 on the unit circle has three local maxima (found here by
    brute force over the angle); three starts end at three different ones and the
    multistart keeps the global one."""
    def obj(x):
        J = x[0] ** 3 - 0.5 * x[1]
        return J, np.array([3 * x[0] ** 2, -0.5]), 1.0 - x @ x, -2 * x
    th = np.linspace(0, 2 * np.pi, 2_000_001)
    Jt = np.cos(th) ** 3 - 0.5 * np.sin(th)
    turn = np.diff(np.sign(np.diff(Jt))) < 0
    local = np.sort(Jt[1:-1][turn])
    assert local.size == 3
    starts = [np.array([0.1, -0.95]), np.array([-0.2, 0.95]), np.array([0.95, -0.2])]
    runs, best = LS.multistart(obj, starts, mu0=0.1, xi=0.5, outer=30, gtol=1e-9, ctol=1e-9)
    assert all(abs(r["C"]) <= 1e-9 for r in runs)
    Js = np.sort([r["J"] for r in runs])
    assert np.abs(Js - local).max() < 1e-8
    assert best == 2 and abs(runs[best]["J"] - local[-1]) < 1e-8
