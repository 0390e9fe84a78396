"""Pins of the Hann-envelope synthesis of the oracle (Eqs. (hann), (field),
(vector_potential)): the envelope closes the field at both ends, the potential
is the paper's closed form in the gauge A(t_f) = 0, and it equals the integral of
E computed independently; dE/dt and the fluence are checked the same way."""
import numpy as np
import pytest

import oracle
from paper_1704_08919_gb300 import inputs

K, ORDER, T = 8, 4, 50.0


def fields(n, normalize=True, seed=3, U=2.0):
    x = inputs.random_population(2, K, seed=seed)
    return oracle.synth_hann(x, K, ORDER, 0.0, 2.0, T, U, n, normalize=normalize)


def test_envelope_closes_the_field_and_fixes_the_gauge():
    A, E, Ed, _ = fields(4000)
    assert np.abs(E[:, :, [0, -1]]).max() < 1e-15 * np.abs(E).max()
    assert np.abs(Ed[:, :, [0, -1]]).max() < 1e-12 * np.abs(Ed).max()  # g'(+-T/2) = 0 too
    assert np.all(A[:, :, -1] == 0.0)
    assert np.abs(A[:, :, 0]).max() > 1e-3  # the enveloped field has a DC part: A(t_i) != 0


def test_potential_is_the_integral_of_E():
    """A(t) = int_t^{t_f} E dt', by Simpson's rule on the oracle's own E samples (fine grid)."""
    n = 20000
    A, E, _, _ = fields(n)
    h = T / (2 * n)
    for c in range(2):
        for l in range(2):
            e = E[c, l]
            # integrate from the right end, two half-steps (one Simpson panel) at a time
            acc = np.zeros(n + 1)
            for p in range(n - 1, -1, -1):
                acc[p] = acc[p + 1] + h / 3 * (e[2 * p] + 4 * e[2 * p + 1] + e[2 * p + 2])
            assert np.abs(A[c, l, ::2] - acc).max() < 1e-10 * np.abs(A[c, l]).max()


def test_time_derivatives_converge_at_second_order():
    errs = []
    for n in (2000, 4000):
        A, E, Ed, _ = fields(n)
        h = T / (2 * n)
        dA = (A[:, :, 2:] - A[:, :, :-2]) / (2 * h)
        dE = (E[:, :, 2:] - E[:, :, :-2]) / (2 * h)
        errs.append((np.abs(dA + E[:, :, 1:-1]).max(), np.abs(dE - Ed[:, :, 1:-1]).max()))
    for i in range(2):
        assert 3.5 < errs[0][i] / errs[1][i] < 4.5  # central differences: h^2
    assert errs[1][0] < 2e-5 * np.abs(E).max() and errs[1][1] < 2e-5 * np.abs(Ed).max()


def test_fluence_is_normalised_on_any_fine_grid():
    """E^2 is a trigonometric polynomial: the rectangle rule over one period is exact on
    every grid fine enough, so a grid of another size gives the same fluence."""
    for n in (1500, 2100):
        _, E, _, s = fields(n)
        h = T / (2 * n)
        U = h * np.sum(E[:, :, :-1] ** 2, axis=(1, 2))
        assert np.abs(U - 2.0).max() < 1e-12
    _, _, _, U1 = fields(1500, normalize=False)
    _, _, _, U2 = fields(2100, normalize=False)
    assert np.abs(U1 / U2 - 1).max() < 1e-12


def test_unit_envelope_limit_is_not_the_hann_field():
    """The envelope changes the field (it is not a relabelling of g = 1)."""
    x = inputs.random_population(1, K, seed=5)
    _, E0, _, rc = oracle.synth_field(x, K, ORDER, 0.0, 2.0, T, 2.0, 1000)
    _, E1, _, _ = oracle.synth_hann(x, K, ORDER, 0.0, 2.0, T, 2.0, 1000)
    assert rc == 0
    assert np.abs(E1[0, :, 1000] / E0[0, :, 1000]).max() != pytest.approx(1.0)


def test_chain_rule_and_fluence_gradient_by_finite_differences():
    """synth_vjp_hann is the transpose of the Hann synthesis Jacobian (random sample
    weights), and dU is the gradient of the fluence."""
    n = 300
    x = inputs.random_population(1, K, seed=7)[0] * 0.3
    rng = np.random.default_rng(2)
    wA, wE, wD = (rng.normal(size=(2, 2 * n + 1)) for _ in range(3))
    g, U, dU = oracle.synth_vjp_hann(x, K, ORDER, 0.0, 2.0, T, n, wA, wE, wD)

    def F(z):
        A, E, Ed, Uz = oracle.synth_hann(z[None], K, ORDER, 0.0, 2.0, T, 1.0, n, normalize=False)
        return float(np.sum(wA * A[0]) + np.sum(wE * E[0]) + np.sum(wD * Ed[0])), Uz[0]
    assert abs(F(x)[1] - U) < 1e-13 * U
    for i in range(4 * K):
        e = np.zeros_like(x)
        e[i] = 1e-6
        (fp, up), (fm, um) = F(x + e), F(x - e)
        assert abs((fp - fm) / 2e-6 - g[i]) < 1e-7 * np.abs(g).max(), i
        assert abs((up - um) / 2e-6 - dU[i]) < 1e-7 * max(np.abs(dU).max(), 1e-12), i


def test_lagrangian_gradient_with_the_envelope():
    import math
    k, n, T2 = 4, 2000, 20.0
    sp = dict(K=k, order=3, w_min=0.0, w_max=2.0, T=T2, fluence=1.0, n_steps=n, envelope=1)
    x = inputs.random_population(1, k, seed=6)[0]
    _, _, _, U0 = oracle.synth_hann(x, k, 3, 0.0, 2.0, T2, 1.0, n, normalize=False)
    s = math.sqrt(1.5 / U0[0])
    x[:k] *= s
    x[2 * k:3 * k] *= s
    grid = inputs.small_grid(3, 3, 2)
    r = oracle.al_objective(x, sp, grid, 2.0, 0.3, 0.5)
    assert abs(r["C"] - 0.5) < 1e-12
    for i in range(4 * k):
        e = np.zeros_like(x)
        e[i] = 1e-5
        fd = (oracle.al_objective(x + e, sp, grid, 2.0, 0.3, 0.5)["L"]
              - oracle.al_objective(x - e, sp, grid, 2.0, 0.3, 0.5)["L"]) / 2e-5
        assert abs(fd - r["grad"][i]) < 1e-7 * np.abs(r["grad"]).max(), i
