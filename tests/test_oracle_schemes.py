"""Pins of the oracle's unitary integrators: the second-order split operator
(the paper's integrator, Sec. II.A) and the fourth-order Magnus step (the
higher-order scheme the paper's outlook, Sec. V.C.2, calls for).

Each is tied to things other than itself: unitarity (norm conservation to
1e-12), its convergence order, the Sauter closed form, agreement with the
RK4 oracle at converged step size, and exactness where the scheme is exact.
"""
import math

import numpy as np

import oracle as o
from paper_1704_08919_gb300 import inputs
from tests.test_oracle_pins import sauter_exact, sauter_fields


def _rot_field(ns):
    g = inputs.ROTATING_GAUSSIAN
    dt = (g["t1"] - g["t0"]) / ns
    A, _, _ = o.gaussian_rotating_field(3 * g["E0"], g["w"], g["tau"], g["t0"], dt / 2, 2 * ns + 1)
    return A, dt


P = np.array([[0.3, 0.2, 0.1], [-0.5, 0.4, 0.7], [0.9, -0.6, 0.2]])


def test_split_and_magnus_conserve_the_norm():
    A, dt = _rot_field(4000)
    for fn in (o.dirac_split_modes, o.dirac_magnus_modes):
        f, dev = fn(A, 4000, dt, P)
        assert dev.max() < 1e-12


def test_convergence_orders():
    res = {"split": [], "magnus": []}
    for ns in (500, 1000, 2000):
        A, dt = _rot_field(ns)
        res["split"].append(o.dirac_split_modes(A, ns, dt, P)[0])
        res["magnus"].append(o.dirac_magnus_modes(A, ns, dt, P)[0])
    for name, order in (("split", 2), ("magnus", 4)):
        f = res[name]
        ratio = (f[0] - f[1]) / (f[1] - f[2])
        assert np.all(ratio > 0.9 * 2 ** order), (name, ratio)
        if name == "split":
            assert np.all(np.abs(ratio / 4 - 1) < 0.1), ratio


def test_converge_to_rk4_and_to_the_sauter_closed_form():
    E0, tau, T = 0.25, 5.0, 300.0
    ps = np.array([[0.3, 0.2, 0.1], [-0.5, 0.4, 0.7]])
    ref = np.array([sauter_exact(E0, tau, p) for p in ps])
    ns = 30000
    dt = T / ns
    A, _, _ = sauter_fields(E0, tau, -T / 2, dt / 2, 2 * ns + 1)
    fm, _ = o.dirac_magnus_modes(A, ns, dt, ps)
    assert np.abs(fm / ref - 1).max() < 1e-6
    # second order: Richardson extrapolation of two step sizes reaches the closed form
    fs = []
    for ns in (60000, 120000):
        dt = T / ns
        A, _, _ = sauter_fields(E0, tau, -T / 2, dt / 2, 2 * ns + 1)
        fs.append(o.dirac_split_modes(A, ns, dt, ps)[0])
    # (for tiny n the O(dt^2) mismatch of the end states enters n squared,
    # so the extrapolation is checked where n >= 1e-6 and convergence elsewhere)
    rich = (4 * fs[1] - fs[0]) / 3
    big = ref >= 1e-6
    assert np.abs(rich[big] / ref[big] - 1).max() < 1e-5
    assert np.all(np.abs(fs[1] / ref - 1) < np.abs(fs[0] / ref - 1) / 3.5)
    A, dt = _rot_field(8000)
    fr = o.dirac_modes(A, 8000, dt, P)
    fm, _ = o.dirac_magnus_modes(A, 8000, dt, P)
    assert np.abs(fm / fr - 1).max() < 1e-7


def test_exact_cases():
    # Magnus is exact for a constant Hamiltonian (the commutator vanishes): a
    # constant potential makes no pairs.  The split operator propagates the
    # free Hamiltonian exactly: no field, no pairs; a constant nonzero
    # potential is not exact for it (H_0 and V do not commute).
    ns, dt = 300, 0.07
    A = np.zeros((2, 2 * ns + 1))
    f, _ = o.dirac_split_modes(A, ns, dt, P)
    assert np.abs(f).max() < 1e-28
    A[0], A[1] = 0.4, -0.9
    f, _ = o.dirac_magnus_modes(A, ns, dt, P)
    assert np.abs(f).max() < 1e-28
    f, _ = o.dirac_split_modes(A, ns, dt, P)
    assert f.max() > 1e-20
