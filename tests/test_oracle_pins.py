"""Pins of the FP64 CPU oracle to things other than itself.

Each test ties one oracle routine to what the paper or the mathematics fixes:
values printed by the paper (tests/golden), closed forms (Sauter pulse,
complex error function), an independent formalism (the 6-component kinetic
equation of Sec. II.B), first-order perturbation theory, exact symmetries,
library routines (scipy's B-splines) and the RK4 convergence order.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as o
from paper_1704_08919_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

SX = np.array([[0, 1], [1, 0]], complex)
SY = np.array([[0, -1j], [1j, 0]])
SZ = np.diag([1.0, -1.0]).astype(complex)


def dirac_h(P):
    """H = alpha.P + beta in the Dirac representation, built independently of the oracle."""
    al = [np.kron(SX, s) for s in (SX, SY, SZ)]
    beta = np.kron(SZ, np.eye(2))
    return al[0] * P[0] + al[1] * P[1] + al[2] * P[2] + beta


# --------------------------------------------------------------------------- B-splines


@pytest.mark.parametrize("K,order", [(5, 3), (8, 4), (10, 3), (16, 4), (6, 2), (4, 4)])
def test_bspline_partition_of_unity_and_positivity(K, order):
    # Sec. III: B-splines are non-negative; with clamped knots they sum to one on [w_min, w_max].
    for w in np.linspace(0.3, 2.1, 181):
        B = o.bspline_basis(K, order, 0.3, 2.1, w)
        assert np.all(B >= 0.0)
        assert abs(B.sum() - 1.0) < 1e-14


@pytest.mark.parametrize("K,order", [(5, 3), (8, 4), (10, 3), (16, 4)])
def test_bspline_matches_scipy(K, order):
    # Library routine: scipy's de Boor evaluation on the same clamped knot vector.
    from scipy.interpolate import BSpline
    wmin, wmax = 0.0, 2.0
    n = K - order + 2
    knots = np.concatenate([[wmin] * order, np.linspace(wmin, wmax, n)[1:-1], [wmax] * order])
    ws = np.linspace(wmin, wmax, 97)
    for w in ws:
        B = o.bspline_basis(K, order, wmin, wmax, w)
        ref = np.array([BSpline(knots, np.eye(K)[i], order - 1, extrapolate=False)(w)
                        for i in range(K)])
        if w == wmax:  # scipy leaves the right end point open; the oracle closes it
            ref = np.array([BSpline(knots, np.eye(K)[i], order - 1)(w) for i in range(K)])
        assert np.allclose(B, ref, rtol=0, atol=1e-14)


def test_mode_counts_match_paper_tables():
    # Tables I and II print the number of spectral components for each band.
    g = json.load(open(os.path.join(GOLDEN, "paper_tables.json")))
    for key in ("table_I", "table_II"):
        t = g[key]
        T = 1.0 / t["dnu"]
        assert abs(T - t["T"]) < 1e-9
        M, j0 = o.mode_range(2 * math.pi * t["nu_min"], 2 * math.pi * t["nu_max"], T)
        assert M == t["n_components"]
    # and the DE-batch band [0, 2] with T = 200 has j = 1..63 (DC removed)
    M, j0 = o.mode_range(0.0, 2.0, 200.0)
    assert (M, j0) == (63, 1)


# --------------------------------------------------------------------------- synthesis


def _batch_field(ncand=3, n_steps=2048, seed=5):
    cfg = inputs.DE_BATCH
    P = inputs.random_population(ncand, cfg["K"], seed)
    A, E, s, rc = o.synth_field(P, cfg["K"], cfg["order"], cfg["w_min"], cfg["w_max"], cfg["T"],
                                cfg["fluence"], n_steps)
    assert rc == 0
    return cfg, P, A, E, s


def test_synth_potential_vanishes_at_both_ends():
    # DC removed, so A(-T/2) = A(T/2) = 0.
    cfg, P, A, E, s = _batch_field()
    for c in range(A.shape[0]):
        amax = np.abs(A[c]).max()
        assert np.abs(A[c][:, 0]).max() <= 1e-12 * amax
        assert np.abs(A[c][:, -1]).max() <= 1e-12 * amax


def test_synth_E_is_minus_dA_dt_spectrally():
    # E = -dA/dt (Sec. II.A).  A is a trigonometric polynomial sampled on a
    # periodic grid, so its derivative is exact by FFT.
    cfg, P, A, E, s = _batch_field()
    n = A.shape[-1] - 1
    h = cfg["T"] / n
    k = np.fft.fftfreq(n, d=h) * 2 * np.pi
    for c in range(A.shape[0]):
        for l in range(2):
            dA = np.fft.ifft(1j * k * np.fft.fft(A[c, l, :n])).real
            assert np.abs(-dA - E[c, l, :n]).max() <= 1e-10 * np.abs(E[c, l]).max()


def test_synth_fluence_is_normalised():
    # Eq. (energy) renormalised to U_const (Sec. IV.B): the rectangle rule over
    # one period is exact for the trigonometric polynomial E^2.
    cfg, P, A, E, s = _batch_field()
    n = A.shape[-1] - 1
    h = cfg["T"] / n
    for c in range(A.shape[0]):
        U = h * np.sum(E[c, :, :n] ** 2)
        assert abs(U - cfg["fluence"]) < 1e-12 * cfg["fluence"]


def test_linear_vs_circular_peak_field_ratio_sqrt2():
    # Sec. V.B: at fixed fluence a linearly polarised single mode has a peak
    # field sqrt(2) times the circular one.  One mode: band [0.9, 1.1], T = 2 pi.
    K, order = 4, 4
    lin = np.zeros(4 * K)
    lin[0:K] = 1.0
    circ = np.zeros(4 * K)
    circ[0:K] = 1.0
    circ[2 * K:3 * K] = 1.0
    circ[3 * K:4 * K] = math.pi / 2
    peaks = []
    for prm in (lin, circ):
        A, E, s, rc = o.synth_field(prm, K, order, 0.9, 1.1, 2 * math.pi, 3.0, 64)
        assert rc == 0
        peaks.append(np.sqrt(E[0, 0] ** 2 + E[0, 1] ** 2).max())
    assert abs(peaks[0] / peaks[1] - math.sqrt(2.0)) < 1e-13


def _field_by_hand(aE, aP, K, order, wmin, wmax, T, n_steps):
    """Eq. (field) with g = 1 and s = 1 for one polarisation, written out
    independently of the oracle: spectrum E~_j = sum_i aE_i B_i(Omega_j) and
    Phi_j = sum_i aP_i B_i(Omega_j) with scipy's B-splines (Eqs. (coeff_basis_E),
    (coeff_basis_phi)), E(t) = sum_j E~_j cos(Omega_j t - Phi_j) and A(t) =
    -int_{-T/2}^t E on the half-step grid.  Returns (E, A, (T/2) sum_j E~_j^2)."""
    from scipy.interpolate import BSpline
    n = K - order + 2
    knots = np.concatenate([[wmin] * order, np.linspace(wmin, wmax, n)[1:-1], [wmax] * order])
    dw = 2 * math.pi / T
    W = dw * np.arange(1, int(math.floor(wmax / dw + 1e-12)) + 1)
    W = W[W >= wmin]
    Bm = np.array([BSpline(knots, np.eye(K)[i], order - 1, extrapolate=False)(W) for i in range(K)])
    Bm = np.nan_to_num(Bm)
    Et, Ph = aE @ Bm, aP @ Bm
    t = -0.5 * T + np.arange(2 * n_steps + 1) * (T / (2 * n_steps))
    arg = np.outer(t, W) - Ph
    E = np.cos(arg) @ Et
    A = -((np.sin(arg) - np.sin(-0.5 * T * W - Ph)) / W) @ Et
    return E, A, 0.5 * T * np.sum(Et ** 2)


@pytest.mark.parametrize("pol", [0, 1])
def test_synth_single_amplitude_weight_with_phase_offset(pol):
    # Sec. III, Eqs. (coeff_basis_E), (field): one nonzero amplitude weight a^E_{l,i}
    # and a constant phase weight Phi_0 (partition of unity makes Phi_j = Phi_0 for
    # every mode) give E_l(t) = s sum_j B_i(Omega_j) cos(Omega_j t - Phi_0).  A sign
    # error on Phi or a coefficient/basis mispairing fails this for some i.
    cfg = inputs.DE_BATCH
    K, order, T, U, ns = cfg["K"], cfg["order"], cfg["T"], cfg["fluence"], 512
    phi0 = 0.7
    for i in range(K):
        prm = np.zeros(4 * K)
        prm[2 * pol * K + i] = 1.0
        prm[(2 * pol + 1) * K:(2 * pol + 2) * K] = phi0
        A, E, s, rc = o.synth_field(prm, K, order, cfg["w_min"], cfg["w_max"], T, U, ns)
        assert rc == 0
        e_ref, a_ref, u_raw = _field_by_hand(prm[2 * pol * K:(2 * pol + 1) * K], np.full(K, phi0), K,
                                             order, cfg["w_min"], cfg["w_max"], T, ns)
        sc = math.sqrt(U / u_raw)
        assert abs(s[0] / sc - 1) < 1e-14
        assert np.abs(E[0, pol] - sc * e_ref).max() <= 1e-13 * sc * np.abs(e_ref).max()
        assert np.abs(A[0, pol] - sc * a_ref).max() <= 1e-13 * sc * np.abs(a_ref).max()
        assert np.abs(E[0, 1 - pol]).max() == 0.0 and np.abs(A[0, 1 - pol]).max() == 0.0


@pytest.mark.parametrize("pol", [0, 1])
def test_synth_single_phase_weight(pol):
    # Sec. III, Eqs. (coeff_basis_phi), (field): unit amplitude weights (E~_j = 1) and
    # one nonzero phase weight a^phi_{l,i} = a give E_l(t) = s sum_j cos(Omega_j t - a B_i(Omega_j)).
    cfg = inputs.DE_BATCH
    K, order, T, U, ns = cfg["K"], cfg["order"], cfg["T"], cfg["fluence"], 512
    for i in range(K):
        prm = np.zeros(4 * K)
        prm[2 * pol * K:(2 * pol + 1) * K] = 1.0
        prm[(2 * pol + 1) * K + i] = 2.1
        A, E, s, rc = o.synth_field(prm, K, order, cfg["w_min"], cfg["w_max"], T, U, ns)
        assert rc == 0
        e_ref, a_ref, u_raw = _field_by_hand(np.ones(K), prm[(2 * pol + 1) * K:(2 * pol + 2) * K], K,
                                             order, cfg["w_min"], cfg["w_max"], T, ns)
        sc = math.sqrt(U / u_raw)
        assert np.abs(E[0, pol] - sc * e_ref).max() <= 1e-13 * sc * np.abs(e_ref).max()
        assert np.abs(A[0, pol] - sc * a_ref).max() <= 1e-13 * sc * np.abs(a_ref).max()


def test_synth_random_weights_both_polarisations():
    # Eq. (field) for a general candidate: both polarisations, random amplitude and
    # phase weights, one global scale s from the fluence of both (Eq. (energy)).
    cfg = inputs.DE_BATCH
    K, order, T, U, ns = cfg["K"], cfg["order"], cfg["T"], cfg["fluence"], 256
    prm = inputs.random_population(1, K, seed=17)[0]
    A, E, s, rc = o.synth_field(prm, K, order, cfg["w_min"], cfg["w_max"], T, U, ns)
    assert rc == 0
    refs = [_field_by_hand(prm[2 * l * K:(2 * l + 1) * K], prm[(2 * l + 1) * K:(2 * l + 2) * K], K, order,
                           cfg["w_min"], cfg["w_max"], T, ns) for l in (0, 1)]
    sc = math.sqrt(U / (refs[0][2] + refs[1][2]))
    for l in (0, 1):
        e_ref, a_ref = sc * refs[l][0], sc * refs[l][1]
        assert np.abs(E[0, l] - e_ref).max() <= 1e-12 * np.abs(e_ref).max()
        assert np.abs(A[0, l] - a_ref).max() <= 1e-12 * np.abs(a_ref).max()


def test_zero_fluence_is_degenerate():
    K = 8
    prm = np.zeros((1, 4 * K))
    A, E, s, rc = o.synth_field(prm, K, 4, 0.0, 2.0, 200.0, 2.0, 64)
    assert rc == 4 and s[0] == 0.0 and not np.any(A)


def test_gaussian_rotating_potential_matches_complex_erf():
    # A_x + i A_y = -E0 (tau sqrt(pi)/2) e^{-w^2 tau^2/4} [erf(t/tau - i w tau/2) - erf(t0/tau - i w tau/2)]
    from scipy.special import erf
    g = inputs.ROTATING_GAUSSIAN
    n = g["n_steps"]
    h = (g["t1"] - g["t0"]) / (2 * n)
    A, E, Ed = o.gaussian_rotating_field(g["E0"], g["w"], g["tau"], g["t0"], h, 2 * n + 1)
    t = g["t0"] + h * np.arange(2 * n + 1)
    tau, w = g["tau"], g["w"]
    z = -g["E0"] * tau * math.sqrt(math.pi) / 2 * math.exp(-(w * tau) ** 2 / 4) * (
        erf(t / tau - 0.5j * w * tau) - erf(g["t0"] / tau - 0.5j * w * tau))
    assert np.abs(A[0] - z.real).max() < 1e-13
    assert np.abs(A[1] - z.imag).max() < 1e-13


# --------------------------------------------------------------------------- spinors


def test_spinors_are_eigenvectors_and_orthonormal():
    # Eq. (free_spin1): H u = w u, H v = -w v, u+u = v+v = 2w, u+v = 0.
    rng = np.random.default_rng(3)
    for _ in range(20):
        P = rng.normal(size=3) * 1.5
        w = math.sqrt(1 + P @ P)
        u, v = o.spinors(P)
        H = dirac_h(P)
        for s in range(2):
            assert np.abs(H @ u[s] - w * u[s]).max() < 1e-13 * w
            assert np.abs(H @ v[s] + w * v[s]).max() < 1e-13 * w
        G = np.concatenate([u, v]).conj() @ np.concatenate([u, v]).T
        assert np.abs(G - 2 * w * np.eye(4)).max() < 1e-13 * w


# --------------------------------------------------------------------------- propagation pins


def test_free_and_pure_gauge_fields_make_no_pairs():
    # u+v = 0 (Sec. II.A): no field, or a constant potential, gives f = 0.
    ns = 400
    p = np.array([[0.3, -0.2, 0.5], [0.0, 0.0, 0.0], [1.2, 0.7, -0.4]])
    for a in (0.0, 0.37):
        A = np.zeros((2, 2 * ns + 1))
        A[0] = a
        A[1] = -0.5 * a
        f = o.dirac_modes(A, ns, 0.05, p)
        assert np.abs(f).max() <= 1e-28


def sauter_fields(E0, tau, t0, h, nsamp):
    t = t0 + h * np.arange(nsamp)
    A = np.zeros((2, nsamp))
    E = np.zeros((2, nsamp))
    Ed = np.zeros((2, nsamp))
    A[0] = -E0 * tau * np.tanh(t / tau)
    E[0] = E0 / np.cosh(t / tau) ** 2
    Ed[0] = -2 * E0 / tau * np.tanh(t / tau) / np.cosh(t / tau) ** 2
    return A, E, Ed


def sauter_exact(E0, tau, p):
    """Spin-summed pair density for E = E0 sech^2(t/tau) x (Sauter 1932; fermion
    form as in Hebenstreit, Alkofer, Gies, PRD 78, 061701 (2008))."""
    px, py, pz = p
    e2 = 1 + py * py + pz * pz
    wi = math.sqrt(e2 + (px - E0 * tau) ** 2)
    wo = math.sqrt(e2 + (px + E0 * tau) ** 2)
    a = math.pi * tau / 2
    return (2 * math.sinh(a * (2 * E0 * tau + wi - wo)) * math.sinh(a * (2 * E0 * tau - wi + wo))
            / (math.sinh(math.pi * tau * wi) * math.sinh(math.pi * tau * wo)))


def test_sauter_pulse_closed_form():
    E0, tau, T, ns = 0.25, 5.0, 300.0, 30000
    dt = T / ns
    A, E, Ed = sauter_fields(E0, tau, -T / 2, dt / 2, 2 * ns + 1)
    ps = np.array([[0.0, 0.0, 0.0], [0.3, 0.2, 0.1], [-0.5, 0.4, 0.7], [0.8, -0.3, 0.2]])
    f = o.dirac_modes(A, ns, dt, ps)
    ref = np.array([sauter_exact(E0, tau, p) for p in ps])
    assert np.abs(f / ref - 1).max() < 1e-6


def test_weak_field_first_order_formula():
    # First-order perturbation theory of Eq. (dirac_eq_mom) around H(p), with
    # A(t_i) = A(t_f) = 0:  f = 2 (|A~|^2 - |p.A~|^2 / w^2),  A~ = int A e^{2iwt} dt.
    # The relative deviation is second order in the field: it grows 4x when the field doubles.
    tau, w, T, ns = 8.0, 2.8, 120.0, 24000
    dt = T / ns
    h = dt / 2
    t = -T / 2 + h * np.arange(2 * ns + 1)
    ps = np.array([[0.3, 0.2, 0.1], [-0.5, 0.4, 0.7], [0.1, -0.2, 0.0]])
    devs = []
    for a0 in (1e-3, 2e-3):
        A = np.zeros((2, t.size))
        g = a0 * np.exp(-t ** 2 / tau ** 2)
        A[0] = g * np.cos(w * t)
        A[1] = 0.5 * g * np.sin(w * t)
        f = o.dirac_modes(A, ns, dt, ps)
        ref = []
        for p in ps:
            om = math.sqrt(1 + p @ p)
            ph = np.exp(2j * om * t)
            At = np.array([np.sum(A[0] * ph) * h, np.sum(A[1] * ph) * h, 0.0])
            ref.append(2 * (np.vdot(At, At).real - abs(p @ At) ** 2 / om ** 2))
        devs.append(f / np.array(ref) - 1)
    assert np.abs(devs[0]).max() < 2e-3
    ratio = devs[1] / devs[0]
    assert np.all(np.abs(ratio - 4.0) < 0.05)


def test_dirac_equals_kinetic_equation_and_decides_spin_sum_reading():
    # Sec. II: both formalisms "yield equivalent results": Dirac f of Eq.
    # (pair_prod_homo) = 1 - chi_1 of the 6-component kinetic equation.  The
    # full spin trace agrees; the same-spin-only pairing does not.
    g = inputs.ROTATING_GAUSSIAN
    ns = 8000
    dt = (g["t1"] - g["t0"]) / ns
    A, E, Ed = o.gaussian_rotating_field(g["E0"], g["w"], g["tau"], g["t0"], dt / 2, 2 * ns + 1)
    ps = np.array([[0.3, 0.2, 0.1], [-0.5, 0.4, 0.7], [0.0, 0.9, 0.3], [1.1, -0.2, 0.6]])
    fd = o.dirac_modes(A, ns, dt, ps)
    fq = o.qke6_modes(A, E, Ed, ns, dt, ps)
    fdiag = o.dirac_modes(A, ns, dt, ps, spin_sum=1)
    assert np.abs(fd / fq - 1).max() < 1e-6
    assert np.abs(fdiag / fq - 1).max() > 1e-4
    # linear Sauter pulse: the kinetic equation also reproduces the closed form
    E0, tau, T, ns = 0.25, 5.0, 300.0, 30000
    dt = T / ns
    A, E, Ed = sauter_fields(E0, tau, -T / 2, dt / 2, 2 * ns + 1)
    p = np.array([[0.3, 0.2, 0.1]])
    assert abs(o.qke6_modes(A, E, Ed, ns, dt, p)[0] / sauter_exact(E0, tau, p[0]) - 1) < 1e-6


def _rot_field(ns=2000):
    g = inputs.ROTATING_GAUSSIAN
    dt = (g["t1"] - g["t0"]) / ns
    A, _, _ = o.gaussian_rotating_field(g["E0"] * 3, g["w"], g["tau"], g["t0"], dt / 2, 2 * ns + 1)
    return A, ns, dt


def test_symmetries():
    A, ns, dt = _rot_field()
    rng = np.random.default_rng(11)
    ps = rng.uniform(-1.2, 1.2, size=(6, 3))
    f = o.dirac_modes(A, ns, dt, ps)
    # (i) the field lies in the x-y plane: f(px, py, pz) = f(px, py, -pz)
    fm = o.dirac_modes(A, ns, dt, ps * np.array([1, 1, -1]))
    assert np.abs(fm / f - 1).max() < 1e-12
    # (ii) charge conjugation: f(p; A) = f(-p; -A)
    fc = o.dirac_modes(-A, ns, dt, -ps)
    assert np.abs(fc / f - 1).max() < 1e-12
    # (iii) rotating the field and the momenta by 90 degrees about z changes nothing
    Ar = np.stack([-A[1], A[0]])
    pr = np.stack([-ps[:, 1], ps[:, 0], ps[:, 2]], axis=1)
    fr = o.dirac_modes(Ar, ns, dt, pr)
    assert np.abs(fr / f - 1).max() < 1e-12


def test_rk4_amplification_factor_closed_form():
    # Classical RK4 applied to psi' = -i H psi with constant H multiplies each
    # eigencomponent by R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24, z = -i E dt, per
    # step.  The initial state is the -w eigenvector, so psi(t_f) = R(i w dt)^N v.
    ns, dt = 300, 0.07
    for a in ((0.0, 0.0), (0.4, -0.9)):
        A = np.zeros((2, 2 * ns + 1))
        A[0], A[1] = a
        p = np.array([0.3, -0.7, 0.45])
        P = p - np.array([a[0], a[1], 0.0])
        w = math.sqrt(1 + P @ P)
        z = 1j * w * dt
        R = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
        f, psi = o.dirac_mode(A, ns, dt, p, return_psi=True)
        _, v = o.spinors(P)
        assert np.abs(psi - R ** ns * v).max() < 1e-12
        assert abs(f) < 1e-28


def test_rk4_converges_at_least_fourth_order():
    # The paper's RK4 has convergence order q = 4 (Sec. V.C.2): halving dt cuts
    # the change of f by at least 2^4 (this field is still pre-asymptotic, where
    # the observed order is about 5).
    g = inputs.ROTATING_GAUSSIAN
    p = np.array([[0.3, 0.2, 0.1], [-0.5, 0.4, 0.7]])
    fs = []
    for ns in (1000, 2000, 4000):
        dt = (g["t1"] - g["t0"]) / ns
        A, _, _ = o.gaussian_rotating_field(g["E0"], g["w"], g["tau"], g["t0"], dt / 2, 2 * ns + 1)
        fs.append(o.dirac_modes(A, ns, dt, p))
    ratio = (fs[0] - fs[1]) / (fs[1] - fs[2])
    assert np.all(ratio > 16 * 0.9) and np.all(ratio < 64)


# --------------------------------------------------------------------------- reduction


def test_trapezoid_weights():
    w = o.trapz_weights(11, -2.0, 2.0, 0)
    assert abs(w.sum() - 4.0) < 1e-15
    x = np.linspace(-2, 2, 11)
    assert abs(w @ (3 * x + 1) - 4.0) < 1e-14  # exact for linear functions
    wm = o.trapz_weights(6, 0.0, 2.0, 1)
    assert abs(wm.sum() - 4.0) < 1e-15
    # the mirrored half axis reproduces the trapezoid rule on the full symmetric axis
    full = o.trapz_weights(11, -2.0, 2.0, 0)
    assert np.allclose(wm, np.concatenate([[full[5]], 2 * full[6:]]), rtol=0, atol=1e-15)
    # convergence to a Gaussian integral: error O(h^2) -> tiny for a decayed integrand
    xs = np.linspace(-6, 6, 601)
    assert abs(o.trapz_weights(601, -6, 6, 0) @ np.exp(-xs ** 2) - math.sqrt(math.pi)) < 1e-12


def test_pair_number_is_weighted_sum_and_thread_independent():
    A, ns, dt = _rot_field(600)
    grid = inputs.small_grid(5, 4, 3, ext=1.2)
    N1, n1 = o.pair_number(A[None], ns, dt, grid, nthreads=1)
    N4, n4 = o.pair_number(A[None], ns, dt, grid, nthreads=4)
    assert N1[0] == N4[0] and np.array_equal(n1, n4)
    x, y, z = inputs.grid_axes(grid)
    wx = np.full(x.size, x[1] - x[0]); wx[[0, -1]] /= 2
    wy = np.full(y.size, y[1] - y[0]); wy[[0, -1]] /= 2
    wz = np.full(z.size, z[1] - z[0]); wz[[0, -1]] /= 2
    wz *= 2
    W = wz[:, None, None] * wy[None, :, None] * wx[None, None, :]
    assert abs(np.sum(W * n1[0]) / N1[0] - 1) < 1e-13
    pts = inputs.grid_points(grid)
    f = o.dirac_modes(A, ns, dt, pts)
    assert np.array_equal(f, n1[0].ravel())


# --------------------------------------------------------------------------- differential evolution


def test_splitmix64_published_outputs():
    g = json.load(open(os.path.join(GOLDEN, "splitmix64_seed0.json")))
    for k, hx in enumerate(g["outputs_hex"]):
        assert o.splitmix64_at(g["seed"], k) == int(hx, 16)


def _wide(D):
    return np.full(D, -1e9), np.full(D, 1e9), np.zeros(D, np.uint8)


def test_de_donors_distinct_and_mutation_formula():
    # Step 1: a, b, c distinct and different from x; step 2: u = a + F (b - c).
    NP = 9
    pop = np.diag(np.arange(1.0, NP + 1))  # row k = (k+1) e_k
    lo, hi, per = _wide(NP)
    for gen in range(20):
        tr = o.de_propose(pop, lo, hi, per, 0.5, 1.0, 1234, gen)
        for i in range(NP):
            nz = {j: tr[i, j] for j in range(NP) if tr[i, j] != 0}
            assert len(nz) == 3
            r1 = [j for j, v in nz.items() if v == j + 1]
            r2 = [j for j, v in nz.items() if v == 0.5 * (j + 1)]
            r3 = [j for j, v in nz.items() if v == -0.5 * (j + 1)]
            assert len(r1) == len(r2) == len(r3) == 1
            assert i not in (r1[0], r2[0], r3[0])


def test_de_F0_CR1_copies_donor_and_NP4_uses_the_other_three():
    rng = np.random.default_rng(2)
    pop = rng.random((4, 3))
    lo, hi, per = np.zeros(3), np.ones(3), np.zeros(3, np.uint8)
    for gen in range(10):
        tr = o.de_propose(pop, lo, hi, per, 0.0, 1.0, 77, gen)
        for i in range(4):
            match = [k for k in range(4) if np.array_equal(tr[i], pop[k])]
            assert len(match) == 1 and match[0] != i


def test_de_CR0_takes_exactly_one_coordinate():
    rng = np.random.default_rng(4)
    NP, D = 12, 7
    pop = rng.random((NP, D))
    lo, hi, per = np.zeros(D), np.ones(D), np.zeros(D, np.uint8)
    tr = o.de_propose(pop, lo, hi, per, 0.0, 0.0, 99, 3)
    for i in range(NP):
        diff = np.flatnonzero(tr[i] != pop[i])
        assert len(diff) == 1
        j = diff[0]
        assert tr[i, j] in pop[:, j]


def test_de_crossover_fraction():
    NP, D, CR = 200, 500, 0.37
    pop = np.tile(np.arange(NP, dtype=float)[:, None], (1, D)) / NP
    lo, hi, per = np.full(D, -10.0), np.full(D, 10.0), np.zeros(D, np.uint8)
    tr = o.de_propose(pop, lo, hi, per, 0.0, CR, 5, 0)
    taken = (tr != pop).sum()
    n = NP * D
    # forced index adds ~ (1-CR) per row; binomial std ~ sqrt(n CR (1-CR))
    expect = n * CR + NP * (1 - CR)
    assert abs(taken - expect) < 5 * math.sqrt(n * CR * (1 - CR))


def test_de_bounds_clip_and_wrap():
    K = 3
    lo, hi, per = inputs.param_bounds(K)
    pop = inputs.random_population(30, K, 8)
    for gen in range(30):
        tr = o.de_propose(pop, lo, hi, per, 1.9, 0.9, 31, gen)
        assert np.all(tr >= lo) and np.all(tr <= hi)
        assert np.all(tr[:, per.astype(bool)] < hi[per.astype(bool)])


def test_de_select_ties_and_nan():
    pop = np.zeros((3, 2))
    trial = np.ones((3, 2))
    fit = np.array([1.0, 2.0, 3.0])
    tfit = np.array([1.0, 1.5, np.nan])
    p2, f2 = o.de_select(pop, fit, trial, tfit)
    assert np.array_equal(p2, np.array([[1, 1], [0, 0], [0, 0]], float))
    assert np.array_equal(f2, np.array([1.0, 2.0, 3.0]))


def test_de_reaches_sphere_maximum():
    # DE (Sec. IV.B) on a textbook function: maximise -|x - x*|^2 on [-5, 5]^5.
    D, NP = 5, 20
    lo, hi, per = np.full(D, -5.0), np.full(D, 5.0), np.zeros(D, np.uint8)
    xs = np.array([1.0, -2.0, 0.5, 3.0, -0.25])
    pop = np.random.default_rng(0).uniform(-5, 5, (NP, D))
    fit = -((pop - xs) ** 2).sum(1)
    for gen in range(400):
        tr = o.de_propose(pop, lo, hi, per, 0.8, 0.9, 2024, gen)
        tf = -((tr - xs) ** 2).sum(1)
        pop, fit = o.de_select(pop, fit, tr, tf)
    assert fit.max() > -1e-10
