"""FP64 CPU oracle for the pair-number hot path (TEST INFRASTRUCTURE ONLY).

Only tests/, __graft_entry__.smoke() and the cpu_baseline / reference legs of
bench.py may import this package.  The product path (paper_1704_08919_gb300)
never imports it and shares no code with it.

Thin ctypes wrapper over pp_oracle.c; every function states the passage of
arXiv 1704.08919 it follows.  Functions with no independent pin: none (see the
tests under tests/test_oracle_*.py for the pin of each routine).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

_d = ctypes.c_double
_i = ctypes.c_int
_u64 = ctypes.c_uint64
_pd = ctypes.POINTER(ctypes.c_double)
_pi = ctypes.POINTER(ctypes.c_int)
_pu8 = ctypes.POINTER(ctypes.c_uint8)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_bspline_basis.argtypes = [_i, _i, _d, _d, _d, _pd]
        L.orc_mode_range.argtypes = [_d, _d, _d, _pi]
        L.orc_spectrum.argtypes = [_pd, _i, _i, _d, _d, _d, _pd, _pd, _pd]
        L.orc_synth_field.argtypes = [_pd, _i, _i, _i, _d, _d, _d, _d, _i, _i, _pd, _pd, _pd]
        L.orc_gaussian_rotating_field.argtypes = [_d, _d, _d, _d, _d, _i, _pd, _pd, _pd]
        L.orc_gaussian_rotating_field.restype = None
        L.orc_spinors.argtypes = [_pd, ctypes.c_void_p, ctypes.c_void_p]
        L.orc_spinors.restype = None
        L.orc_dirac_mode.argtypes = [_pd, _i, _i, _d, _pd, _i, ctypes.c_void_p]
        L.orc_dirac_mode.restype = _d
        L.orc_dirac_modes.argtypes = [_pd, _i, _i, _d, _pd, _i, _i, _pd, _i]
        L.orc_dirac_split_modes.argtypes = [_pd, _i, _i, _d, _pd, _i, _pd, _pd, _i]
        L.orc_dirac_magnus_modes.argtypes = [_pd, _i, _i, _d, _pd, _i, _pd, _pd, _i]
        L.orc_qke6_modes.argtypes = [_pd, _pd, _pd, _i, _i, _d, _pd, _i, _pd, _i]
        L.orc_trapz_weights.argtypes = [_i, _d, _d, _i, _pd]
        L.orc_trapz_weights.restype = None
        L.orc_pair_number.argtypes = [_pd, _i, _i, _pi, _d, _i, _i, _i, _d, _d, _d, _d, _d, _d,
                                      _i, _i, _pd, _pd, _i]
        L.orc_splitmix64_at.argtypes = [_u64, _u64]
        L.orc_splitmix64_at.restype = _u64
        L.orc_de_propose.argtypes = [_pd, _i, _i, _pd, _pd, _pu8, _d, _d, _u64, _u64, _pd]
        L.orc_de_select.argtypes = [_pd, _pd, _pd, _pd, _i, _i]
        L.orc_num_threads.argtypes = [_i]
        _vp = ctypes.c_void_p
        L.pp_oracle_synth_field.argtypes = [_vp, ctypes.c_int32, _vp, _vp, ctypes.c_int32, _vp, _vp, _vp]
        L.pp_oracle_pair_number.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, _vp, _d, _vp, ctypes.c_int32,
                                            ctypes.c_int32, _vp, _vp, _vp]
        L.pp_oracle_de_propose.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp, _d, _d, _u64,
                                           _u64, _vp, _vp]
        L.pp_oracle_de_select.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int32, ctypes.c_int32, _vp]
        L.pp_oracle_de_step.argtypes = [_vp, _vp, ctypes.c_int32, _vp, _vp, ctypes.c_int32, ctypes.c_int32, _vp,
                                        _vp, _vp, _d, _d, _u64, _u64, _vp, _vp, _vp]
        L.orc_synth_hann.argtypes = [_pd, _i, _i, _i, _d, _d, _d, _d, _i, _i, _i, _pd, _pd, _pd,
                                     _pd]
        L.orc_synth_vjp_hann.argtypes = [_pd, _i, _i, _d, _d, _d, _i, _i, _pd, _pd, _pd, _pd, _pd,
                                         _pd]
        L.orc_synth_raw.argtypes = [_pd, _i, _i, _i, _d, _d, _d, _i, _i, _pd, _pd, _pd, _pd]
        L.orc_fluence_raw.argtypes = [_pd, _i, _i, _d, _d, _d, _pd, _pd]
        L.orc_qke6_adjoint_mode.argtypes = [_pd, _pd, _pd, _i, _i, _d, _pd, _d, _pd, _pd, _pd]
        L.orc_qke6_adjoint_mode.restype = _d
        L.orc_qke6_grad.argtypes = [_pd, _pd, _pd, _i, _i, _d, _pd, _pd, _i, _pd, _pd, _pd, _pd,
                                    _pd, _i]
        L.orc_synth_vjp.argtypes = [_pd, _i, _i, _d, _d, _d, _i, _i, _pd, _pd, _pd, _pd]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(_pd)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads(n=0):
    return lib().orc_num_threads(n)


def bspline_basis(K, order, wmin, wmax, w):
    """B_i(w), i < K: Cox-de Boor recursion with clamped knots (Sec. III)."""
    B = np.zeros(K)
    rc = lib().orc_bspline_basis(K, order, wmin, wmax, w, _p(B))
    if rc:
        raise ValueError("orc_bspline_basis rc=%d" % rc)
    return B


def mode_range(wmin, wmax, T):
    """(M, j_first): modes Omega_j = j 2pi/T with j >= 1 inside [wmin, wmax] (Sec. III)."""
    j0 = ctypes.c_int(0)
    M = lib().orc_mode_range(wmin, wmax, T, ctypes.byref(j0))
    return M, j0.value


def spectrum(params, K, order, wmin, wmax, T):
    """(Omega[M], amp[2,M], phase[2,M]) sampled from the B-spline model, Eqs. (coeff_basis_E/phi)."""
    M, _ = mode_range(wmin, wmax, T)
    params = _f64(params)
    Om, amp, ph = np.zeros(M), np.zeros(2 * M), np.zeros(2 * M)
    rc = lib().orc_spectrum(_p(params), K, order, wmin, wmax, T, _p(Om), _p(amp), _p(ph))
    if rc < 0:
        raise ValueError("orc_spectrum rc=%d" % rc)
    return Om, amp.reshape(2, M), ph.reshape(2, M)


def synth_field(params, K, order, wmin, wmax, T, U, n_steps, want_E=True):
    """A[c,2,2n+1], E (or None), scale[c], status: Eqs. (field), (energy), renormalised (Sec. IV.B)."""
    params = _f64(params).reshape(-1, 4 * K)
    nc = params.shape[0]
    ld = 2 * n_steps + 1
    A = np.zeros((nc, 2, ld))
    E = np.zeros((nc, 2, ld)) if want_E else None
    s = np.zeros(nc)
    rc = lib().orc_synth_field(_p(params), nc, K, order, wmin, wmax, T, U, n_steps, ld, _p(A),
                               _p(E) if want_E else None, _p(s))
    return A, E, s, rc


def gaussian_rotating_field(E0, w, tau, t0, h, nsamp):
    """E = E0 exp(-t^2/tau^2)(cos wt, sin wt), A = -int_{t0}^t E (Gauss-Legendre), Edot analytic."""
    A, E, Ed = np.zeros((2, nsamp)), np.zeros((2, nsamp)), np.zeros((2, nsamp))
    lib().orc_gaussian_rotating_field(E0, w, tau, t0, h, nsamp, _p(A), _p(E), _p(Ed))
    return A, E, Ed


def spinors(P):
    """(u[2,4], v[2,4]) adiabatic free spinors at kinetic momentum P, Eq. (free_spin1)."""
    P = _f64(P)
    u = np.zeros((2, 4), dtype=np.complex128)
    v = np.zeros((2, 4), dtype=np.complex128)
    lib().orc_spinors(_p(P), u.ctypes.data, v.ctypes.data)
    return u, v


def dirac_mode(A, n_steps, dt, p, spin_sum=0, return_psi=False):
    """f(t_f, p) for one mode by RK4 on Eq. (dirac_eq_mom); Eq. (pair_prod_homo)."""
    A = _f64(A).reshape(2, -1)
    p = _f64(p)
    psi = np.zeros(8, dtype=np.complex128)
    f = lib().orc_dirac_mode(_p(A), A.shape[1], n_steps, dt, _p(p), spin_sum, psi.ctypes.data)
    return (f, psi.reshape(2, 4)) if return_psi else f


def dirac_modes(A, n_steps, dt, p, spin_sum=0, nthreads=0):
    """f for a list of momenta p[nm,3] (threads over modes)."""
    A = _f64(A).reshape(2, -1)
    p = _f64(p).reshape(-1, 3)
    out = np.zeros(p.shape[0])
    rc = lib().orc_dirac_modes(_p(A), A.shape[1], n_steps, dt, _p(p), p.shape[0], spin_sum,
                               _p(out), nthreads)
    if rc:
        raise ValueError("orc_dirac_modes rc=%d" % rc)
    return out


def dirac_split_modes(A, n_steps, dt, p, nthreads=0):
    """(f, norm deviation) per momentum with the second-order split operator (Sec. II.A)."""
    A = _f64(A).reshape(2, -1)
    p = _f64(p).reshape(-1, 3)
    out = np.zeros(p.shape[0])
    dev = np.zeros(p.shape[0])
    rc = lib().orc_dirac_split_modes(_p(A), A.shape[1], n_steps, dt, _p(p), p.shape[0], _p(out),
                                     _p(dev), nthreads)
    if rc:
        raise ValueError("orc_dirac_split_modes rc=%d" % rc)
    return out, dev


def dirac_magnus_modes(A, n_steps, dt, p, nthreads=0):
    """(f, norm deviation) per momentum with the fourth-order Magnus step."""
    A = _f64(A).reshape(2, -1)
    p = _f64(p).reshape(-1, 3)
    out = np.zeros(p.shape[0])
    dev = np.zeros(p.shape[0])
    rc = lib().orc_dirac_magnus_modes(_p(A), A.shape[1], n_steps, dt, _p(p), p.shape[0],
                                      _p(out), _p(dev), nthreads)
    if rc:
        raise ValueError("orc_dirac_magnus_modes rc=%d" % rc)
    return out, dev


def qke6_modes(A, E, Edot, n_steps, dt, p, nthreads=0):
    """f = 1 - chi_1 from the 6-component kinetic equation, Eqs. (qke), (matrix)."""
    A = _f64(A).reshape(2, -1)
    E = _f64(E).reshape(2, -1)
    Ed = _f64(Edot).reshape(2, -1)
    p = _f64(p).reshape(-1, 3)
    out = np.zeros(p.shape[0])
    rc = lib().orc_qke6_modes(_p(A), _p(E), _p(Ed), A.shape[1], n_steps, dt, _p(p), p.shape[0],
                              _p(out), nthreads)
    if rc:
        raise ValueError("orc_qke6_modes rc=%d" % rc)
    return out


def trapz_weights(n, a, b, mirror=0):
    w = np.zeros(n)
    lib().orc_trapz_weights(n, a, b, int(mirror), _p(w))
    return w


def pair_number(A, n_steps, dt, grid, spin_sum=0, want_n=True, nthreads=0):
    """(N[c], n[c,nz,ny,nx]) : Eq. (opt_prob) with trapezoid weights over the grid.

    grid = dict(nx, ny, nz, x0, x1, y0, y1, z0, z1, mirror_z).
    """
    A = _f64(A)
    nc, _, ld = A.shape
    ns = np.ascontiguousarray(np.broadcast_to(np.asarray(n_steps, dtype=np.int32), (nc,)))
    g = grid
    nm = g["nx"] * g["ny"] * g["nz"]
    N = np.zeros(nc)
    n = np.zeros((nc, g["nz"], g["ny"], g["nx"])) if want_n else None
    rc = lib().orc_pair_number(_p(A), nc, ld, ns.ctypes.data_as(_pi), dt, g["nx"], g["ny"], g["nz"],
                               g["x0"], g["x1"], g["y0"], g["y1"], g["z0"], g["z1"],
                               int(g.get("mirror_z", 0)), spin_sum, _p(n) if want_n else None,
                               _p(N), nthreads)
    if rc:
        raise ValueError("orc_pair_number rc=%d" % rc)
    del nm
    return N, n


def splitmix64_at(seed, k):
    """k-th output of SplitMix64 seeded with `seed` (Steele, Lea, Flood 2014)."""
    return lib().orc_splitmix64_at(seed & (2**64 - 1), k & (2**64 - 1))


def de_propose(pop, lo, hi, periodic, F, CR, seed, gen):
    """Trial vectors of DE/rand/1/bin, steps 1-3 of Sec. IV.B."""
    pop = _f64(pop)
    NP, D = pop.shape
    lo, hi = _f64(lo), _f64(hi)
    per = np.ascontiguousarray(periodic, dtype=np.uint8)
    trial = np.zeros_like(pop)
    rc = lib().orc_de_propose(_p(pop), NP, D, _p(lo), _p(hi), per.ctypes.data_as(_pu8), F, CR,
                              seed, gen, _p(trial))
    if rc:
        raise ValueError("orc_de_propose rc=%d" % rc)
    return trial


def de_select(pop, fit, trial, trial_fit):
    """Greedy selection, step 4 of Sec. IV.B, maximising N (ties go to the trial)."""
    pop = _f64(pop).copy()
    fit = _f64(fit).copy()
    trial, trial_fit = _f64(trial), _f64(trial_fit)
    NP, D = pop.shape
    rc = lib().orc_de_select(_p(pop), _p(fit), _p(trial), _p(trial_fit), NP, D)
    if rc:
        raise ValueError("orc_de_select rc=%d" % rc)
    return pop, fit


# ----------------------------------------------------------------------------- local search


def synth_raw(params, K, order, wmin, wmax, T, n_steps):
    """(A, E, Edot [c,2,2n+1], U[c]): Eq. (field) with g = 1 and no renormalisation,
    and the fluence of Eq. (energy) over one period (Sec. IV.A keeps U by a penalty)."""
    params = _f64(params).reshape(-1, 4 * K)
    nc = params.shape[0]
    ld = 2 * n_steps + 1
    A, E, Ed = np.zeros((nc, 2, ld)), np.zeros((nc, 2, ld)), np.zeros((nc, 2, ld))
    U = np.zeros(nc)
    rc = lib().orc_synth_raw(_p(params), nc, K, order, wmin, wmax, T, n_steps, ld, _p(A), _p(E),
                             _p(Ed), _p(U))
    if rc:
        raise ValueError("orc_synth_raw rc=%d" % rc)
    return A, E, Ed, U


def fluence_raw(params, K, order, wmin, wmax, T):
    """(U, dU/dparams[4K]) of the un-normalised field, Eq. (energy)."""
    params = _f64(params).reshape(4 * K)
    U = np.zeros(1)
    dU = np.zeros(4 * K)
    rc = lib().orc_fluence_raw(_p(params), K, order, wmin, wmax, T, _p(U), _p(dU))
    if rc:
        raise ValueError("orc_fluence_raw rc=%d" % rc)
    return float(U[0]), dU


def qke6_adjoint_mode(A, E, Edot, n_steps, dt, p, weight=1.0):
    """(f, gA, gE, gEd): f = 1 - chi_1 of one mode and d(weight f)/d(samples), Eqs. (adj), (grad)."""
    A, E, Ed = (_f64(x).reshape(2, -1) for x in (A, E, Edot))
    ld = A.shape[1]
    g = [np.zeros((2, ld)) for _ in range(3)]
    f = lib().orc_qke6_adjoint_mode(_p(A), _p(E), _p(Ed), ld, n_steps, dt, _p(_f64(p)), weight,
                                    _p(g[0]), _p(g[1]), _p(g[2]))
    return f, g[0], g[1], g[2]


def qke6_grad(A, E, Edot, n_steps, dt, p, w, nthreads=0):
    """(J, f[m], gA, gE, gEd): J = sum_m w_m f(p_m) and dJ/d(samples), Eqs. (opt_prob), (grad)."""
    A, E, Ed = (_f64(x).reshape(2, -1) for x in (A, E, Edot))
    ld = A.shape[1]
    p = _f64(p).reshape(-1, 3)
    w = _f64(w).reshape(-1)
    nm = p.shape[0]
    f = np.zeros(nm)
    J = np.zeros(1)
    g = [np.zeros((2, ld)) for _ in range(3)]
    rc = lib().orc_qke6_grad(_p(A), _p(E), _p(Ed), ld, n_steps, dt, _p(p), _p(w), nm, _p(f), _p(J),
                             _p(g[0]), _p(g[1]), _p(g[2]), nthreads)
    if rc:
        raise ValueError("orc_qke6_grad rc=%d" % rc)
    return float(J[0]), f, g[0], g[1], g[2]


def synth_vjp(params, K, order, wmin, wmax, T, n_steps, gA, gE, gEd):
    """dJ/dparams[4K] from dJ/d(samples of A, E, Edot), through Eqs. (field), (coeff_basis_E/phi)."""
    params = _f64(params).reshape(4 * K)
    gA, gE, gEd = (_f64(x).reshape(2, -1) for x in (gA, gE, gEd))
    out = np.zeros(4 * K)
    rc = lib().orc_synth_vjp(_p(params), K, order, wmin, wmax, T, n_steps, gA.shape[1], _p(gA),
                             _p(gE), _p(gEd), _p(out))
    if rc:
        raise ValueError("orc_synth_vjp rc=%d" % rc)
    return out


def grid_modes(grid):
    """(p[m,3], w[m]): the grid momenta (x fastest) and their trapezoid weights, Eq. (opt_prob)."""
    g = grid

    def ax(n, a, b):
        return np.array([a]) if n == 1 else a + (b - a) * np.arange(n) / (n - 1)
    x, y, z = ax(g["nx"], g["x0"], g["x1"]), ax(g["ny"], g["y0"], g["y1"]), ax(g["nz"], g["z0"], g["z1"])
    wx = trapz_weights(g["nx"], g["x0"], g["x1"])
    wy = trapz_weights(g["ny"], g["y0"], g["y1"])
    wz = trapz_weights(g["nz"], g["z0"], g["z1"], int(g.get("mirror_z", 0)))
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    WZ, WY, WX = np.meshgrid(wz, wy, wx, indexing="ij")
    p = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    return p, (WX * WY * WZ).ravel()


def synth_vjp_hann(params, K, order, wmin, wmax, T, n_steps, gA, gE, gEd):
    """(grad[4K], U, dU[4K]): the chain rule and the fluence of the un-normalised
    Hann-envelope field (Eqs. (hann), (field), (vector_potential))."""
    params = _f64(params).reshape(4 * K)
    gA, gE, gEd = (_f64(x).reshape(2, -1) for x in (gA, gE, gEd))
    grad, dU, U = np.zeros(4 * K), np.zeros(4 * K), np.zeros(1)
    rc = lib().orc_synth_vjp_hann(_p(params), K, order, wmin, wmax, T, n_steps, gA.shape[1], _p(gA),
                                  _p(gE), _p(gEd), _p(grad), _p(U), _p(dU))
    if rc:
        raise ValueError("orc_synth_vjp_hann rc=%d" % rc)
    return grad, float(U[0]), dU


def al_objective(params, spec, grid, U_const, lam, mu, nthreads=0):
    """The augmented Lagrangian of Sec. IV.A for one parameter vector:
    L = -J - lam C + C^2 / (2 mu), C = U_const - U, with J from the QKE (Eq. (opt_prob)),
    and its gradient, Eq. (grad): grad L = -grad J - (lam - C / mu) grad C.
    Returns dict(L, grad, J, C, gJ, gC)."""
    K, n = spec["K"], spec["n_steps"]
    args = (K, spec["order"], spec["w_min"], spec["w_max"], spec["T"])
    hann = spec.get("envelope", 0) == 1
    if hann:
        A, E, Ed, _ = synth_hann(params, *args, 1.0, n, normalize=False)
    else:
        A, E, Ed, _ = synth_raw(params, *args, n)
    p, w = grid_modes(grid)
    J, _, gA, gE, gEd = qke6_grad(A[0], E[0], Ed[0], n, spec["T"] / n, p, w, nthreads)
    if hann:
        gJ, U, dU = synth_vjp_hann(params, *args, n, gA, gE, gEd)
    else:
        gJ = synth_vjp(params, *args, n, gA, gE, gEd)
        U, dU = fluence_raw(params, *args)
    C = U_const - U
    gC = -dU
    L = -J - lam * C + C * C / (2.0 * mu)
    grad = -gJ - (lam - C / mu) * gC
    return {"L": L, "grad": grad, "J": J, "C": C, "gJ": gJ, "gC": gC}


def synth_hann(params, K, order, wmin, wmax, T, U, n_steps, normalize=True):
    """(A, E, Edot [c,2,2n+1], scale[c]): Eq. (field) with the Hann envelope of Eq. (hann),
    A from Eq. (vector_potential) in the gauge A(t_f) = 0; scale = s (normalize) or U_raw."""
    params = _f64(params).reshape(-1, 4 * K)
    nc = params.shape[0]
    ld = 2 * n_steps + 1
    A, E, Ed = np.zeros((nc, 2, ld)), np.zeros((nc, 2, ld)), np.zeros((nc, 2, ld))
    s = np.zeros(nc)
    rc = lib().orc_synth_hann(_p(params), nc, K, order, wmin, wmax, T, U, int(normalize), n_steps,
                              ld, _p(A), _p(E), _p(Ed), _p(s))
    if rc:
        raise ValueError("orc_synth_hann rc=%d" % rc)
    return A, E, Ed, s
