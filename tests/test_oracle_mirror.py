"""The oracle's host mirror of the library's entry points (pp_oracle_synth_field,
pp_oracle_pair_number, pp_oracle_de_propose / _select / _step): same arguments as
the CUDA library's calls, host arrays, FP64 on the CPU.  Pinned here to the
oracle's own routines, which the other oracle tests pin to the paper; the ctypes
argument structs are the package's own (the mirror declares the same layout)."""
import ctypes

import numpy as np

import oracle
import paper_1704_08919_gb300 as pp
from paper_1704_08919_gb300 import inputs

K = 6
SPEC = dict(K=K, order=4, w_min=0.0, w_max=2.0, T=40.0, fluence=2.0, n_steps=400)
GRID = dict(nx=5, ny=4, nz=3, x0=-1.0, x1=1.0, y0=-0.8, y1=0.9, z0=0.0, z1=1.0, mirror_z=1)


def ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def mirror_synth(X, spec):
    n = spec["n_steps"]
    A = np.zeros((X.shape[0], 2, 2 * n + 1))
    E, s = np.zeros_like(A), np.zeros(X.shape[0])
    rc = oracle.lib().pp_oracle_synth_field(ptr(X), X.shape[0], ctypes.byref(pp._spec(spec)), ptr(A), 2 * n + 1,
                                           ptr(E), ptr(s), None)
    return rc, A, E, s


def mirror_pair_number(A, n_steps, dt, grid, scheme=0, precision=0):
    nc, _, ld = A.shape
    N = np.zeros(nc)
    n = np.zeros((nc, grid["nz"], grid["ny"], grid["nx"]))
    ns = None if n_steps is None else np.asarray(n_steps, dtype=np.int32)
    rc = oracle.lib().pp_oracle_pair_number(ptr(np.ascontiguousarray(A)), nc, ld, ptr(ns), dt,
                                           ctypes.byref(pp._grid(grid)), precision, scheme, ptr(N), ptr(n), None)
    return rc, N, n


def test_synthesis_is_the_oracles():
    X = inputs.random_population(3, K, seed=2)
    rc, A, E, s = mirror_synth(X, SPEC)
    Ao, Eo, so, rco = oracle.synth_field(X, K, 4, 0.0, 2.0, 40.0, 2.0, 400)
    assert rc == 0 == rco
    assert np.array_equal(A, Ao) and np.array_equal(E, Eo) and np.array_equal(s, so)
    rc, A1, _, _ = mirror_synth(X, dict(SPEC, envelope=1))
    Ah, _, _, _ = oracle.synth_hann(X, K, 4, 0.0, 2.0, 40.0, 2.0, 400)
    assert rc == 0 and np.array_equal(A1, Ah)


def test_pair_number_is_the_oracles_for_every_scheme():
    X = inputs.random_population(2, K, seed=3)
    _, A, _, _ = mirror_synth(X, SPEC)
    dt = SPEC["T"] / SPEC["n_steps"]
    rc, N, n = mirror_pair_number(A, None, dt, GRID)
    No, no = oracle.pair_number(A, SPEC["n_steps"], dt, GRID)
    assert rc == 0 and np.array_equal(N, No) and np.array_equal(n, no)
    p, w = oracle.grid_modes(GRID)
    for scheme, fn in ((1, oracle.lib().orc_dirac_magnus_modes), (2, oracle.lib().orc_dirac_split_modes)):
        rc, N, n = mirror_pair_number(A, [400, 400], dt, GRID, scheme=scheme, precision=2)
        assert rc == 0
        for c in range(2):
            f = np.zeros(len(w))
            Ac = np.ascontiguousarray(A[c])
            fn(Ac.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), Ac.shape[1], 400, dt,
               np.ascontiguousarray(p).ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(w),
               f.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None, 0)
            assert np.array_equal(n[c].ravel(), f)
            assert abs(N[c] - float(np.sum(w * f))) <= 1e-15 * abs(N[c])


def test_de_step_is_propose_synthesise_score_select():
    NP = 6
    lo, hi, per = inputs.param_bounds(K)
    pop = inputs.random_population(NP, K, seed=4)
    _, A, _, _ = mirror_synth(pop, SPEC)
    dt = SPEC["T"] / SPEC["n_steps"]
    _, fit, _ = mirror_pair_number(A, None, dt, GRID)
    p1, f1 = pop.copy(), fit.copy()
    trial, tfit = np.zeros_like(pop), np.zeros(NP)
    rc = oracle.lib().pp_oracle_de_step(ptr(p1), ptr(f1), NP, ctypes.byref(pp._spec(SPEC)),
                                       ctypes.byref(pp._grid(GRID)), 0, 0, ptr(lo), ptr(hi),
                                       ptr(per.astype(np.uint8)), 0.8, 0.9, 5, 3, ptr(trial), ptr(tfit), None)
    assert rc == 0
    to = oracle.de_propose(pop, lo, hi, per, 0.8, 0.9, 5, 3)
    assert np.array_equal(trial, to)
    _, At, _, _ = mirror_synth(to, SPEC)
    _, Nt, _ = mirror_pair_number(At, None, dt, GRID)
    assert np.array_equal(tfit, Nt)
    keep = Nt >= fit
    assert np.array_equal(p1, np.where(keep[:, None], to, pop))
    assert np.array_equal(f1, np.where(keep, Nt, fit))


def test_mirror_rejects_what_the_library_rejects():
    L = oracle.lib()
    X = inputs.random_population(1, K, seed=1)
    A = np.zeros((1, 2, 801))
    assert mirror_synth(X, dict(SPEC, envelope=2))[0] == pp.PP_ERR_INVALID_ARG
    assert mirror_pair_number(A, None, 0.1, GRID, scheme=3)[0] == pp.PP_ERR_INVALID_ARG
    assert mirror_pair_number(A, None, 0.1, GRID, precision=3)[0] == pp.PP_ERR_INVALID_ARG
    assert mirror_pair_number(A, None, -0.1, GRID)[0] == pp.PP_ERR_INVALID_ARG
    assert mirror_pair_number(A, [500], 0.1, GRID)[0] == pp.PP_ERR_INVALID_ARG  # 2 n_steps + 1 > ld
    pop = np.zeros((3, 4 * K))
    rc = L.pp_oracle_de_propose(ptr(pop), 3, 4 * K, ptr(pop[0]), ptr(pop[0]), None, 0.5, 0.5, 1, 0,
                                ptr(pop.copy()), None)
    assert rc == pp.PP_ERR_INVALID_ARG  # fewer than 4 individuals
    zero = np.zeros((1, 4 * K))
    rc, A0, _, s0 = mirror_synth(zero, SPEC)
    assert rc == pp.PP_ERR_DEGENERATE_FIELD and np.all(A0 == 0.0) and s0[0] == 0.0
