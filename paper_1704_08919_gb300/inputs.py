"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module holds workload descriptions, random draws and the given field of
the rotating-Gaussian workload -- none of the method's arithmetic -- so that the
CUDA path and the CPU oracle can be fed the same inputs without sharing any code.  Numbers are drawn with numpy's PCG64
(`numpy.random.default_rng(seed)`).

Workloads (sizes follow the paper's pulse model, Sec. III, and momentum
windows, Sec. V, scaled to the configurations below):

* ``ROTATING_GAUSSIAN``: one rotating field
  E(t) = E0 exp(-t^2/tau^2) (cos w t, sin w t, 0), E0 = 0.1, w = 0.7, tau = 10,
  t in [-40, 40], dt = 0.02 (4000 RK4 steps), A(-40) = 0; grid 32 x 32 x 16 on
  [-1.5, 1.5]^2 x [0, 1.5] with the p_z mirror.
* ``UNEVEN_BATCH``: a population of 128 slots with pulse lengths T = 0.02 n,
  n uniform in [2500, 20000] (one RK4-grid step count per slot), K = 8 cubic
  B-splines on [0, 2], fluence 2.0; momentum grids of side 32, 48, 64, 80 or 96
  (n_z = side / 2) over [-2, 2]^2 x [0, 2], mirrored, by the quintile of the
  slot's initial peak field; DE with F = 0.8, CR = 0.9.
* ``SURROGATE_DE``: surrogate-screened DE on the DE_BATCH solver settings: a
  network 32 -> 256 -> 256 -> 256 -> 1 trained on 50,000 seeded random pulses
  scored exactly (2,048 more held out), population 128, 8 proposals per
  individual per generation of which the network keeps one.
* ``LOCAL_SEARCH``: the multistart augmented-Lagrangian search of Sec. IV.A on
  the QKE: 16 starts, K = 8 (32 parameters), cubic B-splines on [0, 2], T = 50,
  16384 RK4 steps (the QKE is stiff near zeros of E: at T = 200 and 8192 steps it
  does not converge for such pulses), grid 32 x 32 x 16 over [-2, 2]^2 x [0, 2]
  mirrored, U_const = 2.0, starts uniform in the bounds with the amplitudes
  scaled to U_const.
* ``LARGE_SCALE``: population 1024, K = 16 (64 parameters), cubic B-splines on
  [0, 2], T = 400, 20000 steps, fluence 2.0, grid 128 x 128 x 64 over
  [-2.5, 2.5]^2 x [0, 2.5] mirrored, DE F = 0.8, CR = 0.9, surrogate-screened
  (8 proposals per individual) with the network refitted every 20 generations on
  the pulses scored so far.
* ``DE_BATCH``: a population of 64 B-spline pulses (K = 8 control points per
  amplitude and phase per polarisation, cubic splines on [0, 2], T = 200,
  8192 RK4 steps, fluence 2.0) on a 64 x 64 x 32 grid over [-2, 2]^2 x [0, 2]
  with the p_z mirror; DE with F = 0.8, CR = 0.9.
"""
import math

import numpy as np

ROTATING_GAUSSIAN = dict(
    name="rotating-gaussian E0=0.1 w=0.7 tau=10 t=[-40,40] dt=0.02 grid 32x32x16",
    E0=0.1, w=0.7, tau=10.0, t0=-40.0, t1=40.0, n_steps=4000,
    grid=dict(nx=32, ny=32, nz=16, x0=-1.5, x1=1.5, y0=-1.5, y1=1.5, z0=0.0, z1=1.5, mirror_z=1),
)

DE_BATCH = dict(
    name="de-batch 64 B-spline pulses K=8 T=200 8192 steps grid 64x64x32",
    NP=64, K=8, order=4, w_min=0.0, w_max=2.0, T=200.0, fluence=2.0, n_steps=8192,
    F=0.8, CR=0.9,
    grid=dict(nx=64, ny=64, nz=32, x0=-2.0, x1=2.0, y0=-2.0, y1=2.0, z0=0.0, z1=2.0, mirror_z=1),
)

SURROGATE_DE = dict(
    name="surrogate-screened DE: pop 128, 8 proposals/individual, MLP 32-256-256-256-1 on 50k "
         "exact samples, solver as de-batch (K=8 T=200 8192 steps grid 64x64x32)",
    NP=128, R=8, hidden=256, n_train=50000, n_heldout=2048, generations=60,
    epochs=60, batch=256, lr0=2e-3, lr1=5e-5,
    train_seed=424242, heldout_seed=434343, pop_seed=7, de_seed=77,
)


LOCAL_SEARCH = dict(
    name="local search: 16 starts K=8 T=50 16384 steps grid 32x32x16, QKE adjoint + AL-BFGS",
    nstart=16, K=8, order=4, w_min=0.0, w_max=2.0, T=50.0, n_steps=16384, U_const=2.0,
    grid=dict(nx=32, ny=32, nz=16, x0=-2.0, x1=2.0, y0=-2.0, y1=2.0, z0=0.0, z1=2.0, mirror_z=1),
    mu0=0.1, xi=0.5, outer=6, max_iter=30, gtol=1e-4, ctol=1e-3, seed=2024,
)


LARGE_SCALE = dict(
    name="large-scale: pop 1024 K=16 T=400 20000 steps grid 128x128x64, screened DE (R=8)",
    NP=1024, K=16, order=4, w_min=0.0, w_max=2.0, T=400.0, fluence=2.0, n_steps=20000,
    F=0.8, CR=0.9, R=8, generations=200, refit_every=20, pop_seed=31, de_seed=310,
    grid=dict(nx=128, ny=128, nz=64, x0=-2.5, x1=2.5, y0=-2.5, y1=2.5, z0=0.0, z1=2.5, mirror_z=1),
)


UNEVEN_BATCH = dict(
    name="uneven-batch 128 slots T~U[50,400] dt=0.02 grids 32..96 by peak-field quintile",
    NP=128, K=8, order=4, w_min=0.0, w_max=2.0, fluence=2.0, dt=0.02, n_min=2500, n_max=20000,
    sides=(32, 48, 64, 80, 96), ext=2.0, F=0.8, CR=0.9,
)


def uneven_steps(cfg, seed):
    """Step count of every slot (uniform integers in [n_min, n_max])."""
    rng = np.random.default_rng(seed)
    return rng.integers(cfg["n_min"], cfg["n_max"] + 1, size=cfg["NP"])


def uneven_specs(cfg, steps):
    return [dict(K=cfg["K"], order=cfg["order"], w_min=cfg["w_min"], w_max=cfg["w_max"],
                 T=float(n) * cfg["dt"], fluence=cfg["fluence"], n_steps=int(n)) for n in steps]


def grids_by_rank(cfg, peaks):
    """Slot grids by the quintile of each slot's peak field (weakest fields get the
    smallest grid): sides[q] x sides[q] x sides[q]/2 for quintile q."""
    peaks = np.asarray(peaks)
    order = np.argsort(peaks, kind="stable")
    q = np.empty(len(peaks), dtype=int)
    q[order] = (np.arange(len(peaks)) * len(cfg["sides"])) // len(peaks)
    e = cfg["ext"]
    return [dict(nx=cfg["sides"][k], ny=cfg["sides"][k], nz=cfg["sides"][k] // 2, x0=-e, x1=e,
                 y0=-e, y1=e, z0=0.0, z1=e, mirror_z=1) for k in q]


def field_spec(cfg):
    """The pulse-model settings of a workload as a plain dict."""
    return dict(K=cfg["K"], order=cfg["order"], w_min=cfg["w_min"], w_max=cfg["w_max"],
                T=cfg["T"], fluence=cfg["fluence"], n_steps=cfg["n_steps"])


def param_bounds(K):
    """(lo, hi, periodic) for the 4K parameters [a^E_x, a^phi_x, a^E_y, a^phi_y].

    Amplitude weights lie in [0, 1]; phase weights in [0, 2 pi) and wrap.
    """
    lo = np.zeros(4 * K)
    hi = np.empty(4 * K)
    per = np.zeros(4 * K, dtype=np.uint8)
    for blk in range(4):
        sl = slice(blk * K, (blk + 1) * K)
        if blk % 2 == 0:
            hi[sl] = 1.0
        else:
            hi[sl] = 2.0 * math.pi
            per[sl] = 1
    return lo, hi, per


def random_population(NP, K, seed):
    """NP parameter vectors drawn uniformly inside param_bounds(K)."""
    lo, hi, _ = param_bounds(K)
    rng = np.random.default_rng(seed)
    return lo + rng.random((NP, 4 * K)) * (hi - lo)


def grid_axes(grid):
    """(x, y, z) node coordinates of a momentum grid (linspace, end points included)."""
    def ax(n, a, b):
        return np.array([a]) if n == 1 else np.linspace(a, b, n)
    return (ax(grid["nx"], grid["x0"], grid["x1"]), ax(grid["ny"], grid["y0"], grid["y1"]),
            ax(grid["nz"], grid["z0"], grid["z1"]))


def grid_points(grid):
    """All grid momenta as an array [nz*ny*nx, 3], x fastest."""
    x, y, z = grid_axes(grid)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def strided_modes(grid, count, seed):
    """`count` distinct flat mode indices spread over the grid (sorted)."""
    nm = grid["nx"] * grid["ny"] * grid["nz"]
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(nm, size=min(count, nm), replace=False))


def rotating_gaussian_potential(cfg, n_samples):
    """The vector potential of the ROTATING_GAUSSIAN field on n_samples points of
    its half-step grid, t_k = t0 + k (t1 - t0) / (n_samples - 1): A(t) = -int_{t0}^t E
    with E_x + i E_y = E0 exp(-t^2/tau^2 + i w t), written in closed form with the
    complex error function,
        int exp(-t^2/tau^2 + i w t) dt = (sqrt(pi) tau / 2) exp(-w^2 tau^2 / 4) erf(t/tau - i w tau / 2),
    so A_x + i A_y = -E0 (sqrt(pi) tau / 2) exp(-w^2 tau^2 / 4) [erf(z(t)) - erf(z(t0))].
    Returns A[2][n_samples] (rows A_x, A_y)."""
    from scipy.special import erf
    E0, w, tau, t0, t1 = cfg["E0"], cfg["w"], cfg["tau"], cfg["t0"], cfg["t1"]
    t = t0 + np.arange(n_samples) * ((t1 - t0) / (n_samples - 1))
    pref = E0 * math.sqrt(math.pi) * tau / 2 * math.exp(-(w * tau) ** 2 / 4)
    z = t / tau - 0.5j * w * tau
    a = -pref * (erf(z) - erf(t0 / tau - 0.5j * w * tau))
    return np.stack([a.real, a.imag])


def small_grid(nx, ny, nz, ext=2.0, mirror_z=1):
    return dict(nx=nx, ny=ny, nz=nz, x0=-ext, x1=ext, y0=-ext, y1=ext, z0=0.0, z1=ext,
                mirror_z=mirror_z)
