"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances: FP64 path 1e-9 relative on N; on n(p)
    |n_gpu - n_ref| <= 1e-9 n + 2 d sqrt(n) + d^2,   d = 32 * 2^-53 * sqrt(n_steps),
where d bounds the FP64 rounding walk of a transition amplitude over n_steps
RK4 steps (n = |amplitude|^2, so an amplitude error d moves n by 2 d sqrt(n));
FP32 path 1e-4 relative on N, and per mode the same form with 1e-4 and
    d32 = 4 * 2^-24 * (w_max dt) * sqrt(n_steps),
the walk of a compensated FP32 sum of increments no larger than w_max dt
(w_max = sqrt(1 + (|p|_max + |A|_max)^2)).  Comparisons between two GPU results
on grids whose nodes differ by an ulp use the FP64 form on both sides.  Field
synthesis 1e-12 relative to max |A|; DE bit-exact.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1704_08919_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_08919_gb300 import build
    build.build()
    import paper_1704_08919_gb300 as pp
    pp.lib()
    pp.set_skip_copies(0)
    pp.set_wait_limit(0)
    assert pp.sync_status() == pp.PP_OK
    return pp


DEV = "cuda:0"


def d64(n_steps):
    return 32 * 2.0 ** -53 * math.sqrt(n_steps)


def d32(n_steps, dt, pmax, amax):
    wmax = math.sqrt(1 + (pmax + amax) ** 2)
    return 4 * 2.0 ** -24 * wmax * dt * math.sqrt(n_steps)


def n_excess(n_gpu, n_ref, n_steps, rel=1e-9, d=None):
    """max over modes of |n_gpu - n_ref| / (rel n + 2 d sqrt(n) + d^2); <= 1 passes."""
    n_gpu = np.asarray(n_gpu).ravel()
    n_ref = np.asarray(n_ref).ravel()
    if d is None:
        d = d64(n_steps)
    tol = rel * np.abs(n_ref) + 2 * d * np.sqrt(np.abs(n_ref)) + d * d
    return float(np.max(np.abs(n_gpu - n_ref) / tol))


def rotating_gaussian():
    g = inputs.ROTATING_GAUSSIAN
    ns = g["n_steps"]
    dt = (g["t1"] - g["t0"]) / ns
    A, _, _ = oracle.gaussian_rotating_field(g["E0"], g["w"], g["tau"], g["t0"], dt / 2, 2 * ns + 1)
    return g, ns, dt, A


@pytest.fixture(scope="module")
def gauss_ref():
    g, ns, dt, A = rotating_gaussian()
    N, n = oracle.pair_number(A[None], ns, dt, g["grid"])
    return g, ns, dt, A, N, n


def test_rotating_gaussian_fp64_full_grid(pp, gauss_ref):
    g, ns, dt, A, No, no = gauss_ref
    At = torch.tensor(A[None], device=DEV)
    N, n = pp.pair_number(At, dt, g["grid"], precision="fp64", want_n=True)
    assert pp.sync_status() == pp.PP_OK
    N, n = N.cpu().numpy(), n.cpu().numpy()
    assert abs(N[0] / No[0] - 1) < 1e-9
    assert n_excess(n, no, ns) <= 1.0


def test_rotating_gaussian_fp32(pp, gauss_ref):
    g, ns, dt, A, No, no = gauss_ref
    At = torch.tensor(A[None], device=DEV)
    N, n = pp.pair_number(At, dt, g["grid"], precision="fp32", want_n=True)
    assert pp.sync_status() == pp.PP_OK
    N, n = N.cpu().numpy(), n.cpu().numpy()
    assert abs(N[0] / No[0] - 1) < 1e-4
    gr = g["grid"]
    pmax = math.sqrt(gr["x1"] ** 2 + gr["y1"] ** 2 + gr["z1"] ** 2)
    assert n_excess(n, no, ns, rel=1e-4, d=d32(ns, dt, pmax, np.abs(A).max())) <= 1.0


def oracle_n(scheme, A, n_steps, dt, pts):
    """The oracle twin of a scheme: f for the momenta pts."""
    if scheme == "rk4":
        return oracle.dirac_modes(A, n_steps, dt, pts)
    if scheme == "magnus4":
        return oracle.dirac_magnus_modes(A, n_steps, dt, pts)[0]
    return oracle.dirac_split_modes(A, n_steps, dt, pts)[0]


def weighted_N(grid, n):
    x, y, z = inputs.grid_axes(grid)

    def tw(a, mirror):
        if a.size == 1:
            return np.ones(1)
        w = np.full(a.size, a[1] - a[0])
        w[[0, -1]] /= 2
        return w * (2 if mirror else 1)
    W = (tw(z, grid["mirror_z"])[:, None, None] * tw(y, 0)[None, :, None]
         * tw(x, 0)[None, None, :])
    return float(np.sum(W.ravel() * np.asarray(n).ravel()))


@pytest.mark.parametrize("n_steps", [1, 7, 127, 128, 129, 255, 256, 257, 511, 512, 513, 1023,
                                     1025, 1100])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32fast"])
@pytest.mark.parametrize("scheme", ["rk4", "magnus4", "split2"])
def test_ragged_steps_and_modes(pp, n_steps, precision, scheme):
    # step counts around the shared-memory tiles (128..1024 steps depending on
    # scheme and precision) and a mode count (5*7*3 = 105) that fills no block;
    # each scheme against its own oracle twin
    dt = 0.05
    t0 = -0.5 * n_steps * dt
    A, _, _ = oracle.gaussian_rotating_field(0.3, 0.9, 3.0, t0, dt / 2, 2 * n_steps + 1)
    grid = inputs.small_grid(5, 7, 3, ext=1.3)
    no = oracle_n(scheme, A, n_steps, dt, inputs.grid_points(grid))
    No = weighted_N(grid, no)
    N, n = pp.pair_number(torch.tensor(A[None], device=DEV), dt, grid, precision=precision,
                          want_n=True, scheme=scheme)
    assert pp.sync_status() == pp.PP_OK
    N, n = N.cpu().numpy(), n.cpu().numpy()
    tol = 1e-9 if precision == "fp64" else 1e-4
    assert abs(N[0] / No - 1) < tol
    if precision == "fp64":
        assert n_excess(n, no, n_steps) <= 1.0


def test_uneven_steps_batch_and_single_mode_axes(pp):
    # candidates of different lengths in one launch; a grid with single-node axes
    dt = 0.04
    lens = [300, 777, 1500, 64]
    ld = 2 * max(lens) + 1
    A = np.zeros((len(lens), 2, ld))
    for c, ns in enumerate(lens):
        Ac, _, _ = oracle.gaussian_rotating_field(0.2 + 0.05 * c, 0.8, 4.0, -0.5 * ns * dt, dt / 2,
                                                  2 * ns + 1)
        A[c, :, :2 * ns + 1] = Ac
    grid = dict(nx=6, ny=1, nz=1, x0=-1.0, x1=1.0, y0=0.3, y1=0.3, z0=0.2, z1=0.2, mirror_z=0)
    for precision, tol in (("fp64", 1e-9), ("fp32", 1e-4)):
        N, n = pp.pair_number(torch.tensor(A, device=DEV), dt, grid, precision=precision,
                              n_steps=lens, want_n=True)
        assert pp.sync_status() == pp.PP_OK
        N, n = N.cpu().numpy(), n.cpu().numpy()
        for c, ns in enumerate(lens):
            No, no = oracle.pair_number(A[c:c + 1, :, :2 * ns + 1], ns, dt, grid)
            assert abs(N[c] / No[0] - 1) < tol, (precision, c)


def test_free_field_gives_zero(pp):
    A = torch.zeros((2, 2, 2 * 300 + 1), dtype=torch.float64, device=DEV)
    A[1] += 0.4  # constant potential: pure gauge
    grid = inputs.small_grid(8, 8, 4)
    for precision in ("fp64", "fp32"):
        N, n = pp.pair_number(A, 0.05, grid, precision=precision, want_n=True)
        assert pp.sync_status() == pp.PP_OK
        assert n.abs().max().item() < (1e-28 if precision == "fp64" else 1e-10)


def test_pz_mirror_symmetry_on_gpu(pp):
    g, ns, dt, A = rotating_gaussian()
    At = torch.tensor(A[None], device=DEV)
    full = dict(nx=9, ny=9, nz=9, x0=-1.2, x1=1.2, y0=-1.2, y1=1.2, z0=-1.2, z1=1.2, mirror_z=0)
    half = dict(full, nz=5, z0=0.0, mirror_z=1)
    Nf, nf = pp.pair_number(At, dt, full, precision="fp64", want_n=True)
    Nh, nh = pp.pair_number(At, dt, half, precision="fp64", want_n=True)
    nf, nh = nf.cpu().numpy()[0], nh.cpu().numpy()[0]
    # the two grids place p_z an ulp apart, so the rounding walks differ
    assert n_excess(nf[4:], nh, ns, rel=1e-12, d=2 * d64(ns)) <= 1.0
    assert n_excess(nf[:5][::-1], nh, ns, rel=1e-12, d=2 * d64(ns)) <= 1.0
    assert abs(Nf.item() / Nh.item() - 1) < 1e-10


def test_synthesis_matches_oracle(pp):
    cfg = inputs.DE_BATCH
    params = inputs.random_population(5, cfg["K"], seed=3)
    for n_steps in (8192, 1000):
        spec = dict(inputs.field_spec(cfg), n_steps=n_steps)
        A, E, s = pp.synth_field(torch.tensor(params, device=DEV), spec, want_E=True, want_scale=True)
        assert pp.sync_status() == pp.PP_OK
        Ao, Eo, so, rc = oracle.synth_field(params, cfg["K"], cfg["order"], cfg["w_min"],
                                            cfg["w_max"], cfg["T"], cfg["fluence"], n_steps)
        assert rc == 0
        A, E, s = A.cpu().numpy(), E.cpu().numpy(), s.cpu().numpy()
        assert np.abs(s / so - 1).max() < 1e-13
        for c in range(len(params)):
            assert np.abs(A[c] - Ao[c]).max() < 1e-12 * np.abs(Ao[c]).max()
            assert np.abs(E[c] - Eo[c]).max() < 1e-12 * np.abs(Eo[c]).max()


def test_synthesis_paper_band_and_order3(pp):
    # Table II band (j = 100..150, 51 modes), paper's order k = 3, N_s = 5
    T = 5000.0
    K, order = 5, 3
    params = inputs.random_population(2, K, seed=9)
    spec = dict(K=K, order=order, w_min=2 * math.pi * 0.02, w_max=2 * math.pi * 0.03, T=T,
                fluence=50.0, n_steps=4000)
    A, E, s = pp.synth_field(torch.tensor(params, device=DEV), spec, want_E=True)
    assert pp.sync_status() == pp.PP_OK
    Ao, Eo, so, rc = oracle.synth_field(params, K, order, spec["w_min"], spec["w_max"], T, 50.0, 4000)
    A, E = A.cpu().numpy(), E.cpu().numpy()
    for c in range(2):
        assert np.abs(A[c] - Ao[c]).max() < 1e-11 * np.abs(Ao[c]).max()
        assert np.abs(E[c] - Eo[c]).max() < 1e-11 * np.abs(Eo[c]).max()


def test_degenerate_field_is_reported(pp):
    cfg = inputs.DE_BATCH
    params = torch.zeros((2, 4 * cfg["K"]), dtype=torch.float64, device=DEV)
    params[1, 0:cfg["K"]] = 0.5
    spec = dict(inputs.field_spec(cfg), n_steps=200)
    A, _, s = pp.synth_field(params, spec, want_scale=True)
    assert pp.sync_status() == pp.PP_ERR_DEGENERATE_FIELD
    assert A[0].abs().max().item() == 0.0 and s[0].item() == 0.0 and s[1].item() > 0
    assert pp.sync_status() == pp.PP_OK  # the status word was cleared


def test_de_propose_and_select_bit_exact(pp):
    K = 8
    lo, hi, per = inputs.param_bounds(K)
    pop = inputs.random_population(64, K, seed=11)
    lo_t, hi_t = torch.tensor(lo, device=DEV), torch.tensor(hi, device=DEV)
    per_t = torch.tensor(per, device=DEV)
    pop_t = torch.tensor(pop, device=DEV)
    for gen in (0, 1, 17, 2 ** 40):
        for F, CR in ((0.8, 0.9), (1.7, 0.3), (0.0, 1.0)):
            tr = pp.de_propose(pop_t, lo_t, hi_t, per_t, F, CR, 123456789, gen).cpu().numpy()
            tro = oracle.de_propose(pop, lo, hi, per, F, CR, 123456789, gen)
            assert np.array_equal(tr, tro)
    # select: ties go to the trial, NaN never replaces
    fit = np.linspace(0, 1, 64)
    tfit = fit.copy()
    tfit[::3] += 0.5
    tfit[1::3] -= 0.5
    tfit[5] = np.nan
    trial = oracle.de_propose(pop, lo, hi, per, 0.8, 0.9, 5, 0)
    p_t, f_t = pop_t.clone(), torch.tensor(fit, device=DEV)
    pp.de_select(p_t, f_t, torch.tensor(trial, device=DEV), torch.tensor(tfit, device=DEV))
    po, fo = oracle.de_select(pop, fit, trial, tfit)
    assert np.array_equal(p_t.cpu().numpy(), po) and np.array_equal(f_t.cpu().numpy(), fo)


def test_de_step_matches_oracle_sequence(pp):
    cfg = inputs.DE_BATCH
    K = cfg["K"]
    spec = dict(inputs.field_spec(cfg), n_steps=400)
    grid = inputs.small_grid(6, 5, 3, ext=1.5)
    lo, hi, per = inputs.param_bounds(K)
    pop = inputs.random_population(8, K, seed=21)
    dt = spec["T"] / spec["n_steps"]
    Ao, _, _, _ = oracle.synth_field(pop, K, cfg["order"], cfg["w_min"], cfg["w_max"], cfg["T"],
                                     cfg["fluence"], spec["n_steps"], want_E=False)
    fit, _ = oracle.pair_number(Ao, spec["n_steps"], dt, grid, want_n=False)
    p_t, f_t = torch.tensor(pop, device=DEV), torch.tensor(fit, device=DEV)
    lo_t, hi_t, per_t = (torch.tensor(x, device=DEV) for x in (lo, hi, per))
    tr_t = torch.empty_like(p_t)
    tf_t = torch.empty_like(f_t)
    for gen in range(3):
        pp.de_step(p_t, f_t, spec, grid, lo_t, hi_t, per_t, 0.8, 0.9, 99, gen, precision="fp64",
                   trial_out=tr_t, trial_fit_out=tf_t)
        assert pp.sync_status() == pp.PP_OK
        tr = oracle.de_propose(pop, lo, hi, per, 0.8, 0.9, 99, gen)
        assert np.array_equal(tr, tr_t.cpu().numpy())
        At, _, _, _ = oracle.synth_field(tr, K, cfg["order"], cfg["w_min"], cfg["w_max"], cfg["T"],
                                         cfg["fluence"], spec["n_steps"], want_E=False)
        tfit, _ = oracle.pair_number(At, spec["n_steps"], dt, grid, want_n=False)
        assert np.abs(tf_t.cpu().numpy() / tfit - 1).max() < 1e-9
        # select on the GPU's trial fitness so that both sides take the same decisions
        pop, fit = oracle.de_select(pop, fit, tr, tf_t.cpu().numpy())
        assert np.array_equal(pop, p_t.cpu().numpy())
        assert np.array_equal(fit, f_t.cpu().numpy())


def test_de_batch_full_size_sampled_modes(pp):
    # The DE-batch workload at full size (64 x 64 x 32 grid, 8192 steps) in the
    # launch configuration the bench times; modes sampled for the oracle.
    cfg = inputs.DE_BATCH
    spec = inputs.field_spec(cfg)
    params = inputs.random_population(3, cfg["K"], seed=1)
    A, _, _ = pp.synth_field(torch.tensor(params, device=DEV), spec)
    dt = cfg["T"] / cfg["n_steps"]
    N64, n64 = pp.pair_number(A, dt, cfg["grid"], precision="fp64", want_n=True)
    N32, n32 = pp.pair_number(A, dt, cfg["grid"], precision="fp32", want_n=True)
    assert pp.sync_status() == pp.PP_OK
    N64, N32 = N64.cpu().numpy(), N32.cpu().numpy()
    n64, n32 = n64.cpu().numpy(), n32.cpu().numpy()
    assert np.abs(N32 / N64 - 1).max() < 1e-4
    Ah = A.cpu().numpy()
    pts = inputs.grid_points(cfg["grid"])
    for c in range(2):
        idx = inputs.strided_modes(cfg["grid"], 48, seed=c)
        # include the largest mode of this candidate
        idx = np.unique(np.concatenate([idx, [int(np.argmax(n64[c]))]]))
        no = oracle.dirac_modes(Ah[c], cfg["n_steps"], dt, pts[idx])
        ng = n64[c].ravel()[idx]
        assert n_excess(ng, no, cfg["n_steps"]) <= 1.0


def test_de_batch_full_grid_against_the_oracle(pp):
    # The metric's own check at the DE-batch size (Sec. II.A, Eqs. (pair_prod_homo),
    # (opt_prob)): the oracle's N over the whole 64 x 64 x 32 grid and 8192 RK4 steps of
    # one candidate, synthesised by each side from the same parameters, against the
    # timed path (Magnus-4, FP32 without compensation: 1e-4) and the FP64 RK4 path (1e-9).
    cfg = inputs.DE_BATCH
    params = inputs.random_population(1, cfg["K"], seed=1)
    ns, dt = cfg["n_steps"], cfg["T"] / cfg["n_steps"]
    Ao, _, _, rc = oracle.synth_field(params, cfg["K"], cfg["order"], cfg["w_min"], cfg["w_max"], cfg["T"],
                                      cfg["fluence"], ns, want_E=False)
    assert rc == 0
    No, no = oracle.pair_number(Ao, ns, dt, cfg["grid"])
    A, _, _ = pp.synth_field(torch.tensor(params, device=DEV), inputs.field_spec(cfg))
    Nf, _ = pp.pair_number(A, dt, cfg["grid"], precision="fp32fast", scheme="magnus4")
    N64, n64 = pp.pair_number(A, dt, cfg["grid"], precision="fp64", scheme="rk4", want_n=True)
    assert pp.sync_status() == pp.PP_OK
    assert abs(Nf.item() / No[0] - 1) < 1e-4
    assert abs(N64.item() / No[0] - 1) < 1e-9
    assert n_excess(n64.cpu().numpy(), no, ns) <= 1.0


def test_large_scale_size_sampled_modes(pp):
    """The large-scale configuration's size (K = 16, T = 400, 20000 steps, grid
    128 x 128 x 64 over [-2.5, 2.5]^2 x [0, 2.5]) for one candidate: FP64 RK4 on the
    GPU against the oracle on sampled modes (including the largest), and the timed
    FP32 Magnus path against FP64 on N."""
    cfg = inputs.LARGE_SCALE
    spec = inputs.field_spec(cfg)
    params = inputs.random_population(1, cfg["K"], seed=cfg["pop_seed"])
    A, _, _ = pp.synth_field(torch.tensor(params, device=DEV), spec)
    dt = cfg["T"] / cfg["n_steps"]
    N64, n64 = pp.pair_number(A, dt, cfg["grid"], precision="fp64", scheme="rk4", want_n=True)
    N32, _ = pp.pair_number(A, dt, cfg["grid"], precision="fp32fast", scheme="magnus4")
    assert pp.sync_status() == pp.PP_OK
    assert abs(N32.item() / N64.item() - 1) < 1e-4
    n64 = n64[0].cpu().numpy().ravel()
    idx = inputs.strided_modes(cfg["grid"], 16, seed=4)
    idx = np.unique(np.concatenate([idx, [int(np.argmax(n64))]]))
    no = oracle.dirac_modes(A[0].cpu().numpy(), cfg["n_steps"], dt, inputs.grid_points(cfg["grid"])[idx])
    assert n_excess(n64[idx], no, cfg["n_steps"]) <= 1.0


def test_uneven_batch_full_size(pp):
    """The uneven-batch workload at full size (128 slots, 2500..20000 steps, grids
    32..96 by peak-field quintile) in the timed path (FP32-fast Magnus): three slots
    (shortest, longest, finest grid) against FP64 RK4 through the uniform path, and
    sampled modes of the longest against the oracle."""
    U = inputs.UNEVEN_BATCH
    steps = inputs.uneven_steps(U, 1)
    specs = inputs.uneven_specs(U, steps)
    pop = torch.tensor(inputs.random_population(U["NP"], U["K"], seed=1), device=DEV)
    peaks = []
    for c, sp in enumerate(specs):
        _, E, _ = pp.synth_field(pop[c:c + 1].contiguous(), sp, want_E=True)
        peaks.append(torch.sqrt(E[0, 0] ** 2 + E[0, 1] ** 2).max().item())
    grids = inputs.grids_by_rank(U, peaks)
    b = pp.Batch(specs, grids, U["dt"], precision="fp32fast", scheme="magnus4")
    A = b.synth(pop)
    N, _ = b.pair_number(A)
    assert pp.sync_status() == pp.PP_OK
    sizes = [g["nx"] * g["ny"] * g["nz"] for g in grids]
    picks = sorted({int(np.argmin(steps)), int(np.argmax(steps)), int(np.argmax(sizes))})
    for c in picks:
        ns = int(steps[c])
        Ac = A[c:c + 1, :, :2 * ns + 1].contiguous()
        N64, n64 = pp.pair_number(Ac, U["dt"], grids[c], precision="fp64", scheme="rk4",
                                  want_n=c == int(np.argmax(steps)))
        assert pp.sync_status() == pp.PP_OK
        assert abs(N[c].item() / N64.item() - 1) < 1e-4, c
        if n64 is not None:
            nn = n64[0].cpu().numpy().ravel()
            idx = inputs.strided_modes(grids[c], 12, seed=c)
            idx = np.unique(np.concatenate([idx, [int(np.argmax(nn))]]))
            no = oracle.dirac_modes(Ac[0].cpu().numpy(), ns, U["dt"], inputs.grid_points(grids[c])[idx])
            assert n_excess(nn[idx], no, ns) <= 1.0
    b.close()


@pytest.mark.parametrize("scheme", ["magnus4", "split2"])
def test_unitary_schemes_on_the_rotating_gaussian(pp, gauss_ref, scheme):
    g, ns, dt, A, No_rk4, _ = gauss_ref
    pts = inputs.grid_points(g["grid"])
    sub = inputs.strided_modes(g["grid"], 600, seed=5)
    no_sub = oracle_n(scheme, A, ns, dt, pts[sub])
    At = torch.tensor(A[None], device=DEV)
    N64, n64 = pp.pair_number(At, dt, g["grid"], precision="fp64", want_n=True, scheme=scheme)
    N32, _ = pp.pair_number(At, dt, g["grid"], precision="fp32", scheme=scheme)
    assert pp.sync_status() == pp.PP_OK
    assert n_excess(n64.cpu().numpy().ravel()[sub], no_sub, ns) <= 1.0
    assert abs(N32.item() / N64.item() - 1) < 1e-4
    # against the RK4 oracle: the fourth-order scheme agrees far inside 1e-4 at this dt
    if scheme == "magnus4":
        assert abs(N64.item() / No_rk4[0] - 1) < 1e-6


def test_magnus_fp32_at_full_de_batch_size(pp):
    cfg = inputs.DE_BATCH
    spec = inputs.field_spec(cfg)
    params = inputs.random_population(4, cfg["K"], seed=2)
    A, _, _ = pp.synth_field(torch.tensor(params, device=DEV), spec)
    dt = cfg["T"] / cfg["n_steps"]
    N_rk4, _ = pp.pair_number(A, dt, cfg["grid"], precision="fp64", scheme="rk4")
    N_m64, n_m64 = pp.pair_number(A, dt, cfg["grid"], precision="fp64", scheme="magnus4",
                                  want_n=True)
    N_m32, _ = pp.pair_number(A, dt, cfg["grid"], precision="fp32", scheme="magnus4")
    assert pp.sync_status() == pp.PP_OK
    assert (N_m32 / N_rk4 - 1).abs().max().item() < 1e-4
    assert (N_m32 / N_m64 - 1).abs().max().item() < 1e-5
    Ah = A.cpu().numpy()
    pts = inputs.grid_points(cfg["grid"])
    idx = inputs.strided_modes(cfg["grid"], 24, seed=3)
    no = oracle.dirac_magnus_modes(Ah[0], cfg["n_steps"], dt, pts[idx])[0]
    assert n_excess(n_m64[0].cpu().numpy().ravel()[idx], no, cfg["n_steps"]) <= 1.0


def magnus_theta_bound(A, dt, grid):
    """Largest per-step bound on th = |dt h_eff| over the grid, as pp.h defines it for
    PP_MAGNUS4 (restated here from that definition, in FP64)."""
    Px, Py = max(abs(grid["x0"]), abs(grid["x1"])), max(abs(grid["y0"]), abs(grid["y1"]))
    Em = math.sqrt(1 + max(grid["z0"] ** 2, grid["z1"] ** 2))
    a0x, ahx, a1x = A[0, 0:-1:2], A[0, 1::2], A[0, 2::2]
    a0y, ahy, a1y = A[1, 0:-1:2], A[1, 1::2], A[1, 2::2]
    ax, ay = dt * (a0x + 4 * ahx + a1x) / 6, dt * (a0y + 4 * ahy + a1y) / 6
    d6 = dt * dt / 6
    dx, dy, c = d6 * (a0x - a1x), d6 * (a1y - a0y), d6 * (a0x * a1y - a0y * a1x)
    bx = dt * Px + np.abs(ax) + Em * np.abs(dy)
    by = dt * Py + np.abs(ay) + Em * np.abs(dx)
    bz = dt * Em + np.abs(dy) * Px + np.abs(dx) * Py + np.abs(c)
    return float(np.sqrt(bx ** 2 + by ** 2 + bz ** 2).max())


@pytest.mark.parametrize("target", [0.19, 0.4, 0.8])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32fast"])
def test_magnus_beyond_the_series_range(pp, target, precision):
    # Sec. V.C.2 (a unitary fourth-order step): the Magnus step must stay exact when
    # th = |dt h_eff| leaves the range of its polynomials (th <= 0.2).  At 0.19 every
    # tile uses the polynomials; at 0.4 and 0.8 the argument-halved form.  Against the
    # oracle twin, which exponentiates the 4x4 Omega by its full Taylor series.
    grid = inputs.small_grid(6, 5, 3, ext=1.3)
    dt = 0.05
    for _ in range(3):  # scale dt until the bound hits the target
        ns = int(round(24.0 / dt))
        A, _, _ = oracle.gaussian_rotating_field(0.3, 0.9, 3.0, -0.5 * ns * dt, dt / 2, 2 * ns + 1)
        dt *= target / magnus_theta_bound(A, dt, grid)
    ns = int(round(24.0 / dt))
    A, _, _ = oracle.gaussian_rotating_field(0.3, 0.9, 3.0, -0.5 * ns * dt, dt / 2, 2 * ns + 1)
    assert abs(magnus_theta_bound(A, dt, grid) - target) < 0.01
    no = oracle.dirac_magnus_modes(A, ns, dt, inputs.grid_points(grid))[0]
    No = weighted_N(grid, no)
    N, n = pp.pair_number(torch.tensor(A[None], device=DEV), dt, grid, precision=precision,
                          want_n=True, scheme="magnus4")
    assert pp.sync_status() == pp.PP_OK
    N, n = N.cpu().numpy(), n.cpu().numpy()
    if precision == "fp64":
        assert abs(N[0] / No - 1) < 1e-9
        assert n_excess(n, no, ns) <= 1.0
    else:
        assert abs(N[0] / No - 1) < 1e-4


@pytest.mark.parametrize("precision", ["fp32", "fp32fast"])
def test_magnus_fp32_tracked_norm_over_many_tiles(pp, precision):
    # The FP32 series step applies exp(-i H.sigma) / cos th, so the state grows by
    # 1 / cos th per step: here th ~ 0.19 for ~2600 steps (a growth of ~1e21 without
    # the power-of-two rescaling between tiles, past the FP32 range in its square).
    # N must match the oracle twin, and the rescaling, being exact, must not show:
    # every launch configuration (tiles of 256 or 1024 steps) gives the same N bit for bit.
    grid = inputs.small_grid(6, 5, 3, ext=1.3)
    dt, T = 0.05, 312.0
    for _ in range(3):
        ns = int(round(T / dt))
        A, _, _ = oracle.gaussian_rotating_field(0.3, 0.9, 3.0, -0.5 * ns * dt, dt / 2, 2 * ns + 1)
        dt *= 0.19 / magnus_theta_bound(A, dt, grid)
    ns = int(round(T / dt))
    A, _, _ = oracle.gaussian_rotating_field(0.3, 0.9, 3.0, -0.5 * ns * dt, dt / 2, 2 * ns + 1)
    assert ns > 2000 and abs(magnus_theta_bound(A, dt, grid) - 0.19) < 0.01
    No = weighted_N(grid, oracle.dirac_magnus_modes(A, ns, dt, inputs.grid_points(grid))[0])
    At = torch.tensor(A[None], device=DEV)
    pp.clear_tuning()
    N0, _ = pp.pair_number(At, dt, grid, precision=precision, scheme="magnus4")
    _, ms, N_last = pp.tune_pair_number(At, dt, grid, precision=precision, scheme="magnus4")
    assert pp.sync_status() == pp.PP_OK
    pp.clear_tuning()
    assert np.isfinite(N0.item()) and abs(N0.item() / No - 1) < 1e-4
    assert torch.equal(N0, N_last)


@pytest.mark.parametrize("precision,scheme", [("fp32", "magnus4"), ("fp32fast", "magnus4"),
                                              ("fp32", "rk4"), ("fp32fast", "split2"),
                                              ("fp64", "rk4")])
def test_tuner_picks_a_config_and_results_do_not_depend_on_it(pp, precision, scheme):
    cfg = inputs.DE_BATCH
    spec = dict(inputs.field_spec(cfg), n_steps=1500)
    params = inputs.random_population(3, cfg["K"], seed=23)
    A, _, _ = pp.synth_field(torch.tensor(params, device=DEV), spec)
    grid = inputs.small_grid(20, 19, 7, ext=2.0)  # 2660 modes: partial CTAs for every size
    dt = spec["T"] / spec["n_steps"]
    pp.clear_tuning()
    N_default, _ = pp.pair_number(A, dt, grid, precision=precision, scheme=scheme)
    chosen, ms, N_last = pp.tune_pair_number(A, dt, grid, precision=precision, scheme=scheme)
    N_tuned, _ = pp.pair_number(A, dt, grid, precision=precision, scheme=scheme)
    assert pp.sync_status() == pp.PP_OK
    configs = pp.launch_configs()
    assert len(configs) == len(ms) == 6
    assert 0 <= chosen < 6 and all(t > 0 for t in ms) and ms[chosen] == min(ms)
    # the momentum sum is taken over fixed groups of 128 modes: bitwise equal N
    assert torch.equal(N_default, N_last) and torch.equal(N_default, N_tuned)
    pp.clear_tuning()


def test_results_are_bitwise_reproducible(pp):
    g, ns, dt, A = rotating_gaussian()
    At = torch.tensor(A[None], device=DEV).repeat(3, 1, 1)
    out = [pp.pair_number(At, dt, g["grid"], precision=p)[0].cpu().numpy()
           for p in ("fp32", "fp32", "fp64", "fp64", "fp32fast", "fp32fast")]
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[2], out[3])
    assert np.array_equal(out[4], out[5])


def test_bounded_wait_timeout_reports_and_context_survives(pp):
    # The propagation kernel waits on a barrier that nothing completes (its tile
    # copies are switched off); the bounded wait gives up, the kernel records
    # PP_ERR_TIMEOUT and returns; the next normal call works.
    g, ns, dt, A = rotating_gaussian()
    At = torch.tensor(A[None], device=DEV)
    grid = inputs.small_grid(8, 8, 2)
    old = pp.set_wait_limit(2000)
    pp.set_skip_copies(1)
    try:
        N, _ = pp.pair_number(At, dt, grid, precision="fp32")
        st = pp.sync_status()
    finally:
        pp.set_skip_copies(0)
        pp.set_wait_limit(old)
    assert st == pp.PP_ERR_TIMEOUT
    assert math.isnan(N.item())
    N2, _ = pp.pair_number(At, dt, grid, precision="fp32")
    assert pp.sync_status() == pp.PP_OK and math.isfinite(N2.item())


def test_invalid_arguments_raise(pp):
    A = torch.zeros((1, 2, 11), dtype=torch.float64, device=DEV)
    with pytest.raises(pp.PPError) as e:
        pp.pair_number(A, 0.1, inputs.small_grid(2, 2, 2), n_steps=[6])
    assert e.value.code == pp.PP_ERR_INVALID_ARG


def test_release_scratch_then_reuse(pp):
    """pp_release_scratch frees the scratch; the next call allocates it again and
    gives the same result."""
    g, ns, dt, A = rotating_gaussian()
    At = torch.tensor(A[None], device=DEV)
    grid = inputs.small_grid(8, 8, 2)
    N1, _ = pp.pair_number(At, dt, grid, precision="fp64")
    pp.release_scratch()
    N2, _ = pp.pair_number(At, dt, grid, precision="fp64")
    assert pp.sync_status() == pp.PP_OK
    assert torch.equal(N1, N2)


def test_empty_inputs_are_no_ops(pp):
    """Zero candidates: every scoring entry point returns at once with empty results
    and leaves no error behind (the launch-configuration tuner, which needs a
    workload to time, refuses them instead)."""
    cfg = inputs.DE_BATCH
    n = 200
    spec = dict(inputs.field_spec(cfg), n_steps=n)
    grid = inputs.small_grid(3, 3, 2)
    dt = spec["T"] / n
    P = torch.empty((0, 4 * cfg["K"]), dtype=torch.float64, device=DEV)
    A, E, s = pp.synth_field(P, spec, want_E=True, want_scale=True)
    assert A.shape == (0, 2, 2 * n + 1) and s.shape == (0,)
    for precision in ("fp64", "fp32", "fp32fast"):
        N, nn = pp.pair_number(A, dt, grid, precision=precision, want_n=True)
        assert N.shape == (0,) and nn.shape[0] == 0
    N, _ = pp.pair_number_static(A, dt, grid, precision="fp32")
    assert N.shape == (0,)
    Ar, Er, Edr, Ur = pp.synth_field_raw(P, spec)
    assert Ar.shape == (0, 2, 2 * n + 1)
    J, _ = pp.qke_pair_number(Ar, Er, Edr, dt, grid, "fp32")
    assert J.shape == (0,)
    g = torch.empty((0, 6, 2 * n + 1), dtype=torch.float64, device=DEV)
    grad, U, dU = pp.synth_vjp(P, spec, g)
    assert grad.shape == (0, 4 * cfg["K"])
    J, gJ, U, dU = pp.qke_gradient(P, spec, grid, "fp32")
    assert J.shape == (0,) and gJ.shape == (0, 4 * cfg["K"])
    assert pp.sync_status() == pp.PP_OK
    with pytest.raises(pp.PPError):
        pp.tune_pair_number(A, dt, grid)
    assert pp.sync_status() == pp.PP_OK
