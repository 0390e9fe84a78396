"""The Hann envelope (Eq. (hann)) on the GPU against the oracle: the GPU writes
the enveloped field as a trigonometric polynomial with transformed coefficients,
the oracle evaluates the paper's closed form (Eq. (vector_potential)) directly."""
import numpy as np
import pytest

import oracle
from paper_1704_08919_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

K, ORDER, T = 8, 4, 50.0
DEV = "cuda:0"


@pytest.fixture(scope="module")
def pp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_08919_gb300 import build
    build.build()
    import paper_1704_08919_gb300 as pp
    pp.lib()
    assert pp.sync_status() == pp.PP_OK
    return pp


def spec(n, wmin=0.0, U=2.0):
    return dict(K=K, order=ORDER, w_min=wmin, w_max=2.0, T=T, fluence=U, n_steps=n, envelope=1)


@pytest.mark.parametrize("n,wmin", [(203, 0.0), (1000, 0.0), (999, 0.5)])
def test_synthesis_matches_oracle(pp, n, wmin):
    x = inputs.random_population(3, K, seed=n)
    A, E, s = pp.synth_field(torch.tensor(x, device=DEV), spec(n, wmin), want_E=True, want_scale=True)
    Ao, Eo, _, so = oracle.synth_hann(x, K, ORDER, wmin, 2.0, T, 2.0, n)
    assert pp.sync_status() == pp.PP_OK
    assert np.abs(A.cpu().numpy() - Ao).max() < 1e-12 * np.abs(Ao).max()
    assert np.abs(E.cpu().numpy() - Eo).max() < 1e-12 * np.abs(Eo).max()
    assert np.abs(s.cpu().numpy() / so - 1).max() < 1e-13


def test_raw_synthesis_with_time_derivative(pp):
    n = 600
    x = inputs.random_population(2, K, seed=9) * 0.1
    A, E, Ed, U = pp.synth_field_raw(torch.tensor(x, device=DEV), spec(n))
    Ao, Eo, Edo, Uo = oracle.synth_hann(x, K, ORDER, 0.0, 2.0, T, 1.0, n, normalize=False)
    assert pp.sync_status() == pp.PP_OK
    for g, o in ((A, Ao), (E, Eo), (Ed, Edo)):
        assert np.abs(g.cpu().numpy() - o).max() < 1e-12 * np.abs(o).max()
    assert np.abs(U.cpu().numpy() / Uo - 1).max() < 1e-12


def test_pair_number_of_an_enveloped_pulse(pp):
    n = 1200
    grid = inputs.small_grid(7, 6, 3)
    x = inputs.random_population(2, K, seed=11)
    A, _, _ = pp.synth_field(torch.tensor(x, device=DEV), spec(n))
    N, _ = pp.pair_number(A, T / n, grid, precision="fp64", scheme="rk4")
    assert pp.sync_status() == pp.PP_OK
    Ao, _, _, _ = oracle.synth_hann(x, K, ORDER, 0.0, 2.0, T, 2.0, n)
    No, _ = oracle.pair_number(Ao, n, T / n, grid)
    assert np.abs(N.cpu().numpy() / No - 1).max() < 1e-9


def test_de_step_with_the_envelope(pp):
    n = 400
    grid = inputs.small_grid(5, 5, 2)
    sp = spec(n)
    x = inputs.random_population(6, K, seed=13)
    lo, hi, per = inputs.param_bounds(K)
    pop = torch.tensor(x, device=DEV)
    A, _, _ = pp.synth_field(pop, sp)
    fit, _ = pp.pair_number(A, T / n, grid, precision="fp64", scheme="rk4")
    trial = torch.empty_like(pop)
    tfit = torch.empty_like(fit)
    lt, ht, pt = (torch.tensor(v, device=DEV) for v in (lo, hi, per))
    pp.de_step(pop, fit, sp, grid, lt, ht, pt, 0.8, 0.9, 5, 0, precision="fp64", scheme="rk4",
               trial_out=trial, trial_fit_out=tfit)
    assert pp.sync_status() == pp.PP_OK
    to = oracle.de_propose(x, lo, hi, per, 0.8, 0.9, 5, 0)
    assert np.array_equal(trial.cpu().numpy(), to)
    Ao, _, _, _ = oracle.synth_hann(to, K, ORDER, 0.0, 2.0, T, 2.0, n)
    No, _ = oracle.pair_number(Ao, n, T / n, grid)
    assert np.abs(tfit.cpu().numpy() / No - 1).max() < 1e-9


# ---- the chain rule through the envelope (the local search's gradient), on the
# small QKE workload of the local-search tests: K = 4, order 3, T = 20
KQ, ORDQ, TQ = 4, 3, 20.0


def qspec(n):
    return dict(K=KQ, order=ORDQ, w_min=0.0, w_max=2.0, T=TQ, fluence=1.0, n_steps=n, envelope=1)


def qparams(nc, seed, U=1.5):
    """nc random parameter vectors with the amplitude weights scaled so that the
    enveloped field has fluence U."""
    lo, hi, _ = inputs.param_bounds(KQ)
    rng = np.random.default_rng(seed)
    X = lo + rng.random((nc, 4 * KQ)) * (hi - lo)
    _, _, _, U0 = oracle.synth_hann(X, KQ, ORDQ, 0.0, 2.0, TQ, 1.0, 100, normalize=False)
    for x, u in zip(X, U0):
        s = np.sqrt(U / u)
        x[:KQ] *= s
        x[2 * KQ:3 * KQ] *= s
    return X


def dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


@pytest.mark.parametrize("n,wmin", [(300, 0.0), (777, 0.3)])
def test_chain_rule_matches_oracle(pp, n, wmin):
    """pp_synth_vjp with the envelope against the oracle's transpose of the closed
    form, for random sample weights; the fluence and its gradient too."""
    X = inputs.random_population(3, K, seed=n) * 0.3
    rng = np.random.default_rng(n)
    g = rng.normal(size=(3, 6, 2 * n + 1))
    sp = spec(n, wmin)
    grad, U, dU = pp.synth_vjp(dev(X), sp, dev(g))
    assert pp.sync_status() == pp.PP_OK
    grad, U, dU = grad.cpu().numpy(), U.cpu().numpy(), dU.cpu().numpy()
    for c in range(3):
        go, Uo, dUo = oracle.synth_vjp_hann(X[c], K, ORDER, wmin, 2.0, T, n,
                                            g[c, 0:2], g[c, 2:4], g[c, 4:6])
        assert np.abs(grad[c] - go).max() < 1e-11 * np.abs(go).max()
        assert abs(U[c] / Uo - 1) < 1e-13
        assert np.abs(dU[c] - dUo).max() < 1e-13 * np.abs(dUo).max()


def test_parameter_gradient_matches_oracle(pp):
    n = 2000
    grid = inputs.small_grid(5, 5, 3)
    X = qparams(3, 4)
    J, gJ, U, dU = pp.qke_gradient(dev(X), qspec(n), grid, "fp64")
    J32, gJ32, _, _ = pp.qke_gradient(dev(X), qspec(n), grid, "fp32")
    assert pp.sync_status() == pp.PP_OK
    for c in range(3):
        o = oracle.al_objective(X[c], qspec(n), grid, 2.0, 0.0, 1.0)
        assert np.isfinite(o["J"])
        assert abs(J[c].item() / o["J"] - 1) < 1e-9
        assert np.abs(gJ[c].cpu().numpy() - o["gJ"]).max() < 1e-9 * np.abs(o["gJ"]).max()
        assert np.abs(dU[c].cpu().numpy() + o["gC"]).max() < 1e-12 * np.abs(o["gC"]).max()
        assert abs(U[c].item() - (2.0 - o["C"])) < 1e-12
        assert abs(J32[c].item() / o["J"] - 1) < 1e-4
        assert np.linalg.norm(gJ32[c].cpu().numpy() - o["gJ"]) < 1e-3 * np.linalg.norm(o["gJ"])


def test_local_search_first_iterates_match_oracle(pp):
    """The GPU local search over enveloped pulses takes the oracle's first BFGS iterates."""
    from oracle import localsearch as LS
    n = 2000
    grid = inputs.small_grid(4, 4, 2)
    starts = qparams(2, 9)
    kw = dict(mu0=0.1, xi=0.5, outer=1, max_iter=3, gtol=1e-12, ctol=1e-12)
    r = pp.local_search(starts, qspec(n), grid, 2.0, precision="fp64", **kw)
    assert pp.sync_status() == pp.PP_OK

    def obj(z):
        o = oracle.al_objective(z, qspec(n), grid, 2.0, 0.0, 1.0)
        return o["J"], o["gJ"], o["C"], o["gC"]
    for i in range(2):
        o = LS.augmented_lagrangian(obj, starts[i], **kw)
        assert r["evals"][i] == o["evals"]
        assert np.abs(r["x"][i] - o["x"]).max() < 1e-7 * np.abs(o["x"]).max()
        assert abs(r["J"][i] / o["J"] - 1) < 1e-8
