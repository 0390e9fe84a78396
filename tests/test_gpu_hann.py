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


def test_paths_without_the_envelope_reject_it(pp):
    x = torch.tensor(inputs.random_population(2, K, seed=1), device=DEV)
    with pytest.raises(pp.PPError) as e:
        pp.qke_gradient(x, spec(100), inputs.small_grid(2, 2, 1))
    assert e.value.code == pp.PP_ERR_NOT_IMPLEMENTED
    with pytest.raises(pp.PPError):
        pp.Batch([spec(100), spec(120)], [inputs.small_grid(2, 2, 1)] * 2, T / 100)
    assert pp.sync_status() == pp.PP_OK
