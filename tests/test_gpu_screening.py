"""Surrogate-screened DE (pp_de_screened_step) and the training entry points
(pp_mlp_init, pp_mlp_fit, pp_mlp_log_targets) on the GPU.

The screened step is checked as a composition of entry points that are tested
on their own against the oracle: with one proposal it is plain DE bit for bit;
with R proposals its predictions are the network's forward pass on the
proposals of generations R g + r, and the trial it scores is their argmax.  A
small end-to-end run shows that the trained network reaches plain DE's best N
with fewer exact solver calls."""
import math

import numpy as np
import pytest

from paper_1704_08919_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

K = 8
SPEC = dict(K=K, order=4, w_min=0.0, w_max=2.0, T=50.0, fluence=2.0, n_steps=1024)
GRID = inputs.small_grid(16, 16, 8)


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


def bounds():
    return (torch.tensor(x, device="cuda") for x in inputs.param_bounds(K))


def start(pp, NP, seed):
    pop = torch.tensor(inputs.random_population(NP, K, seed=seed), device="cuda")
    A, _, _ = pp.synth_field(pop, SPEC)
    fit, _ = pp.pair_number(A, SPEC["T"] / SPEC["n_steps"], GRID, precision="fp32fast",
                            scheme="magnus4")
    return pop, fit


def test_init_statistics(pp):
    net = pp.Surrogate(32, 256, max_batch=256)
    net.init(5)
    p = net.get_params().cpu().double().numpy()
    H, d = 256, 32
    W1 = p[:H * d]
    b1 = p[H * d:H * d + H]
    W2 = p[H * d + H:H * d + H + H * H]
    assert np.all(b1 == 0.0) and p[-1] == 0.0
    assert abs(W1.mean()) < 4 * math.sqrt(2.0 / d) / math.sqrt(W1.size)
    assert abs(W1.std() / math.sqrt(2.0 / d) - 1) < 0.05
    assert abs(W2.std() / math.sqrt(2.0 / H) - 1) < 0.02
    net.init(5)
    assert np.array_equal(net.get_params().cpu().double().numpy(), p)  # counter-based: reproducible
    net.close()


def test_log_targets(pp):
    N = torch.tensor([1e-12, 3.5e-4, 0.0, 2.0], dtype=torch.float64, device="cuda")
    t = pp.log_targets(N, 1e-30, -5.0, 2.0).cpu().numpy()
    ref = (np.log10(np.maximum(N.cpu().numpy(), 1e-30)) + 5.0) / 2.0
    assert np.allclose(t, ref.astype(np.float32), rtol=1e-6, atol=1e-6)


def test_fit_reduces_loss(pp):
    rng = np.random.default_rng(3)
    X = rng.uniform(-0.5, 0.5, (3000, 32))  # 3000 rows: ragged last slice of 256
    y = np.tanh(X @ rng.normal(size=32))
    net = pp.Surrogate(32, 256, max_batch=256)
    net.init(2)
    Xg = torch.tensor(X, dtype=torch.float32, device="cuda")
    tg = torch.tensor(y, dtype=torch.float32, device="cuda")
    before = float(np.mean((net.forward(Xg[:256].contiguous()).cpu().numpy() - y[:256]) ** 2))
    L = net.fit(Xg, tg, 256, 20, 2e-3, 1e-4).cpu().numpy()
    after = float(np.mean((net.forward(Xg[:256].contiguous()).cpu().numpy() - y[:256]) ** 2))
    assert pp.sync_status() == pp.PP_OK
    assert np.all(np.isfinite(L)) and L[-1] < 0.1 * L[0]
    assert after < 0.05 * before
    net.close()


M64 = (1 << 64) - 1


def sm64(s, k):
    """SplitMix64 output k of seed s (Steele, Lea, Flood 2014), restated for the test."""
    z = (s + (k + 1) * 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def epoch_order(n, seed, e):
    """Row order of epoch e as pp.h defines it for pp_mlp_fit: a 4-round Feistel network
    on b-bit integers (b even, 2^b >= n), applied again while the value is >= n."""
    hb = 0
    while (1 << (2 * hb)) < n:
        hb += 1
    mask = (1 << hb) - 1
    keys = [sm64(seed, 4 * e + i) for i in range(4)]
    out = []
    for x in range(n):
        while True:
            L, R = x >> hb, x & mask
            for k in keys:
                L, R = R, L ^ (sm64(k, R) & mask)
            x = (L << hb) | R
            if x < n:
                break
        out.append(x)
    return out


@pytest.mark.parametrize("seed", [0, 99])
def test_fit_visits_rows_in_the_documented_order(pp, seed):
    # pp_mlp_fit equals pp_mlp_train_step on the rows of each slice gathered in the
    # documented order (seed 0: as given), bit for bit; constant learning rate
    n, batch, epochs, lr = 700, 128, 3, 1e-3
    rng = np.random.default_rng(5)
    X = torch.tensor(rng.uniform(-0.5, 0.5, (n, 32)), dtype=torch.float32, device="cuda")
    t = torch.tensor(rng.normal(size=n), dtype=torch.float32, device="cuda")
    a = pp.Surrogate(32, 128, max_batch=128)
    b = pp.Surrogate(32, 128, max_batch=128)
    a.init(4)
    b.init(4)
    a.fit(X, t, batch, epochs, lr, lr, seed=seed)
    orders = []
    for e in range(epochs):
        order = list(range(n)) if seed == 0 else epoch_order(n, seed, e)
        assert sorted(order) == list(range(n))
        orders.append(order)
        idx = torch.tensor(order, device="cuda")
        for r0 in range(0, n, batch):
            rows = idx[r0:r0 + batch]
            b.train_step(X[rows].contiguous(), t[rows].contiguous(), lr)
    assert pp.sync_status() == pp.PP_OK
    assert torch.equal(a.get_params(), b.get_params())
    if seed:
        assert orders[0] != orders[1] and orders[0] != list(range(n))
    a.close()
    b.close()


def test_one_proposal_is_plain_de(pp):
    lo, hi, per = bounds()
    pop0, fit0 = start(pp, 16, 21)
    net = pp.Surrogate(32, 256, max_batch=64)
    net.init(9)
    a_pop, a_fit = pop0.clone(), fit0.clone()
    b_pop, b_fit = pop0.clone(), fit0.clone()
    for g in range(3):
        pp.de_step(a_pop, a_fit, SPEC, GRID, lo, hi, per, 0.8, 0.9, 31, g, precision="fp32fast",
                   scheme="magnus4")
        pp.de_screened_step(b_pop, b_fit, SPEC, GRID, lo, hi, per, 0.8, 0.9, 31, g, 1, net,
                            precision="fp32fast", scheme="magnus4")
    assert pp.sync_status() == pp.PP_OK
    assert torch.equal(a_pop, b_pop) and torch.equal(a_fit, b_fit)
    net.close()


@pytest.mark.parametrize("NP,R,gen", [(16, 4, 0), (13, 8, 5)])
def test_screened_step_is_the_composition(pp, NP, R, gen):
    lo, hi, per = bounds()
    pop0, fit0 = start(pp, NP, 40 + NP)
    net = pp.Surrogate(32, 256, max_batch=R * NP)
    net.init(3)
    pop, fit = pop0.clone(), fit0.clone()
    trial = torch.empty_like(pop)
    tfit = torch.empty_like(fit)
    pred = torch.empty(R * NP, dtype=torch.float32, device="cuda")
    pp.de_screened_step(pop, fit, SPEC, GRID, lo, hi, per, 0.8, 0.9, 77, gen, R, net,
                        precision="fp32fast", scheme="magnus4", trial_out=trial,
                        trial_fit_out=tfit, pred_out=pred)
    props = torch.cat([pp.de_propose(pop0, lo, hi, per, 0.8, 0.9, 77, gen * R + r)
                       for r in range(R)])
    y = net.forward(pp.mlp_features(props, lo, hi))
    assert pp.sync_status() == pp.PP_OK
    assert torch.equal(y, pred)
    yy = y.cpu().numpy().reshape(R, NP)
    best = np.argmax(yy, axis=0)  # first maximum
    P = props.cpu().numpy().reshape(R, NP, -1)
    assert np.array_equal(trial.cpu().numpy(), P[best, np.arange(NP)])
    A, _, _ = pp.synth_field(trial, SPEC)
    Nx, _ = pp.pair_number(A, SPEC["T"] / SPEC["n_steps"], GRID, precision="fp32fast",
                           scheme="magnus4")
    assert torch.equal(Nx, tfit)
    take = (tfit >= fit0).cpu().numpy()
    exp_pop = np.where(take[:, None], trial.cpu().numpy(), pop0.cpu().numpy())
    assert np.array_equal(pop.cpu().numpy(), exp_pop)
    assert np.array_equal(fit.cpu().numpy(), np.where(take, tfit.cpu().numpy(), fit0.cpu().numpy()))
    net.close()


@pytest.mark.parametrize("NP,R,gen", [(16, 4, 1), (13, 8, 2)])
def test_global_screening_is_the_composition(pp, NP, R, gen):
    lo, hi, per = bounds()
    pop0, fit0 = start(pp, NP, 60 + NP)
    net = pp.Surrogate(32, 256, max_batch=R * NP)
    net.init(4)
    pop, fit = pop0.clone(), fit0.clone()
    trial = torch.empty_like(pop)
    tfit = torch.empty_like(fit)
    pred = torch.empty(R * NP, dtype=torch.float32, device="cuda")
    kept = torch.empty(NP, dtype=torch.int32, device="cuda")
    pp.de_screened_step(pop, fit, SPEC, GRID, lo, hi, per, 0.8, 0.9, 78, gen, R, net,
                        precision="fp32fast", scheme="magnus4", mode="global", trial_out=trial,
                        trial_fit_out=tfit, pred_out=pred, kept_out=kept)
    props = torch.cat([pp.de_propose(pop0, lo, hi, per, 0.8, 0.9, 78, gen * R + r)
                       for r in range(R)])
    y = net.forward(pp.mlp_features(props, lo, hi))
    assert pp.sync_status() == pp.PP_OK
    assert torch.equal(y, pred)
    yv = y.cpu().numpy()
    order = np.lexsort((np.arange(R * NP), -yv.astype(np.float64)))  # descending, ties to lower k
    k = kept.cpu().numpy()
    assert np.array_equal(k, order[:NP])
    assert np.array_equal(trial.cpu().numpy(), props.cpu().numpy()[k])
    A, _, _ = pp.synth_field(trial, SPEC)
    Nx, _ = pp.pair_number(A, SPEC["T"] / SPEC["n_steps"], GRID, precision="fp32fast",
                           scheme="magnus4")
    assert torch.equal(Nx, tfit)
    # selection: individual i takes its exactly best kept proposal when it is >= its fitness
    exp_pop, exp_fit = pop0.cpu().numpy().copy(), fit0.cpu().numpy().copy()
    tf, tr = tfit.cpu().numpy(), trial.cpu().numpy()
    for i in range(NP):
        rows = [r for r in range(NP) if k[r] % NP == i]
        if rows:
            r = max(rows, key=lambda q: (tf[q], -q))
            if tf[r] >= exp_fit[i]:
                exp_pop[i], exp_fit[i] = tr[r], tf[r]
    assert np.array_equal(pop.cpu().numpy(), exp_pop)
    assert np.array_equal(fit.cpu().numpy(), exp_fit)
    net.close()


def test_screened_step_rejects_bad_arguments(pp):
    lo, hi, per = bounds()
    pop, fit = start(pp, 8, 3)
    net = pp.Surrogate(32, 256, max_batch=16)
    with pytest.raises(pp.PPError):
        pp.de_screened_step(pop, fit, SPEC, GRID, lo, hi, per, 0.8, 0.9, 1, 0, 20, net)  # 160 rows
    with pytest.raises(pp.PPError):
        pp.de_screened_step(pop, fit, SPEC, GRID, lo, hi, per, 0.8, 0.9, 1, 0, 0, net)
    with pytest.raises(KeyError):
        pp.de_screened_step(pop, fit, SPEC, GRID, lo, hi, per, 0.8, 0.9, 1, 0, 2, net, mode="best")
    small = pp.Surrogate(16, 256, max_batch=64)
    with pytest.raises(pp.PPError):
        pp.de_screened_step(pop, fit, SPEC, GRID, lo, hi, per, 0.8, 0.9, 1, 0, 2, small)
    assert pp.sync_status() == pp.PP_OK
    net.close()
    small.close()


@pytest.mark.parametrize("mode", ["individual", "global"])
def test_trained_network_saves_exact_calls(pp, mode):
    """Train on 8192 exact evaluations of random pulses, then run plain and
    screened DE (8 proposals) from the same population with the same seed: the
    screened run reaches plain DE's best N with at most half the exact calls,
    in every one of three seeds."""
    from paper_1704_08919_gb300 import screening as scr
    lo, hi, per = bounds()
    P, N, _ = scr.score_random(pp, 8192, SPEC, GRID, 11)
    Pt, Nt, _ = scr.score_random(pp, 1024, SPEC, GRID, 12)
    lt = scr.LogTarget(N)
    net = pp.Surrogate(32, 256, max_batch=1024)
    net.init(1)
    net.fit(pp.mlp_features(P, lo, hi), lt.targets(pp, N), 256, 60, 2e-3, 5e-5)
    held = scr.held_out_error(pp, net, lt, Pt, Nt, lo, hi)
    assert held["spearman"] > 0.8, held
    gains = []
    for s in range(3):
        pop0, fit0 = start(pp, 32, 100 + s)
        plain = scr.run_de(pp, pop0, fit0, SPEC, GRID, 40, 500 + s, 0.8, 0.9)
        target = plain["best"][-1]
        screened = scr.run_de(pp, pop0, fit0, SPEC, GRID, 40, 500 + s, 0.8, 0.9, net=net, R=8,
                              lt=lt, mode=mode)
        c = scr.calls_to_reach(screened, target)
        gains.append(scr.calls_to_reach(plain, target) / c if c else 0.0)
    assert pp.sync_status() == pp.PP_OK
    assert min(gains) >= 2.0, (gains, held)
    net.close()


def test_online_refit_fires_lowers_the_loss_and_selection_stays_exact(pp):
    """The online refit of the large-scale configuration ("retrained every 20
    generations on newly scored pulses") at a small size: a network fitted on the
    initial population's 64 exact evaluations screens 10 generations (R = 8) and is
    refitted every 5 on every pulse scored so far.  The refit runs twice, each time
    on more rows, and lowers the network's loss on them; the network's parameters
    change; and the final fitness is the exact pair number of the final population,
    bit for bit, so selection never saw a prediction."""
    from paper_1704_08919_gb300 import screening as scr
    lo, hi, per = bounds()
    P0, N0, _ = scr.score_random(pp, 64, SPEC, GRID, 21)
    lt = scr.LogTarget(N0)
    net = pp.Surrogate(32, 256, max_batch=512)
    net.init(3)
    X0 = pp.mlp_features(P0, lo, hi)
    net.fit(X0, lt.targets(pp, N0), 32, 100, 2e-3, 5e-5)
    w0 = net.get_params().clone()
    pop0, fit0 = start(pp, 16, 7)
    r = scr.run_de(pp, pop0, fit0, SPEC, GRID, 10, 31, 0.8, 0.9, net=net, R=8, lt=lt,
                   online=(5, 8, 32, 2e-4), seen=(X0, N0))
    assert [x["generation"] for x in r["refits"]] == [4, 9]
    assert r["refits"][0]["rows"] == 64 + 5 * 16 and r["refits"][1]["rows"] == 64 + 10 * 16
    for x in r["refits"]:
        assert x["loss_after"] < x["loss_before"], r["refits"]
    assert not torch.equal(net.get_params(), w0)
    A, _, _ = pp.synth_field(r["pop"], SPEC)
    N, _ = pp.pair_number(A, SPEC["T"] / SPEC["n_steps"], GRID, precision="fp32fast", scheme="magnus4")
    assert pp.sync_status() == pp.PP_OK
    assert torch.equal(N, r["fit"])
    assert r["best"][-1] >= r["best"][0] and r["calls"][-1] == 16 * 11
    net.close()
