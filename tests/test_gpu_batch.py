"""Uneven batches (pp_batch_*): slots with their own pulse length, step count and
momentum grid scored in one persistent launch, and DE loops captured in CUDA
graphs -- against the FP64 CPU oracle, slot by slot, and against the uniform
entry points (bitwise: the batch runs the same per-mode arithmetic)."""
import math

import numpy as np
import pytest

import oracle
from paper_1704_08919_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"

DT = 0.05
STEPS = [400, 500, 650, 820, 500]
K, ORDER = 6, 4


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


def specs():
    return [dict(K=K, order=ORDER, w_min=0.0, w_max=2.0, T=n * DT, fluence=2.0, n_steps=n)
            for n in STEPS]


def grids():
    return [inputs.small_grid(6, 5, 3, ext=1.5), inputs.small_grid(8, 7, 2, ext=2.0),
            inputs.small_grid(5, 5, 5, ext=1.2), dict(nx=9, ny=4, nz=3, x0=-1.0, x1=1.5, y0=-2.0,
                                                       y1=0.5, z0=-0.5, z1=0.7, mirror_z=0),
            inputs.small_grid(16, 16, 2, ext=1.8)]


def oracle_fields(params):
    out = []
    for c, sp in enumerate(specs()):
        A, _, _, rc = oracle.synth_field(params[c:c + 1], K, ORDER, 0.0, 2.0, sp["T"], 2.0,
                                         sp["n_steps"], want_E=False)
        assert rc == 0
        out.append(A[0])
    return out


def test_batch_synthesis_matches_oracle(pp):
    params = inputs.random_population(len(STEPS), K, seed=41)
    b = pp.Batch(specs(), grids(), DT, precision="fp64", scheme="rk4")
    A = b.synth(torch.tensor(params, device=DEV)).cpu().numpy()
    assert pp.sync_status() == pp.PP_OK
    for c, Ao in enumerate(oracle_fields(params)):
        n = Ao.shape[-1]
        assert np.abs(A[c, :, :n] - Ao).max() < 1e-12 * np.abs(Ao).max()
    b.close()


@pytest.mark.parametrize("precision,scheme", [("fp64", "rk4"), ("fp64", "magnus4"),
                                              ("fp32", "magnus4"), ("fp32fast", "magnus4"),
                                              ("fp32", "rk4"), ("fp32fast", "split2")])
def test_batch_pair_number_matches_oracle_and_uniform_path(pp, precision, scheme):
    params = inputs.random_population(len(STEPS), K, seed=43)
    b = pp.Batch(specs(), grids(), DT, precision=precision, scheme=scheme)
    A = b.synth(torch.tensor(params, device=DEV))
    N, n = b.pair_number(A, want_n=True)
    assert pp.sync_status() == pp.PP_OK
    off = 0
    for c, (ns, g) in enumerate(zip(STEPS, grids())):
        nm = g["nx"] * g["ny"] * g["nz"]
        Nu, nu = pp.pair_number(A[c:c + 1, :, :2 * ns + 1].contiguous(), DT, g, precision=precision,
                                scheme=scheme, want_n=True)
        assert torch.equal(N[c:c + 1], Nu)
        assert torch.equal(n[off:off + nm], nu.reshape(-1))
        if precision == "fp64":
            Ao = A[c, :, :2 * ns + 1].cpu().numpy()
            pts = inputs.grid_points(g)
            fo = (oracle.dirac_modes(Ao, ns, DT, pts) if scheme == "rk4"
                  else oracle.dirac_magnus_modes(Ao, ns, DT, pts)[0])
            x, y, z = inputs.grid_axes(g)

            def tw(a, mirror):
                w = np.full(a.size, a[1] - a[0])
                w[[0, -1]] /= 2
                return w * (2 if mirror else 1)
            W = (tw(z, g["mirror_z"])[:, None, None] * tw(y, 0)[None, :, None] * tw(x, 0)[None, None, :])
            assert abs(N[c].item() / float(np.sum(W.ravel() * fo)) - 1) < 1e-9
        off += nm
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32fast"])
def test_batch_magnus_beyond_the_series_range(pp, precision):
    # a step large enough that th = |dt h_eff| exceeds the Magnus polynomials' range
    # (0.2) on every slot: the batch builds each slot's step bound from its own grid,
    # takes the argument-halved step and still equals the uniform path bit for bit
    # (and the oracle twin in FP64)
    dt, steps = 0.3, [100, 140, 90, 120]
    sp = [dict(K=K, order=ORDER, w_min=0.0, w_max=2.0, T=n * dt, fluence=2.0, n_steps=n) for n in steps]
    gr = [inputs.small_grid(6, 5, 3, ext=1.5), inputs.small_grid(4, 4, 2, ext=2.0),
          inputs.small_grid(5, 3, 2, ext=1.0), inputs.small_grid(3, 4, 2, ext=1.7)]
    params = inputs.random_population(len(steps), K, seed=53)
    b = pp.Batch(sp, gr, dt, precision=precision, scheme="magnus4")
    A = b.synth(torch.tensor(params, device=DEV))
    N, _ = b.pair_number(A)
    assert pp.sync_status() == pp.PP_OK
    for c, (ns, g) in enumerate(zip(steps, gr)):
        Nu, _ = pp.pair_number(A[c:c + 1, :, :2 * ns + 1].contiguous(), dt, g, precision=precision,
                               scheme="magnus4")
        assert torch.equal(N[c:c + 1], Nu)
        if precision == "fp64":
            Ao = A[c, :, :2 * ns + 1].cpu().numpy()
            fo = oracle.dirac_magnus_modes(Ao, ns, dt, inputs.grid_points(g))[0]
            x, y, z = inputs.grid_axes(g)

            def tw(a, mirror):
                w = np.full(a.size, a[1] - a[0])
                w[[0, -1]] /= 2
                return w * (2 if mirror else 1)
            W = (tw(z, g["mirror_z"])[:, None, None] * tw(y, 0)[None, :, None] * tw(x, 0)[None, None, :])
            assert abs(N[c].item() / float(np.sum(W.ravel() * fo)) - 1) < 1e-9
    b.close()


def test_batch_tuner_keeps_results_bitwise(pp):
    params = inputs.random_population(len(STEPS), K, seed=47)
    b = pp.Batch(specs(), grids(), DT, precision="fp32fast", scheme="magnus4")
    A = b.synth(torch.tensor(params, device=DEV))
    N0, _ = b.pair_number(A)
    chosen, ms = b.tune(A)
    N1, _ = b.pair_number(A)
    assert pp.sync_status() == pp.PP_OK
    assert 0 <= chosen < 6 and b.config() == chosen and all(t > 0 for t in ms)
    assert torch.equal(N0, N1)
    b.close()


def _de_setup(pp, seed=5):
    lo, hi, per = inputs.param_bounds(K)
    pop = torch.tensor(inputs.random_population(len(STEPS), K, seed=seed), device=DEV)
    return (pop, torch.tensor(lo, device=DEV), torch.tensor(hi, device=DEV),
            torch.tensor(per, device=DEV))


def test_batch_graph_loop_equals_single_steps(pp):
    pop0, lo, hi, per = _de_setup(pp)
    b = pp.Batch(specs(), grids(), DT, precision="fp32fast", scheme="magnus4")
    fit0, _ = b.pair_number(b.synth(pop0))
    popA, fitA = pop0.clone(), fit0.clone()
    popB, fitB = pop0.clone(), fit0.clone()
    b.set_generation(3)
    for _ in range(5):
        b.de_step(popA, fitA, lo, hi, per, 0.8, 0.9, 77)
    b.set_generation(3)
    b.de_run(popB, fitB, lo, hi, per, 0.8, 0.9, 77, 3)  # generations 3, 4, 5
    b.de_run(popB, fitB, lo, hi, per, 0.8, 0.9, 77, 2)  # recaptured: 6, 7
    assert pp.sync_status() == pp.PP_OK
    assert torch.equal(popA, popB) and torch.equal(fitA, fitB)
    assert not torch.equal(popA, pop0)  # something was accepted
    # relaunching the same captured graph continues the generations
    b.set_generation(3)
    popC, fitC = pop0.clone(), fit0.clone()
    b.de_run(popC, fitC, lo, hi, per, 0.8, 0.9, 77, 1)
    b.de_run(popC, fitC, lo, hi, per, 0.8, 0.9, 77, 1)
    popD, fitD = pop0.clone(), fit0.clone()
    b.set_generation(3)
    b.de_step(popD, fitD, lo, hi, per, 0.8, 0.9, 77)
    b.de_step(popD, fitD, lo, hi, per, 0.8, 0.9, 77)
    assert torch.equal(popC, popD) and torch.equal(fitC, fitD)
    b.close()


def test_batch_de_step_matches_oracle_sequence(pp):
    pop0, lo, hi, per = _de_setup(pp, seed=9)
    b = pp.Batch(specs(), grids(), DT, precision="fp64", scheme="rk4")
    fit0, _ = b.pair_number(b.synth(pop0))
    pop, fit = pop0.clone(), fit0.clone()
    b.set_generation(11)
    b.de_step(pop, fit, lo, hi, per, 0.8, 0.9, 1234)
    assert pp.sync_status() == pp.PP_OK
    lo_h, hi_h, per_h = (x.cpu().numpy() for x in (lo, hi, per))
    tr = oracle.de_propose(pop0.cpu().numpy(), lo_h, hi_h, per_h, 0.8, 0.9, 1234, 11)
    tfit = []
    for c, (ns, g) in enumerate(zip(STEPS, grids())):
        A, _, _, _ = oracle.synth_field(tr[c:c + 1], K, ORDER, 0.0, 2.0, ns * DT, 2.0, ns,
                                        want_E=False)
        N, _ = oracle.pair_number(A, ns, DT, g, want_n=False)
        tfit.append(N[0])
    tfit = np.array(tfit)
    po, fo = oracle.de_select(pop0.cpu().numpy(), fit0.cpu().numpy(), tr, tfit)
    accepted = tfit >= fit0.cpu().numpy()
    # same decisions (no ties near 1e-9 here), same vectors, fitness within 1e-9
    assert np.array_equal(pop.cpu().numpy(), po)
    assert np.abs(fit.cpu().numpy() / fo - 1).max() < 1e-9
    b.close()


def test_batch_rejects_inconsistent_specs(pp):
    sp = specs()
    sp[2] = dict(sp[2], K=7)
    with pytest.raises(pp.PPError):
        pp.Batch(sp, grids(), DT)
    sp = specs()
    sp[1] = dict(sp[1], T=sp[1]["T"] * 1.01)
    with pytest.raises(pp.PPError) as e:
        pp.Batch(sp, grids(), DT)
    assert e.value.code == pp.PP_ERR_INVALID_ARG
    with pytest.raises(pp.PPError):
        pp.Batch(specs()[:3], grids()[:3], DT)
    sp = specs()
    sp[3] = dict(sp[3], envelope=1)  # envelopes must match across slots
    with pytest.raises(pp.PPError) as e:
        pp.Batch(sp, grids(), DT)
    assert e.value.code == pp.PP_ERR_INVALID_ARG


def test_batch_with_the_hann_envelope(pp):
    """Slots of different length with the Hann envelope of Eq. (hann): the batch
    synthesis equals the oracle's closed form, and the batch pair numbers equal the
    uniform path's bit for bit and the oracle's to 1e-9."""
    params = inputs.random_population(len(STEPS), K, seed=45)
    sp = [dict(x, envelope=1) for x in specs()]
    b = pp.Batch(sp, grids(), DT, precision="fp64", scheme="rk4")
    A = b.synth(torch.tensor(params, device=DEV))
    N, _ = b.pair_number(A)
    assert pp.sync_status() == pp.PP_OK
    An = A.cpu().numpy()
    for c, (s, g) in enumerate(zip(sp, grids())):
        ns = s["n_steps"]
        Ao, _, _, _ = oracle.synth_hann(params[c:c + 1], K, ORDER, 0.0, 2.0, s["T"], 2.0, ns)
        assert np.abs(An[c, :, :2 * ns + 1] - Ao[0]).max() < 1e-12 * np.abs(Ao).max()
        Nu, _ = pp.pair_number(A[c:c + 1, :, :2 * ns + 1].contiguous(), DT, g, precision="fp64",
                               scheme="rk4")
        assert torch.equal(N[c:c + 1], Nu)
        if c < 2:
            No, _ = oracle.pair_number(Ao, ns, DT, g)
            assert abs(N[c].item() / No[0] - 1) < 1e-9
    b.close()


@pytest.mark.parametrize("precision,scheme", [("fp64", "rk4"), ("fp32fast", "magnus4"), ("fp32", "rk4")])
def test_pair_number_with_a_grid_per_candidate(pp, precision, scheme):
    # pp_pair_number_grids: candidate c on grids[c] equals pp_pair_number of c alone on that grid,
    # bit for bit (N and n(p), the n(p) arrays concatenated), with uneven step counts; one
    # shared grid is pp_pair_number itself
    params = inputs.random_population(len(STEPS), K, seed=61)
    b = pp.Batch(specs(), grids(), DT, precision="fp64", scheme="rk4")
    A = b.synth(torch.tensor(params, device=DEV))
    N, n = pp.pair_number_grids(A, DT, grids(), precision=precision, scheme=scheme, n_steps=STEPS, want_n=True)
    assert pp.sync_status() == pp.PP_OK
    off = 0
    for c, (ns, g) in enumerate(zip(STEPS, grids())):
        Nu, nu = pp.pair_number(A[c:c + 1, :, :2 * ns + 1].contiguous(), DT, g, precision=precision, scheme=scheme,
                                want_n=True)
        nm = g["nx"] * g["ny"] * g["nz"]
        assert torch.equal(N[c:c + 1], Nu)
        assert torch.equal(n[off:off + nm], nu.reshape(-1))
        off += nm
    Ns, _ = pp.pair_number_grids(A, DT, [grids()[0]], precision=precision, scheme=scheme, n_steps=STEPS)
    Nu, _ = pp.pair_number(A, DT, grids()[0], precision=precision, scheme=scheme, n_steps=STEPS)
    assert torch.equal(Ns, Nu)
    b.close()
