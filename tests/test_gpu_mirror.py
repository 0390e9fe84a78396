"""The CUDA library against the oracle's host mirror, call for call: the same
ctypes argument objects (pulse model, grid, sizes, DE constants) go to
pp_synth_field / pp_pair_number / pp_de_propose / pp_de_step with device arrays
and to pp_oracle_* with host arrays, and the results are compared within the
tolerances of the parity tests (FP64: 1e-9 on N, 1e-12 of max |A| on the field,
DE trials bit for bit)."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1704_08919_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

K = 6
SPEC = dict(K=K, order=4, w_min=0.0, w_max=2.0, T=40.0, fluence=2.0, n_steps=500)
GRID = dict(nx=7, ny=6, nz=3, x0=-1.2, x1=1.2, y0=-1.0, y1=1.1, z0=0.0, z1=1.0, mirror_z=1)


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


def hptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def dptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("envelope", [0, 1])
def test_synthesis_and_pair_number_through_both_libraries(pp, envelope):
    L, O = pp.lib(), oracle.lib()
    spec, grid = pp._spec(dict(SPEC, envelope=envelope)), pp._grid(GRID)
    nc, n = 3, SPEC["n_steps"]
    ld = 2 * n + 1
    X = inputs.random_population(nc, K, seed=11 + envelope)
    Ah = np.zeros((nc, 2, ld))
    assert O.pp_oracle_synth_field(hptr(X), nc, ctypes.byref(spec), hptr(Ah), ld, None, None, None) == 0
    Xd = torch.tensor(X, device="cuda")
    Ad = torch.empty((nc, 2, ld), dtype=torch.float64, device="cuda")
    assert L.pp_synth_field(dptr(Xd), nc, ctypes.byref(spec), dptr(Ad), ld, None, None, None) == pp.PP_OK
    assert pp.sync_status() == pp.PP_OK
    assert np.abs(Ad.cpu().numpy() - Ah).max() < 1e-12 * np.abs(Ah).max()
    dt = SPEC["T"] / n
    nm = GRID["nx"] * GRID["ny"] * GRID["nz"]
    Nh, nh = np.zeros(nc), np.zeros((nc, nm))
    assert O.pp_oracle_pair_number(hptr(Ah), nc, ld, None, dt, ctypes.byref(grid), 0, 0, hptr(Nh), hptr(nh),
                                   None) == 0
    Nd = torch.empty(nc, dtype=torch.float64, device="cuda")
    nd = torch.empty((nc, nm), dtype=torch.float64, device="cuda")
    Ahd = torch.tensor(Ah, device="cuda")  # the same potential on both sides
    assert L.pp_pair_number(dptr(Ahd), nc, ld, None, dt, ctypes.byref(grid), 0, 0, dptr(Nd), dptr(nd),
                            None) == pp.PP_OK
    assert pp.sync_status() == pp.PP_OK
    assert np.abs(Nd.cpu().numpy() / Nh - 1).max() < 1e-9
    big = nh >= 1e-6 * nh.max()
    nn = nd.cpu().numpy()
    assert np.all(np.abs(nn[big] / nh[big] - 1) < 1e-9)
    assert np.all(np.abs(nn[~big] - nh[~big]) < 1e-9 * nh.max())


def test_de_generation_through_both_libraries(pp):
    L, O = pp.lib(), oracle.lib()
    spec, grid = pp._spec(SPEC), pp._grid(GRID)
    NP, D = 8, 4 * K
    lo, hi, per = inputs.param_bounds(K)
    per = per.astype(np.uint8)
    pop = inputs.random_population(NP, K, seed=21)
    ld = 2 * SPEC["n_steps"] + 1
    A = np.zeros((NP, 2, ld))
    O.pp_oracle_synth_field(hptr(pop), NP, ctypes.byref(spec), hptr(A), ld, None, None, None)
    fit = np.zeros(NP)
    O.pp_oracle_pair_number(hptr(A), NP, ld, None, SPEC["T"] / SPEC["n_steps"], ctypes.byref(grid), 0, 0,
                            hptr(fit), None, None)
    # host side
    ph, fh = pop.copy(), fit.copy()
    th, tfh = np.zeros_like(pop), np.zeros(NP)
    args = (0.8, 0.9, 77, 4)
    assert O.pp_oracle_de_step(hptr(ph), hptr(fh), NP, ctypes.byref(spec), ctypes.byref(grid), 0, 0, hptr(lo),
                               hptr(hi), hptr(per), *args, hptr(th), hptr(tfh), None) == 0
    # device side, same arguments
    dev = {k: torch.tensor(v, device="cuda") for k, v in dict(pop=pop, fit=fit, lo=lo, hi=hi, per=per).items()}
    td = torch.empty((NP, D), dtype=torch.float64, device="cuda")
    tfd = torch.empty(NP, dtype=torch.float64, device="cuda")
    assert L.pp_de_step(dptr(dev["pop"]), dptr(dev["fit"]), NP, ctypes.byref(spec), ctypes.byref(grid), 0, 0,
                        dptr(dev["lo"]), dptr(dev["hi"]), dptr(dev["per"]), *args, dptr(td), dptr(tfd),
                        None) == pp.PP_OK
    assert pp.sync_status() == pp.PP_OK
    assert np.array_equal(td.cpu().numpy(), th)
    assert np.abs(tfd.cpu().numpy() / tfh - 1).max() < 1e-9
    # the selection decisions agree wherever the trial and parent are not within rounding of a tie
    clear = np.abs(tfh / fit - 1) > 1e-8
    assert np.array_equal(dev["pop"].cpu().numpy()[clear], ph[clear])
    # and pp_de_propose alone gives the mirror's proposals
    tp = torch.empty((NP, D), dtype=torch.float64, device="cuda")
    pop0 = torch.tensor(pop, device="cuda")
    assert L.pp_de_propose(dptr(pop0), NP, D, dptr(dev["lo"]), dptr(dev["hi"]),
                           dptr(dev["per"]), 0.8, 0.9, 77, 4, dptr(tp), None) == pp.PP_OK
    th2 = np.zeros_like(pop)
    assert O.pp_oracle_de_propose(hptr(pop), NP, D, hptr(lo), hptr(hi), hptr(per), 0.8, 0.9, 77, 4, hptr(th2),
                                  None) == 0
    assert pp.sync_status() == pp.PP_OK
    assert np.array_equal(tp.cpu().numpy(), th2) and np.array_equal(th2, th)
