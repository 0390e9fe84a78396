"""pp_pair_number_static: the pair number without any device allocation.

Some callers cannot allocate device memory (their device memory is owned by
their own allocator, or allocation is forbidden once they are running); this
entry point keeps its scratch in a fixed array inside the library.  The test
calls it through the C ABI, twice in a row, and checks it against the
allocating entry point pp_pair_number on the same inputs, within the parity
tolerances used elsewhere (1e-9 relative for FP64, 1e-4 for FP32; both entry
points run the same kernels, so the results agree far more closely).  It also
checks that a request larger than the fixed array is refused with a clear
error.  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

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
    L = pp.lib()
    L.pp_pair_number_static.argtypes = L.pp_pair_number.argtypes
    L.pp_static_scratch_bytes.restype = ctypes.c_size_t
    return pp


def _static(pp, A, dt, grid, precision, scheme, n_steps=None, want_n=True):
    L = pp.lib()
    g = pp._grid(grid)
    ncand, _, ld = A.shape
    N = torch.full((ncand,), float("nan"), dtype=torch.float64, device=A.device)
    n = (torch.full((ncand, g.nz, g.ny, g.nx), float("nan"), dtype=torch.float64, device=A.device)
         if want_n else None)
    ns = None
    if n_steps is not None:
        arr = (ctypes.c_int32 * ncand)(*n_steps)
        ns = ctypes.cast(arr, ctypes.c_void_p)
    rc = L.pp_pair_number_static(pp._ptr(A), ncand, ld, ns, float(dt), ctypes.byref(g),
                                 pp.PRECISIONS[precision], pp.SCHEMES[scheme], pp._ptr(N),
                                 pp._ptr(n), pp._stream(None))
    return rc, N, n


@pytest.mark.parametrize("precision,scheme,tol", [("fp32", "magnus4", 1e-4), ("fp64", "rk4", 1e-9),
                                                  ("fp32", "rk4", 1e-4), ("fp64", "split2", 1e-9)])
def test_static_scratch_matches_allocating_entry_point(pp, precision, scheme, tol):
    cfg = inputs.DE_BATCH
    spec = dict(inputs.field_spec(cfg), n_steps=2048)
    params = inputs.random_population(4, cfg["K"], seed=17)
    A, _, _ = pp.synth_field(torch.tensor(params, device="cuda"), spec)
    grid = inputs.small_grid(24, 20, 9, ext=2.0)
    dt = spec["T"] / spec["n_steps"]
    N_ref, n_ref = pp.pair_number(A, dt, grid, precision=precision, scheme=scheme, want_n=True)
    for call in range(2):  # two calls in a row share the same static scratch
        rc, N, n = _static(pp, A, dt, grid, precision, scheme)
        assert rc == pp.PP_OK, pp.lib().pp_last_error()
        assert pp.sync_status() == pp.PP_OK
        assert torch.isfinite(N).all() and torch.isfinite(n).all()
        assert (N / N_ref - 1).abs().max().item() < tol
        big = n_ref > 1e-6 * n_ref.max()
        assert (n[big] / n_ref[big] - 1).abs().max().item() < 1e3 * tol


def test_static_scratch_uneven_steps(pp):
    dt = 0.04
    lens = [300, 777, 64]
    ld = 2 * max(lens) + 1
    A = torch.zeros((len(lens), 2, ld), dtype=torch.float64, device="cuda")
    t = torch.arange(ld, dtype=torch.float64, device="cuda") * dt / 2
    for c, ns in enumerate(lens):
        tc = t[:2 * ns + 1] - ns * dt / 2
        A[c, 0, :2 * ns + 1] = 0.3 * torch.exp(-tc ** 2 / 9.0) * torch.cos(0.9 * tc)
        A[c, 1, :2 * ns + 1] = 0.3 * torch.exp(-tc ** 2 / 9.0) * torch.sin(0.9 * tc)
    grid = inputs.small_grid(8, 6, 3, ext=1.2)
    N_ref, _ = pp.pair_number(A, dt, grid, precision="fp64", n_steps=lens)
    for call in range(2):
        rc, N, _ = _static(pp, A, dt, grid, "fp64", "rk4", n_steps=lens, want_n=False)
        assert rc == pp.PP_OK, pp.lib().pp_last_error()
        assert pp.sync_status() == pp.PP_OK
        assert (N / N_ref - 1).abs().max().item() < 1e-9


def test_static_scratch_refuses_oversized_requests(pp):
    L = pp.lib()
    cap = L.pp_static_scratch_bytes()
    assert cap == 16 << 20
    # 64 candidates x 8192 Magnus steps x 32 B of table alone exceed 16 MiB
    A = torch.zeros((64, 2, 2 * 8192 + 1), dtype=torch.float64, device="cuda")
    rc, N, _ = _static(pp, A, 200.0 / 8192, inputs.small_grid(4, 4, 2), "fp32", "magnus4",
                       want_n=False)
    assert rc == pp.PP_ERR_INVALID_ARG
    msg = L.pp_last_error().decode()
    assert "static scratch" in msg and str(cap) in msg
    assert torch.isnan(N).all()  # nothing was launched
