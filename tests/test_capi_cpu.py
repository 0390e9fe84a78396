"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point that include/pp.h declares, and rejects bad arguments on the
host before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pp():
    from paper_1704_08919_gb300 import build
    build.build()
    import paper_1704_08919_gb300 as pp
    pp.lib()
    return pp


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "pp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pp_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_entry_points():
    names = declared_symbols()
    for n in ("pp_synth_field", "pp_pair_number", "pp_de_propose", "pp_de_select", "pp_de_step",
              "pp_sync_status", "pp_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(pp):
    L = pp.lib()
    for name in declared_symbols():
        assert hasattr(L, name), name
    assert set(pp.EXPORTS) <= set(declared_symbols())
    assert L.pp_version() >= 100


def test_host_validation_rejects_bad_arguments(pp):
    L = pp.lib()
    g = pp.Grid(0, 4, 4, -1, 1, -1, 1, 0, 1, 1)
    rc = L.pp_pair_number(ctypes.c_void_p(8), 1, 101, None, 0.1, ctypes.byref(g), 0, 0,
                          ctypes.c_void_p(8), None, None)
    assert rc == pp.PP_ERR_INVALID_ARG
    assert b"grid sizes" in L.pp_last_error()
    g = pp.Grid(4, 4, 4, -1, 1, -1, 1, 0.5, 1, 1)
    rc = L.pp_pair_number(ctypes.c_void_p(8), 1, 101, None, 0.1, ctypes.byref(g), 0, 0,
                          ctypes.c_void_p(8), None, None)
    assert rc == pp.PP_ERR_INVALID_ARG and b"mirror_z" in L.pp_last_error()
    g = pp.Grid(4, 4, 4, -1, 1, -1, 1, 0, 1, 1)
    rc = L.pp_pair_number(ctypes.c_void_p(8), 1, 101, None, -0.1, ctypes.byref(g), 0, 0,
                          ctypes.c_void_p(8), None, None)
    assert rc == pp.PP_ERR_INVALID_ARG and b"dt" in L.pp_last_error()
    rc = L.pp_pair_number(ctypes.c_void_p(8), 1, 101, None, 0.1, ctypes.byref(g), 7, 0,
                          ctypes.c_void_p(8), None, None)
    assert rc == pp.PP_ERR_INVALID_ARG and b"precision" in L.pp_last_error()
    rc = L.pp_pair_number(ctypes.c_void_p(8), 1, 101, None, 0.1, ctypes.byref(g), 0, 9,
                          ctypes.c_void_p(8), None, None)
    assert rc == pp.PP_ERR_INVALID_ARG and b"scheme" in L.pp_last_error()
    ns = (ctypes.c_int32 * 1)(60)
    rc = L.pp_pair_number(ctypes.c_void_p(8), 1, 101, ctypes.cast(ns, ctypes.c_void_p), 0.1,
                          ctypes.byref(g), 0, 0, ctypes.c_void_p(8), None, None)
    assert rc == pp.PP_ERR_INVALID_ARG and b"n_steps" in L.pp_last_error()
    rc = L.pp_de_propose(ctypes.c_void_p(8), 3, 4, ctypes.c_void_p(8), ctypes.c_void_p(8), None,
                         0.5, 0.9, 1, 0, ctypes.c_void_p(8), None)
    assert rc == pp.PP_ERR_INVALID_ARG and b"NP" in L.pp_last_error()
    rc = L.pp_de_propose(ctypes.c_void_p(8), 8, 4, ctypes.c_void_p(8), ctypes.c_void_p(8), None,
                         0.5, 1.5, 1, 0, ctypes.c_void_p(8), None)
    assert rc == pp.PP_ERR_INVALID_ARG and b"CR" in L.pp_last_error()
    spec = pp.FieldSpec(8, 9, 0.0, 2.0, 200.0, 2.0, 100, 0)
    rc = L.pp_synth_field(ctypes.c_void_p(8), 1, ctypes.byref(spec), ctypes.c_void_p(8), 201, None,
                          None, None)
    assert rc == pp.PP_ERR_INVALID_ARG and b"order" in L.pp_last_error()
    spec = pp.FieldSpec(8, 4, 0.0, 0.01, 200.0, 2.0, 100, 0)
    rc = L.pp_synth_field(ctypes.c_void_p(8), 1, ctypes.byref(spec), ctypes.c_void_p(8), 201, None,
                          None, None)
    assert rc == pp.PP_ERR_INVALID_ARG and b"no mode" in L.pp_last_error()
    spec = pp.FieldSpec(8, 4, 0.0, 2.0, 200.0, 2.0, 100, 0)
    rc = L.pp_synth_field(ctypes.c_void_p(8), 1, ctypes.byref(spec), ctypes.c_void_p(8), 200, None,
                          None, None)
    assert rc == pp.PP_ERR_INVALID_ARG and b"ld" in L.pp_last_error()
    spec = pp.FieldSpec(8, 4, 0.0, 2.0, 200.0, 2.0, 100, 2)
    rc = L.pp_synth_field(ctypes.c_void_p(8), 1, ctypes.byref(spec), ctypes.c_void_p(8), 201, None,
                          None, None)
    assert rc == pp.PP_ERR_NOT_IMPLEMENTED


def test_host_validation_of_the_extension_entry_points(pp):
    """Screening, surrogate, QKE and local-search entry points reject bad arguments
    on the host, before any device work."""
    L = pp.lib()
    P = ctypes.c_void_p(8)
    spec = pp.FieldSpec(8, 4, 0.0, 2.0, 50.0, 1.0, 100, 0)
    grid = pp.Grid(4, 4, 2, -1, 1, -1, 1, 0, 1, 1)
    rc = L.pp_qke_pair_number(P, P, P, 1, 201, 100, 0.0, ctypes.byref(grid), 0, P, None, None)
    assert rc == pp.PP_ERR_INVALID_ARG and b"dt" in L.pp_last_error()
    rc = L.pp_qke_pair_number(P, P, P, 1, 200, 100, 0.5, ctypes.byref(grid), 0, P, None, None)
    assert rc == pp.PP_ERR_INVALID_ARG and b"ld" in L.pp_last_error()
    rc = L.pp_qke_pair_number(P, P, P, 1, 201, 100, 0.5, ctypes.byref(grid), 5, P, None, None)
    assert rc == pp.PP_ERR_INVALID_ARG and b"precision" in L.pp_last_error()
    rc = L.pp_qke_sample_gradient(P, P, P, 1, 201, 100, 0.5, ctypes.byref(grid), 0, P, P, 150, None)
    assert rc == pp.PP_ERR_INVALID_ARG and b"ldg" in L.pp_last_error()
    bad = pp.FieldSpec(8, 0, 0.0, 2.0, 50.0, 1.0, 100, 0)
    rc = L.pp_qke_gradient(P, 1, ctypes.byref(bad), ctypes.byref(grid), 0, P, P, None, None, None)
    assert rc == pp.PP_ERR_INVALID_ARG and b"order" in L.pp_last_error()
    rc = L.pp_synth_field_raw(P, 1, ctypes.byref(spec), P, None, None, 150, None, None)
    assert rc == pp.PP_ERR_INVALID_ARG and b"ld" in L.pp_last_error()
    opt = pp.ALOptions(1.0, 0.5, 3, 10, 1e-6, 1e-6)
    x = (ctypes.c_double * 32)()
    rc = L.pp_local_search(x, 1, ctypes.byref(spec), ctypes.byref(grid), 0, -2.0, ctypes.byref(opt),
                           None, None, None, None, None, None, None)
    assert rc == pp.PP_ERR_INVALID_ARG and b"U_const" in L.pp_last_error()
    rc = L.pp_de_screened_step(P, P, 16, ctypes.byref(spec), ctypes.byref(grid), 0, 1, P, P, None,
                               0.8, 0.9, 1, 0, 8, 0, None, None, None, None, None, None)
    assert rc == pp.PP_ERR_INVALID_ARG and b"mlp" in L.pp_last_error()
    rc = L.pp_mlp_fit(None, P, P, 10, 4, 1, 1e-3, 1e-4, 0, None, None)
    assert rc == pp.PP_ERR_INVALID_ARG
    rc = L.pp_mlp_log_targets(P, 4, 0.0, 0.0, 1.0, P, None)
    assert rc == pp.PP_ERR_INVALID_ARG and b"floor" in L.pp_last_error()
    rc = L.pp_gemm_bf16(P, P, P, 100, 64, 64, 64, None)
    assert rc == pp.PP_ERR_INVALID_ARG


def test_per_candidate_grids_are_checked_on_the_host(pp):
    L = pp.lib()
    good = pp.Grid(4, 4, 4, -1, 1, -1, 1, 0, 1, 1)
    bad = pp.Grid(4, 4, 4, -1, 1, -1, 1, 0.5, 1, 1)  # mirror_z needs z0 = 0
    arr = (pp.Grid * 3)(good, good, good)
    P = ctypes.c_void_p(8)
    rc = L.pp_pair_number_grids(P, 2, 101, None, 0.1, ctypes.cast(arr, ctypes.c_void_p), 3, 0, 0, P, None, None)
    assert rc == pp.PP_ERR_INVALID_ARG and b"n_grids" in L.pp_last_error()
    arr = (pp.Grid * 3)(good, bad, good)
    rc = L.pp_pair_number_grids(P, 3, 101, None, 0.1, ctypes.cast(arr, ctypes.c_void_p), 3, 0, 0, P, None, None)
    assert rc == pp.PP_ERR_INVALID_ARG and b"candidate 1" in L.pp_last_error()
    assert b"mirror_z" in L.pp_last_error()
    arr = (pp.Grid * 2)(good, good)
    ns = (ctypes.c_int32 * 2)(50, 60)  # 2 * 60 + 1 > ld
    rc = L.pp_pair_number_grids(P, 2, 101, ctypes.cast(ns, ctypes.c_void_p), 0.1, ctypes.cast(arr, ctypes.c_void_p),
                                2, 0, 0, P, None, None)
    assert rc == pp.PP_ERR_INVALID_ARG and b"candidate 1" in L.pp_last_error()
    rc = L.pp_pair_number_grids(P, 2, 101, None, 0.1, None, 2, 0, 0, P, None, None)
    assert rc == pp.PP_ERR_INVALID_ARG
    assert L.pp_pair_number_grids(None, 0, 101, None, 0.1, None, 0, 0, 0, None, None, None) == pp.PP_OK


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1704_08919_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, re.M), f
                assert "pp_oracle" not in txt and "liboracle" not in txt, f


def test_envelope_limits_are_checked_on_the_host(pp):
    """The Hann envelope widens the band by one harmonic on each side, so its mode
    limit is 1534 instead of 1536; uneven batches need one envelope for all slots.
    Every call here is refused before any device work."""
    import math
    L = pp.lib()
    T = 1535.5 * math.pi  # w_max = 2: modes j = 1 .. 1535
    hann = pp.FieldSpec(8, 4, 0.0, 2.0, T, 2.0, 100, 1)
    rc = L.pp_synth_field(ctypes.c_void_p(8), 1, ctypes.byref(hann), ctypes.c_void_p(8), 201, None, None, None)
    assert rc == pp.PP_ERR_INVALID_ARG and b"1534" in L.pp_last_error()
    specs = [pp.FieldSpec(8, 4, 0.0, 2.0, 50.0 + c, 2.0, 1000 + 20 * c, 1 if c == 2 else 0) for c in range(4)]
    grids = [pp._grid(dict(nx=2, ny=2, nz=1, x0=-1.0, x1=1.0, y0=-1.0, y1=1.0, z0=0.0, z1=0.0))] * 4
    S, G = (pp.FieldSpec * 4)(*specs), (pp.Grid * 4)(*grids)
    h = ctypes.c_void_p()
    rc = L.pp_batch_create(4, S, G, 0, 0, 0.05, ctypes.byref(h))
    assert rc == pp.PP_ERR_INVALID_ARG and b"envelope" in L.pp_last_error() and not h.value
    for c in range(4):
        S[c].envelope = 2
    rc = L.pp_batch_create(4, S, G, 0, 0, 0.05, ctypes.byref(h))
    assert rc == pp.PP_ERR_NOT_IMPLEMENTED and not h.value


def test_surrogate_sizes_are_checked_on_the_host(pp):
    """The hidden width is a whole number of 128-row GEMM tiles; other widths are
    refused before anything is allocated."""
    L = pp.lib()
    h = ctypes.c_void_p()
    for hidden in (16, 64, 144, 192, 512):
        rc = L.pp_mlp_create(32, hidden, 256, ctypes.byref(h))
        assert rc == pp.PP_ERR_INVALID_ARG and not h.value, hidden
    assert L.pp_mlp_create(0, 256, 256, ctypes.byref(h)) == pp.PP_ERR_INVALID_ARG
    assert L.pp_mlp_create(300, 256, 256, ctypes.byref(h)) == pp.PP_ERR_INVALID_ARG


def test_qke_state_budget_is_a_host_setting(pp):
    """pp_set_qke_state_budget returns the previous setting; a negative value selects
    the default (half the device's memory), reported as -1.  No device work."""
    old = pp.set_qke_state_budget(12345)
    try:
        assert pp.set_qke_state_budget(0) == 12345
        assert pp.set_qke_state_budget(-7) == 0
        assert pp.set_qke_state_budget(-1) == -1
    finally:
        pp.set_qke_state_budget(old)


def test_fma_rate_arguments_are_checked_on_the_host(pp):
    """Refused before any device work: an unknown precision and a NULL output."""
    L = pp.lib()
    out = ctypes.c_double(0.0)
    assert L.pp_fma_rate(7, ctypes.byref(out), None) == pp.PP_ERR_INVALID_ARG
    assert b"precision" in L.pp_last_error()
    assert L.pp_fma_rate(pp.PP_FP32, None, None) == pp.PP_ERR_INVALID_ARG
