"""Host logic of the screened-DE driver (no GPU): the target standardisation and
the exact-call bookkeeping that the gain is computed from."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1704_08919_gb300 import screening as scr  # noqa: E402


def test_log_target_standardises_log10_N():
    N = torch.tensor([1e-6, 1e-4, 1e-2, 0.0], dtype=torch.float64)
    lt = scr.LogTarget(N)
    y = np.log10(np.maximum(N.numpy(), lt.FLOOR))
    assert abs(lt.shift - y.mean()) < 1e-12 and abs(lt.scale - y.std()) < 1e-12
    z = (y - lt.shift) / lt.scale
    assert np.allclose(lt.to_log10(z), y)


def test_log_target_of_constant_data_keeps_unit_scale():
    lt = scr.LogTarget(torch.full((5,), 0.3, dtype=torch.float64))
    assert lt.scale == 1.0


def test_calls_to_reach():
    run = {"best": [0.1, 0.2, 0.2, 0.5, 0.7], "calls": [8, 16, 24, 32, 40]}
    assert scr.calls_to_reach(run, 0.1) == 8
    assert scr.calls_to_reach(run, 0.45) == 32
    assert scr.calls_to_reach(run, 0.7) == 40
    assert scr.calls_to_reach(run, 0.71) is None
