"""The seeded input module (paper_1704_08919_gb300.inputs) on its own: draws stay
inside the parameter bounds, and the rotating-Gaussian potential that the bench
feeds to the GPU equals the oracle's independently integrated one."""
import numpy as np

import oracle
from paper_1704_08919_gb300 import inputs


def test_random_population_inside_bounds_and_seeded():
    lo, hi, per = inputs.param_bounds(8)
    P = inputs.random_population(50, 8, seed=9)
    assert P.shape == (50, 32)
    assert np.all(P >= lo) and np.all(P <= hi)
    assert np.array_equal(P, inputs.random_population(50, 8, seed=9))
    assert not np.array_equal(P, inputs.random_population(50, 8, seed=10))
    assert per.sum() == 16 and np.all(hi[per == 1] == 2 * np.pi)


def test_rotating_gaussian_potential_equals_the_oracles():
    # the closed form (complex erf) against the oracle's Gauss-Legendre integration
    g = inputs.ROTATING_GAUSSIAN
    ns = g["n_steps"]
    dt = (g["t1"] - g["t0"]) / ns
    A = inputs.rotating_gaussian_potential(g, 2 * ns + 1)
    Ao, _, _ = oracle.gaussian_rotating_field(g["E0"], g["w"], g["tau"], g["t0"], dt / 2, 2 * ns + 1)
    assert A.shape == (2, 2 * ns + 1)
    assert np.all(A[:, 0] == 0.0)
    assert np.abs(A - Ao).max() < 1e-13 * np.abs(Ao).max()
