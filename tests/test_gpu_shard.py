"""The sharded DE generation (paper_1704_08919_gb300.shard) driven by the library's
calls on one GPU: with one rank it is pp_de_step's composition, so three
generations must reproduce pp_de_step bit for bit; with the ranks' slices scored
one after another on the same GPU and concatenated (the allgather's result), the
trial fitnesses equal those of the whole population scored at once."""
import pytest

from paper_1704_08919_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

K = 6
SPEC = dict(K=K, order=4, w_min=0.0, w_max=2.0, T=40.0, fluence=2.0, n_steps=800)
GRID = inputs.small_grid(12, 10, 5)


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


def setup(pp, NP, seed=3):
    lo, hi, per = (torch.tensor(x, device="cuda") for x in inputs.param_bounds(K))
    pop = torch.tensor(inputs.random_population(NP, K, seed=seed), device="cuda")
    A, _, _ = pp.synth_field(pop, SPEC)
    fit, _ = pp.pair_number(A, SPEC["T"] / SPEC["n_steps"], GRID, precision="fp32fast", scheme="magnus4")
    return pop, fit, lo, hi, per


def test_one_rank_is_de_step(pp):
    from paper_1704_08919_gb300 import shard
    pop, fit, lo, hi, per = setup(pp, 12)
    a_pop, a_fit = pop.clone(), fit.clone()
    b_pop, b_fit = pop.clone(), fit.clone()
    propose, score, select = shard.library_steps(pp, SPEC, GRID, lo, hi, per, 0.8, 0.9, 41)
    for g in range(3):
        pp.de_step(a_pop, a_fit, SPEC, GRID, lo, hi, per, 0.8, 0.9, 41, g, precision="fp32fast",
                   scheme="magnus4")
        shard.sharded_generation(propose, score, select, None, b_pop, b_fit, g, 0, 1)
    assert pp.sync_status() == pp.PP_OK
    assert torch.equal(a_pop, b_pop) and torch.equal(a_fit, b_fit)
    assert not torch.equal(a_pop, pop)


@pytest.mark.parametrize("world", [2, 3])
def test_slices_scored_apart_equal_the_whole(pp, world):
    from paper_1704_08919_gb300 import shard
    pop, fit, lo, hi, per = setup(pp, 13, seed=5)
    propose, score, select = shard.library_steps(pp, SPEC, GRID, lo, hi, per, 0.8, 0.9, 43)
    trial = propose(pop, 7)
    whole = score(trial)
    parts = [score(trial[a:b]) for a, b in (shard.shard_bounds(13, world, r) for r in range(world))]
    assert pp.sync_status() == pp.PP_OK
    assert torch.equal(torch.cat(parts), whole)
