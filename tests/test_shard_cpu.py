"""One DE population sharded across ranks (paper_1704_08919_gb300.shard) on CPU:
two gloo ranks, each scoring its slice of the trials with the oracle's host
mirror of the library calls (pp_oracle_de_propose, pp_oracle_synth_field,
pp_oracle_pair_number, pp_oracle_de_select), exchange the pair numbers by an
allgather, and must end with the population and fitness of the unsharded run,
bit for bit, generation after generation."""
import ctypes
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

K = 5
SPEC = dict(K=K, order=4, w_min=0.0, w_max=2.0, T=30.0, fluence=2.0, n_steps=300)
GRID = dict(nx=4, ny=3, nz=3, x0=-1.0, x1=1.0, y0=-0.9, y1=0.8, z0=0.0, z1=1.0, mirror_z=1)
NP, GENS, SEED, F, CR = 7, 3, 21, 0.8, 0.9


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def mirror_steps():
    """(propose, score, select) on host arrays through the oracle's mirror calls."""
    import oracle
    import paper_1704_08919_gb300 as pp
    from paper_1704_08919_gb300 import inputs
    L = oracle.lib()
    lo, hi, per = inputs.param_bounds(K)
    per = per.astype(np.uint8)
    spec, grid = pp._spec(SPEC), pp._grid(GRID)
    n = SPEC["n_steps"]
    dt = SPEC["T"] / n

    def propose(pop, gen):
        trial = np.zeros_like(pop)
        rc = L.pp_oracle_de_propose(_ptr(pop), pop.shape[0], pop.shape[1], _ptr(lo), _ptr(hi), _ptr(per),
                                    F, CR, SEED, gen, _ptr(trial), None)
        assert rc == 0
        return trial

    def score(trials):
        trials = np.ascontiguousarray(trials)
        m = trials.shape[0]
        A = np.zeros((m, 2, 2 * n + 1))
        N = np.zeros(m)
        if m:
            assert L.pp_oracle_synth_field(_ptr(trials), m, ctypes.byref(spec), _ptr(A), 2 * n + 1, None, None,
                                           None) == 0
            assert L.pp_oracle_pair_number(_ptr(A), m, 2 * n + 1, None, dt, ctypes.byref(grid), 0, 0, _ptr(N),
                                           None, None) == 0
        return N

    def select(pop, fit, trial, tfit):
        assert L.pp_oracle_de_select(_ptr(pop), _ptr(fit), _ptr(trial), _ptr(np.ascontiguousarray(tfit)),
                                     pop.shape[0], pop.shape[1], None) == 0

    return propose, score, select


def run_generations(rank, world, gather):
    from paper_1704_08919_gb300 import inputs, shard
    propose, score, select = mirror_steps()
    pop = inputs.random_population(NP, K, seed=3)
    fit = score(pop)
    history = []
    for g in range(GENS):
        trial, tfit = shard.sharded_generation(propose, score, select, gather, pop, fit, g, rank, world)
        history.append((pop.copy(), fit.copy(), np.asarray(tfit).copy()))
    return history


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1704_08919_gb300 import shard
    tgather = shard.allgather_fn(dist)

    def gather(n_local, np_total, w):  # host arrays through torch CPU tensors
        return tgather(torch.from_numpy(np.ascontiguousarray(n_local)), np_total, w).numpy()
    try:
        q.put((rank, run_generations(rank, world, gather)))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_shard_bounds_cover_the_population_once():
    from paper_1704_08919_gb300 import shard
    for NPt in (4, 7, 64, 65, 1024):
        for world in (1, 2, 3, 8):
            b = [shard.shard_bounds(NPt, world, r) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == NPt
            assert all(b[r][1] == b[r + 1][0] for r in range(world - 1))
            sizes = [hi - lo for lo, hi in b]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.shard_bounds(8, 2, 2)


def test_two_gloo_ranks_reproduce_the_unsharded_generations():
    import torch.multiprocessing as mp
    ref = run_generations(0, 1, None)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from paper_1704_08919_gb300 import inputs
    for g in range(GENS):
        pop_r, fit_r, tfit_r = ref[g]
        for rank in (0, 1):
            pop, fit, tfit = res[rank][g]
            assert np.array_equal(pop, pop_r) and np.array_equal(fit, fit_r)
            assert np.array_equal(tfit, tfit_r)
    # selection replaced some individuals, so the exchanged pair numbers decided something
    pop0 = inputs.random_population(NP, K, seed=3)
    changed = np.any(ref[-1][0] != pop0, axis=1)
    assert changed.sum() > 0
