"""One DE population scored across ranks (Sec. IV.B, DE/rand/1/bin steps 1-4, with
the pair number N of Eq. (opt_prob) as the objective).

Every rank keeps the whole population (NP rows of 4K parameters: a few KiB) and
draws the same trial vectors.  The proposal is a pure function of the
population, the seed and the generation number (counter-based SplitMix64 keys,
see pp_de_propose), so it is replicated rather than broadcast.  Rank r
synthesises and scores only its contiguous slice of the NP trials; one
allgather of the NP pair numbers (8 B each) gives every rank all trial
fitnesses, and the replicated greedy selection keeps the ranks' populations
identical bit for bit.  Nothing else crosses ranks.  N of a candidate does not
depend on which other candidates share its launch (the momentum sum runs in a
fixed order per candidate), so a sharded generation equals the unsharded one
bit for bit.

The steps are passed in as callables: `library_steps` runs them through libpp on
the GPU, and `allgather_fn` exchanges through torch.distributed (NCCL between
GPUs, gloo between CPU processes).
"""


def shard_bounds(NP, world, rank):
    """The contiguous slice [first, last) of the NP trials that `rank` scores; slice
    sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside a world of %d" % (rank, world))
    return NP * rank // world, NP * (rank + 1) // world


def allgather_fn(dist):
    """gather(N_local, NP, world) -> the NP trial fitnesses in trial order: every
    rank contributes its slice (padded to the largest slice, so each rank sends the
    same number of elements) through dist.all_gather."""
    import torch

    def gather(n_local, NP, world):
        counts = [b - a for a, b in (shard_bounds(NP, world, r) for r in range(world))]
        buf = torch.zeros(max(counts), dtype=n_local.dtype, device=n_local.device)
        buf[:n_local.numel()] = n_local
        parts = [torch.empty_like(buf) for _ in range(world)]
        dist.all_gather(parts, buf)
        return torch.cat([p[:c] for p, c in zip(parts, counts)])
    return gather


def library_steps(pp, spec, grid, lo, hi, periodic, F, CR, seed, precision="fp32fast", scheme="magnus4",
                  stream=None):
    """(propose, score, select) through libpp for device tensors: pp_de_propose of the
    whole population, pp_synth_field + pp_pair_number of a slice of trials, and
    pp_de_select."""
    import torch
    dt = spec["T"] / spec["n_steps"]

    def propose(pop, generation):
        return pp.de_propose(pop, lo, hi, periodic, F, CR, seed, generation, stream=stream)

    def score(trials):
        if trials.shape[0] == 0:
            return torch.empty(0, dtype=torch.float64, device=trials.device)
        A, _, _ = pp.synth_field(trials.contiguous(), spec, stream=stream)
        N, _ = pp.pair_number(A, dt, grid, precision=precision, scheme=scheme, stream=stream)
        return N

    def select(pop, fit, trial, trial_fit):
        pp.de_select(pop, fit, trial, trial_fit, stream=stream)

    return propose, score, select


def sharded_generation(propose, score, select, gather, pop, fit, generation, rank, world):
    """One DE generation of the population pop [NP][D] with fitness fit [NP], both
    updated in place on every rank; returns (trial, trial_fit) of all NP trials."""
    NP = pop.shape[0]
    trial = propose(pop, generation)
    first, last = shard_bounds(NP, world, rank)
    n_local = score(trial[first:last])
    trial_fit = gather(n_local, NP, world) if world > 1 else n_local
    select(pop, fit, trial, trial_fit)
    return trial, trial_fit
