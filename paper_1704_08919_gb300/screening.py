"""Surrogate-screened differential evolution: the driver around the C ABI.

The surrogate (pp_mlp_*) maps the 4K pulse parameters to log10 N.  It is
trained on exact solver evaluations of seeded random pulses, then screens each
DE generation: every individual gets R DE/rand/1/bin proposals, the network
keeps NP of the R NP (each individual's best-ranked one, or the NP best-ranked
overall), and only those are scored by the exact solver (pp_de_screened_step),
so a generation costs NP exact evaluations as plain DE does.  The exact solver
decides: selection only ever compares exact pair numbers.  Optionally the
network is refitted online on the trials the exact solver scored.

Everything here is orchestration: device memory comes from PyTorch, every
computation is a call into the library.
"""
import time

import numpy as np

from . import inputs


def score_random(pp, n, spec, grid, seed, chunk=1024, precision="fp32fast", scheme="magnus4",
                 device="cuda"):
    """n seeded random pulses (uniform inside the parameter bounds) and their exact N.

    Returns (params FP64 [n, 4K], N FP64 [n]) on the device and the seconds taken.
    """
    import torch
    K = spec["K"]
    P = torch.tensor(inputs.random_population(n, K, seed), device=device)
    N = torch.empty(n, dtype=torch.float64, device=device)
    dt = spec["T"] / spec["n_steps"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c0 in range(0, n, chunk):
        sub = P[c0:c0 + chunk]
        A, _, _ = pp.synth_field(sub, spec)
        pp.pair_number(A, dt, grid, precision=precision, scheme=scheme, N_out=N[c0:c0 + chunk])
    torch.cuda.synchronize()
    return P, N, time.perf_counter() - t0


class LogTarget:
    """The standardisation of log10 N used for training (fixed from the training set)."""

    FLOOR = 1e-30

    def __init__(self, N_train):
        y = np.log10(np.maximum(N_train.double().cpu().numpy(), self.FLOOR))
        self.shift = float(y.mean())
        self.scale = float(y.std()) or 1.0

    def targets(self, pp, N):
        return pp.log_targets(N, self.FLOOR, self.shift, self.scale)

    def to_log10(self, y):
        return np.asarray(y, dtype=np.float64) * self.scale + self.shift


def held_out_error(pp, net, lt, P, N, lo, hi):
    """Error of the trained network on held-out pulses, in log10 N."""
    X = pp.mlp_features(P, lo, hi)
    pred = np.empty(X.shape[0])
    for b in range(0, X.shape[0], net.max_batch):
        pred[b:b + net.max_batch] = net.forward(X[b:b + net.max_batch].contiguous()).cpu().numpy()
    pred = lt.to_log10(pred)
    true = np.log10(np.maximum(N.cpu().numpy(), lt.FLOOR))
    err = pred - true
    rank = lambda v: np.argsort(np.argsort(v))  # noqa: E731
    return {"rmse_log10": float(np.sqrt(np.mean(err ** 2))),
            "mae_log10": float(np.mean(np.abs(err))),
            "r2": float(1.0 - np.mean(err ** 2) / np.var(true)),
            "spearman": float(np.corrcoef(rank(pred), rank(true))[0, 1]),
            "n": int(X.shape[0])}


def mean_loss(pp, net, X, t):
    """The network's mean squared error on rows X, t (pp_mlp_loss_grad over slices of
    at most max_batch rows, weighted by slice length)."""
    tot = 0.0
    for b in range(0, X.shape[0], net.max_batch):
        loss, _ = net.loss_grad(X[b:b + net.max_batch].contiguous(), t[b:b + net.max_batch].contiguous())
        tot += loss.item() * min(net.max_batch, X.shape[0] - b)
    return tot / X.shape[0]


def run_de(pp, pop0, fit0, spec, grid, generations, seed, F, CR, net=None, R=8, lt=None,
           online=None, precision="fp32fast", scheme="magnus4", target=None, mode="individual",
           seen=None):
    """`generations` DE generations from (pop0, fit0); plain DE when net is None.

    online = (every, epochs, batch, lr) refits the network on all trials the
    exact solver scored so far (plus `seen` = (features, N) scored before the run,
    if given) every `every` generations, the rows reshuffled in every epoch; mode is the screening mode of
    pp_de_screened_step ("individual" or "global").  Stops early once the best N
    reaches `target` (if given).  Returns the best N after the initial population
    and after every generation, the exact-evaluation count at each of those
    points, the wall-clock seconds (device-synchronised), the final population
    and fitness, and per refit (generation, rows, mean loss on those rows before
    and after, seconds).
    """
    import torch
    lo, hi, per = (torch.tensor(x, device=pop0.device) for x in inputs.param_bounds(spec["K"]))
    pop, fit = pop0.clone(), fit0.clone()
    NP, D = pop.shape
    trial = torch.empty_like(pop)
    tfit = torch.empty_like(fit)
    seen_P, seen_N = ([seen[0]], [seen[1]]) if seen is not None else ([], [])
    refits = []
    best = [fit.max().item()]
    calls = [NP]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for g in range(generations):
        if net is None:
            pp.de_step(pop, fit, spec, grid, lo, hi, per, F, CR, seed, g, precision=precision,
                       scheme=scheme)
        else:
            pp.de_screened_step(pop, fit, spec, grid, lo, hi, per, F, CR, seed, g, R, net,
                                precision=precision, scheme=scheme, mode=mode, trial_out=trial,
                                trial_fit_out=tfit)
            if online is not None:
                every, epochs, batch, lr = online
                seen_P.append(pp.mlp_features(trial, lo, hi))
                seen_N.append(tfit.clone())
                if (g + 1) % every == 0:
                    X = torch.cat(seen_P)
                    t = lt.targets(pp, torch.cat(seen_N))
                    before = mean_loss(pp, net, X, t)
                    torch.cuda.synchronize()
                    t_fit = time.perf_counter()
                    net.fit(X, t, batch, epochs, lr, lr, seed=g + 1)  # rows reshuffled every epoch
                    torch.cuda.synchronize()
                    t_fit = time.perf_counter() - t_fit
                    refits.append({"generation": g, "rows": int(X.shape[0]), "loss_before": before,
                                   "loss_after": mean_loss(pp, net, X, t), "seconds": t_fit})
        best.append(fit.max().item())
        calls.append(calls[-1] + NP)
        if target is not None and best[-1] >= target:
            break
    torch.cuda.synchronize()
    return {"best": best, "calls": calls, "seconds": time.perf_counter() - t0, "pop": pop, "fit": fit,
            "refits": refits}


def calls_to_reach(run, target):
    """Exact evaluations after which run's best N first reached target (None if never)."""
    for b, c in zip(run["best"], run["calls"]):
        if b >= target:
            return c
    return None
