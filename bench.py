"""Throughput of candidate-pulse scoring inside the DE loop (arXiv 1704.08919).

Workload (one "step" = one DE generation of the whole hot path): a population
of 64 B-spline pulses (K = 8, cubic, band [0, 2], T = 200, 8192 RK4 steps,
fluence 2.0), momentum grid 64 x 64 x 32 over [-2, 2]^2 x [0, 2] with the p_z
mirror; per generation: DE/rand/1/bin proposal (F = 0.8, CR = 0.9), synthesis
of the 64 trial pulses, their pair numbers (FP32 propagation, FP64 projection
and momentum sum), greedy selection -- all through pp_de_step.

Prints one JSON line.  `value` is candidate pulses scored per second over all
ranks (64 per rank per step); mode-steps/s, the live roofline of the
propagation kernel, the FP32-vs-FP64 N error, clocks, an end-to-end figure
with host buffers and a CPU-oracle baseline are added.  `--impl reference`
times the FP64 CPU oracle instead (rank 0 only under torchrun).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1704_08919_gb300 import inputs, shard  # noqa: E402

CFG = inputs.DE_BATCH
# Arithmetic of one mode-step (one momentum mode, both spin channels, one
# step) of the propagation kernel, counted from its source: (flop with
# FMA = 2, FP32/FP64 instructions).  FP32 paths use compensated accumulation.
#  rk4:     4 matrix applications, 3 stage updates, increment sum, Fast2Sum
#  magnus4: dt h_eff, |.|^2, tan(th)/th polynomial (FP32, tracked norm; FP64: cos-1 and
#           sinc polynomials), scaled vector, increment, Fast2Sum
#  split2:  coupling factor, stage, free factor, Fast2Sum
WORK = {("fp32", "rk4"): (268, 184), ("fp32", "magnus4"): (116, 84), ("fp32", "split2"): (144, 96),
        ("fp32fast", "rk4"): (244, 160), ("fp32fast", "magnus4"): (92, 52),
        ("fp32fast", "split2"): (112, 64),
        ("fp64", "rk4"): (244, 148), ("fp64", "magnus4"): (114, 64), ("fp64", "split2"): (112, 64)}
# DRAM bytes per candidate per launch of the propagation kernel, from ncu captures
# (profiles/): the FP32-fast Magnus kernel (256 threads, 8 KiB tiles) read 1.090816 MB for 4 candidates.
TRAFFIC_PER_CAND = {("fp32fast", "magnus4"): 1.090816e6 / 4}
FP32_LANES_PER_SM = 128
# GB300 FP64 rate from the part's datasheet figure (no measured FP64 peak exists
# for this pool); FP32 is derived from the device's SM count and maximum clock.
FP64_NOMINAL_TFLOPS = 1.25
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32fast", choices=["fp32fast", "fp32", "fp64"])
    ap.add_argument("--no-tune", action="store_true", help="skip the launch-configuration tuner")
    ap.add_argument("--alt-steps", type=int, default=2,
                    help="timed generations of the compensated FP32 path reported beside the main one")
    ap.add_argument("--scheme", default="magnus4", choices=["magnus4", "rk4", "split2"])
    ap.add_argument("--cpu-modes", type=int, default=8192,
                    help="modes of one candidate in the CPU-oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="de-batch", choices=["de-batch", "uneven", "surrogate", "gemm", "localsearch", "large",
                             "single"],
                    help="de-batch: the 64-candidate DE generation (default); uneven: 128 slots "
                         "of uneven length and grid, generations in one CUDA graph; surrogate: "
                         "exact calls of surrogate-screened DE against plain DE")
    ap.add_argument("--train", type=int, default=None, help="surrogate: training pulses")
    ap.add_argument("--generations", type=int, default=None, help="surrogate: DE generations")
    ap.add_argument("--seeds", type=int, default=5, help="surrogate: DE runs (seeds) per form")
    ap.add_argument("--eval-only", action="store_true",
                    help="localsearch: time the batched gradient evaluation only (no search)")
    ap.add_argument("--small", action="store_true",
                    help="localsearch: a 16 x 16 x 8 grid (profiling runs)")
    ap.add_argument("--qke-state-budget", type=float, default=None,
                    help="localsearch: GiB of device memory the QKE adjoint may keep forward states in "
                         "(default: the library's, half the device memory)")
    ap.add_argument("--qke-steps", type=int, default=None,
                    help="localsearch: RK4 steps per pulse instead of the workload's 16384 (profiling runs)")
    ap.add_argument("--screen", default="global", choices=["individual", "global"],
                    help="surrogate: screening mode reported as the value (default: global, the top NP "
                         "of all 8 NP proposals kept for exact scoring)")
    ap.add_argument("--online", type=int, default=0,
                    help="surrogate: also run a screened DE refitted every N generations (0: off)")
    ap.add_argument("--ncand", type=int, default=CFG["NP"],
                    help="population size (smaller values only for profiling runs)")
    ap.add_argument("--branch", type=int, default=0,
                    help="large: generations run with and without the scheduled refit after --steps")
    ap.add_argument("--refit-epochs", type=int, default=20, help="large: epochs of the scheduled refit")
    ap.add_argument("--no-configs", action="store_true",
                    help="de-batch: skip the sub-records of the other configurations (single-field "
                         "FP64 solve, FP64 DE generation, uneven batch)")
    ap.add_argument("--no-oracle-n", action="store_true",
                    help="de-batch: skip the oracle's full-grid N of one candidate")
    return ap.parse_args()


def device_peaks(local):
    """ALU peaks of this GPU for the roofline: FP32 = SMs (read from the device) x 128
    lanes x 2 flop x the maximum SM clock (nvidia-smi clocks.max.sm, else the clock
    recorded in MEASURED_PEAKS.json); FP64 = the nominal datasheet figure
    (MEASURED_PEAKS.json holds HBM and BF16 figures only).  Beside them, the FMA
    rates this GPU sustains in FP32 and FP64, measured by pp_fma_rate."""
    import torch
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    clk, src = None, None
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(local), "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True,
                             timeout=20).stdout.strip()
        clk, src = float(out.splitlines()[0]), "nvidia-smi clocks.max.sm"
    except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
        pass
    if clk is None:
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                clk, src = float(json.load(f)["sm_max_mhz"]), "MEASURED_PEAKS.json sm_max_mhz"
        except (OSError, KeyError, ValueError):
            clk, src = 2070.0, "GB300 maximum SM clock (datasheet)"
    fp32 = sms * FP32_LANES_PER_SM * 2 * clk * 1e6 / 1e12
    if local not in _FMA_RATES:  # the FMA rate this GPU sustains, measured once per process
        import paper_1704_08919_gb300 as pp
        _FMA_RATES[local] = (pp.fma_rate("fp32") / 1e12, pp.fma_rate("fp64") / 1e12)
    m32, m64 = _FMA_RATES[local]
    return {"sm_count": sms, "sm_max_mhz": clk, "fp32_tflops": fp32, "fp64_tflops": FP64_NOMINAL_TFLOPS,
            "fp32_lanes_per_s": sms * FP32_LANES_PER_SM * clk * 1e6,
            "fp32_source": "nominal, derived: %d SMs (device) x %d FP32 lanes x 2 flop x %g MHz (%s)"
                           % (sms, FP32_LANES_PER_SM, clk, src),
            "fp64_source": "nominal: GB300 FP64 %.2f TFLOP/s datasheet figure" % FP64_NOMINAL_TFLOPS,
            "fp32_measured_tflops": m32, "fp64_measured_tflops": m64,
            "measured_source": "pp_fma_rate: a kernel of independent FMA chains only, a multiple of the SM "
                               "count in CTAs, timed with CUDA events in this process"}


_FMA_RATES = {}


def measured_peak(peaks, fp32, achieved):
    """Roofline fields against the FMA rate measured on this GPU (beside the derived peak)."""
    m = peaks["fp32_measured_tflops"] if fp32 else peaks["fp64_measured_tflops"]
    return {"peak_measured": m, "frac_of_measured": achieved / m, "peak_measured_source": peaks["measured_source"]}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seeds(rank):
    """(population seed, DE seed) of a rank: every rank evolves its own population."""
    return 1 + rank, 1000 + rank


def max_over_ranks(x, dist=None, device=None):
    """The maximum of a per-rank scalar over all ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def throughput(world_size, NP, steps, total_ms):
    """Candidates scored per second by the whole job (weak scaling: NP per rank per step)."""
    return world_size * NP * steps / (total_ms / 1000.0)


def workload_config(precision, NP=None, scheme="rk4"):
    g = CFG["grid"]
    return {
        "workload": CFG["name"], "scheme": scheme,
        "NP": NP or CFG["NP"], "K": CFG["K"], "order": CFG["order"], "T": CFG["T"],
        "n_steps": CFG["n_steps"], "fluence": CFG["fluence"],
        "grid": "%dx%dx%d px,py in [%g,%g], pz in [%g,%g] mirrored" % (
            g["nx"], g["ny"], g["nz"], g["x0"], g["x1"], g["z0"], g["z1"]),
        "F": CFG["F"], "CR": CFG["CR"], "precision": precision,
        "l2": "flushed between timed steps (256 MiB write)",
    }


def units_per_candidate():
    g = CFG["grid"]
    return g["nx"] * g["ny"] * g["nz"] * CFG["n_steps"]


# ----------------------------------------------------------------------------- clocks


class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_median": statistics.median(power)}


# ----------------------------------------------------------------------------- oracle legs


def oracle_sample(A_host, cand, nmodes, seed=0, nthreads=0):
    """The FP64 CPU oracle on `nmodes` strided modes of one candidate: (seconds, n, idx, cores)."""
    import oracle
    idx = inputs.strided_modes(CFG["grid"], nmodes, seed=seed)
    pts = inputs.grid_points(CFG["grid"])[idx]
    dt = CFG["T"] / CFG["n_steps"]
    t0 = time.perf_counter()
    n = oracle.dirac_modes(A_host[cand], CFG["n_steps"], dt, pts, nthreads=nthreads)
    el = time.perf_counter() - t0
    return el, n, idx, oracle.num_threads(nthreads)


def reference_main(args):
    """--impl reference: the FP64 CPU oracle, as it stands, on the host cores."""
    import oracle
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    params = inputs.random_population(CFG["NP"], CFG["K"], seed=1)
    nm = max(256, args.cpu_modes // 4)
    A, _, _, rc = oracle.synth_field(params[:1], CFG["K"], CFG["order"], CFG["w_min"], CFG["w_max"],
                                     CFG["T"], CFG["fluence"], CFG["n_steps"], want_E=False)
    for _ in range(args.warmup):
        oracle_sample(A, 0, 64)
    times = []
    for s in range(args.steps):
        el, _, _, cores = oracle_sample(A, 0, nm, seed=s)
        times.append(el)
    per_mode_step = sum(times) / (args.steps * nm * CFG["n_steps"])
    cand_per_s = 1.0 / (per_mode_step * units_per_candidate())
    sample = ("%d strided modes of one candidate x %d RK4 steps per step; the oracle's synthesis "
              "is excluded; candidates/s extrapolated by mode-steps" % (nm, CFG["n_steps"]))
    line = {
        "metric": "candidate pulses scored/s (DE batch, rel. N err <= 1e-4 vs FP64 oracle)",
        "value": cand_per_s, "unit": "candidates/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup,
        # each step is the bounded sample: its mean wall time, not a whole generation's
        "ms_per_step": 1000.0 * sum(times) / args.steps,
        "ms_per_generation_extrapolated": 1000.0 * CFG["NP"] / cand_per_s,
        "units_per_step": "%d of the %d mode x step units of one candidate" % (
            nm * CFG["n_steps"], units_per_candidate()),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded B-spline pulses)",
        # the same workload as the library arm; this arm computes it in FP64 RK4 (the oracle)
        "config": workload_config(args.precision, None, args.scheme),
        "arm_precision": "fp64", "arm_scheme": "rk4",
        "impl": "reference", "mode_steps_per_s": 1.0 / per_mode_step,
        "cpu_baseline": {"value": cand_per_s, "unit": "candidates/s", "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": cand_per_s, "unit": "candidates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- uneven batch


def measure_uneven(pp, torch, local, peaks, G, precision="fp32fast", scheme="magnus4", tune=True,
                   pop_seed=1, seed=1000, dist=None):
    """The uneven batch: 128 slots of uneven length and grid; G DE generations as one
    CUDA graph launch (pp_batch_de_run), timed with CUDA events after a capture and
    warm-up launch of the same graph.  Returns (record, total_ms)."""
    U = inputs.UNEVEN_BATCH
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    steps = inputs.uneven_steps(U, pop_seed)
    specs = inputs.uneven_specs(U, steps)
    pop = torch.tensor(inputs.random_population(U["NP"], U["K"], seed=pop_seed), device=dev)
    peaks_E = []
    for c, sp in enumerate(specs):
        _, E, _ = pp.synth_field(pop[c:c + 1].contiguous(), sp, want_E=True)
        peaks_E.append(torch.sqrt(E[0, 0] ** 2 + E[0, 1] ** 2).max().item())
    grids = inputs.grids_by_rank(U, peaks_E)
    b = pp.Batch(specs, grids, U["dt"], precision=precision, scheme=scheme)
    lo, hi, per = inputs.param_bounds(U["K"])
    lo_t, hi_t, per_t = (torch.tensor(x, device=dev) for x in (lo, hi, per))
    A = b.synth(pop)
    tuned = None
    if tune:
        chosen, cfg_ms = b.tune(A)
        tuned = {"chosen": pp.launch_configs()[chosen], "ms": [round(x, 2) for x in cfg_ms]}
    fit, _ = b.pair_number(A)
    b.set_generation(0)
    b.de_run(pop, fit, lo_t, hi_t, per_t, U["F"], U["CR"], seed, G)  # capture + warm-up
    torch.cuda.synchronize()
    if pp.sync_status() != pp.PP_OK:
        raise RuntimeError("uneven batch: warm-up failed")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e0.record(stream)
    b.de_run(pop, fit, lo_t, hi_t, per_t, U["F"], U["CR"], seed, G)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if pp.sync_status() != pp.PP_OK:
        raise RuntimeError("uneven batch: device status after the timed region")
    total_ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    modes = np.array([g["nx"] * g["ny"] * g["nz"] for g in grids], dtype=np.float64)
    mode_steps = float(np.sum(modes * steps)) * G
    # accuracy: 4 slots of the final population, this path against FP64 RK4
    idx = list(range(4))
    sub_specs = [specs[i] for i in idx]
    sub_grids = [grids[i] for i in idx]
    bf = pp.Batch(sub_specs, sub_grids, U["dt"], precision=precision, scheme=scheme)
    b64 = pp.Batch(sub_specs, sub_grids, U["dt"], precision="fp64", scheme="rk4")
    As = bf.synth(pop[idx].contiguous())
    Nf, _ = bf.pair_number(As)
    N64, _ = b64.pair_number(As)
    pp.sync_status()
    rel_err = (Nf / N64 - 1).abs().max().item()
    for x in (bf, b64, b):
        x.close()
    if rel_err > 1e-4:
        raise RuntimeError("uneven batch: N error %.3e vs FP64 RK4 exceeds 1e-4" % rel_err)
    flop, inst = WORK[(precision, scheme)]
    fp32 = precision != "fp64"
    pk = peaks["fp32_tflops"] if fp32 else peaks["fp64_tflops"]
    achieved = flop * mode_steps / (total_ms * 1e-3) / 1e12
    rec = {"workload": U["name"], "NP": U["NP"], "precision": precision, "scheme": scheme,
           "generations": G, "ms_per_generation": total_ms / G,
           "candidates_per_s": U["NP"] * G / (total_ms * 1e-3),
           "mode_steps_per_s": mode_steps / (total_ms * 1e-3),
           "steps_per_slot": [int(steps.min()), int(steps.max())],
           "modes_per_slot": [int(modes.min()), int(modes.max())],
           "graph": "%d generations per CUDA graph launch" % G,
           "l2": "not flushed between generations inside the graph (ALU-bound kernel)",
           "n_rel_err_vs_fp64_rk4_max": rel_err, "launch_tuning": tuned, "clocks": clk,
           "roofline": {"bound": "alu", "kernel": "propagate_batch_kernel<%s>" % scheme,
                        "achieved": achieved, "peak": pk, "unit": "TFLOP/s", "frac": achieved / pk,
                        "peak_source": peaks["fp32_source"] if fp32 else peaks["fp64_source"],
                        **measured_peak(peaks, fp32, achieved),
                        "flop_per_mode_step": flop,
                        "note": "whole graph timed (proposal, synthesis, tables, propagation, selection)"},
           # per generation: proposal, spectrum, samples, table, propagation (+ its
           # wide-range twin for Magnus-4), partial sums, selection, generation counter
           "gpu_launches": (9 if scheme == "magnus4" else 8) * G}
    return rec, total_ms


def uneven_main(args):
    """--workload uneven: the uneven batch as its own JSON line; every rank runs its
    own population (weak scaling)."""
    import torch
    import paper_1704_08919_gb300 as pp
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    pp.lib()
    pop_seed, seed = rank_seeds(rank)
    G = args.steps
    rec, total_ms = measure_uneven(pp, torch, local, device_peaks(local), G, args.precision, args.scheme,
                                   not args.no_tune, pop_seed, seed, dist)
    if rank == 0:
        U = inputs.UNEVEN_BATCH
        print(json.dumps({
            "metric": "candidate pulses scored/s (uneven batch, rel. N err <= 1e-4 vs FP64 oracle)",
            "value": throughput(ws, U["NP"], G, total_ms), "unit": "candidates/s", "n_gpus": ws, "steps": G,
            "warmup": G, "ms_per_step": total_ms / G, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
            "scheme": args.scheme, "data": "synthetic (seeded B-spline pulses, uniform in bounds)",
            "config": {"workload": U["name"], "NP": U["NP"], "precision": args.precision,
                       "steps_per_slot": rec["steps_per_slot"], "modes_per_slot": rec["modes_per_slot"],
                       "graph": rec["graph"], "l2": rec["l2"]},
            "mode_steps_per_s": ws * rec["mode_steps_per_s"],
            "n_rel_err_vs_fp64_rk4_max": rec["n_rel_err_vs_fp64_rk4_max"], "launch_tuning": rec["launch_tuning"],
            "roofline": rec["roofline"], "clocks": rec["clocks"], "gpu_launches": rec["gpu_launches"]}),
            flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# ----------------------------------------------------------------------------- surrogate


# both shapes touch more than the 129 MB L2 per launch (201 MB and 153 MB), so the
# launches are timed back to back without an L2 flush
GEMM_SHAPES = ((131072, 256, 256), (16384, 256, 4096))


def measured_peaks():
    """HBM copy bandwidth (GB/s) and bf16 GEMM rate (TFLOP/s) measured on this GPU model,
    else the fallback figures of an earlier GB300 measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


def gemm_measure(pp, torch, reps=20):
    """Live timing of pp_gemm_bf16 (the tensor-core kernel of the surrogate) on two
    shapes: a hidden layer over a large batch (HBM-bound: FP32 output) and a
    long contraction (tensor-bound).  Algorithmic bytes = packed A and B read once
    + FP32 D written once; flop = 2 M N K."""
    import math as _m
    PEAKS = measured_peaks()
    out = []
    for M, N, K in GEMM_SHAPES:
        g = torch.Generator(device="cuda").manual_seed(M + K)
        A = torch.rand((M, K), device="cuda", generator=g) - 0.5
        B = torch.rand((N, K), device="cuda", generator=g) - 0.5
        Ap, _, _ = pp.pack_bf16(A)
        Bp, _, _ = pp.pack_bf16(B)
        del A, B
        D = torch.empty((M, N), dtype=torch.float32, device="cuda")
        for _ in range(3):
            pp.gemm_bf16(Ap, Bp, M, N, K, out=D)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(reps):
            pp.gemm_bf16(Ap, Bp, M, N, K, out=D)
        e1.record(st)
        torch.cuda.synchronize()
        if pp.sync_status() != pp.PP_OK:
            raise RuntimeError("GEMM failed")
        ms = e0.elapsed_time(e1) / reps
        flop = 2.0 * M * N * K
        byts = 2.0 * (M * K + N * K) + 4.0 * M * N
        tf = flop / (ms * 1e-3) / 1e12
        gbs = byts / (ms * 1e-3) / 1e9
        ai = flop / byts
        bound = "tensor" if ai > 1e3 * PEAKS["bf16_tflops"] / PEAKS["hbm_gbs"] else "hbm"
        frac = tf / PEAKS["bf16_tflops"] if bound == "tensor" else gbs / PEAKS["hbm_gbs"]
        out.append({"M": M, "N": N, "K": K, "ms": ms, "tflops": tf, "gbs": gbs,
                    "flop_per_byte": _m.floor(ai * 10) / 10, "bound": bound,
                    "frac": frac, "peak_source": PEAKS["source"],
                    "l2": "inputs larger than L2 (%.0f MB per launch), launches back to back" % (byts / 1e6)})
    return out


# FP32 work per mode-step of the QKE adjoint kernel with every forward state kept
# (forward step and backward step; the variant the default state budget selects at
# the local-search size), from the kernel's executed instruction counts (ncu,
# 7 starts x 16384 modes x 1024 steps): 223.0 FFMA + 153.1 FMUL + 67.0 FADD
# thread-instructions, i.e. 666 flop (FMA = 2) in 443 FP32 instructions.
QKE_ADJ_FLOP = 666
QKE_ADJ_FP32_INSTR = 443


def localsearch_main(args):
    """Multistart augmented-Lagrangian local search (Sec. IV.A) on the QKE: the
    native optimiser drives batched adjoint-gradient evaluations on the GPU."""
    import torch
    import paper_1704_08919_gb300 as pp
    L = inputs.LOCAL_SEARCH
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    pp.lib()
    if args.qke_state_budget is not None:
        pp.set_qke_state_budget(int(args.qke_state_budget * 2 ** 30))
    cur = pp.set_qke_state_budget(-1)
    pp.set_qke_state_budget(cur)
    budget_gib = "default: half the device memory" if cur < 0 else cur / 2 ** 30
    if args.qke_steps:
        L = dict(L, n_steps=args.qke_steps)
    sp = inputs.field_spec(dict(L, fluence=1.0))
    K = L["K"]
    S = args.ncand if args.ncand != CFG["NP"] else L["nstart"]
    if args.small:
        L = dict(L, grid=dict(L["grid"], nx=16, ny=16, nz=8))
    prec = "fp64" if args.precision == "fp64" else "fp32"
    X = inputs.random_population(S, K, seed=L["seed"])
    Xd = torch.tensor(X, device="cuda")
    _, _, U, _ = pp.qke_gradient(Xd, sp, L["grid"], prec, want_grad=False)
    sc = np.sqrt(L["U_const"] / U.cpu().numpy())
    X[:, :K] *= sc[:, None]
    X[:, 2 * K:3 * K] *= sc[:, None]
    Xd = torch.tensor(X, device="cuda")
    # one batched evaluation (all starts): forward + adjoint + chain rule, timed alone
    for _ in range(2):
        pp.qke_gradient(Xd, sp, L["grid"], prec)
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    e0.record(st)
    reps = 3
    for _ in range(reps):
        J0, _, _, _ = pp.qke_gradient(Xd, sp, L["grid"], prec)
    e1.record(st)
    torch.cuda.synchronize()
    eval_ms = e0.elapsed_time(e1) / reps
    g = L["grid"]
    mode_steps = g["nx"] * g["ny"] * g["nz"] * L["n_steps"] * S
    t0 = time.perf_counter()
    if args.eval_only:
        r = None
    else:
        r = pp.local_search(X, sp, L["grid"], L["U_const"], precision=prec, mu0=L["mu0"], xi=L["xi"],
                            outer=L["outer"], max_iter=L["max_iter"], gtol=L["gtol"], ctol=L["ctol"])
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    if pp.sync_status() != pp.PP_OK:
        raise RuntimeError("device status after the local search")
    J0 = J0.cpu().numpy()
    pk = device_peaks(local)
    achieved = QKE_ADJ_FLOP * mode_steps / (eval_ms * 1e-3) / 1e12
    peak = pk["fp32_tflops"]
    print(json.dumps({
        "metric": "local-search gradient evaluations/s (QKE forward + adjoint, all starts batched)",
        "value": S / (eval_ms * 1e-3), "unit": "gradients/s", "n_gpus": 1, "steps": reps,
        "warmup": 2, "ms_per_step": eval_ms, "higher_is_better": True, "scaling": "none",
        "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "f64",
        "data": "synthetic (seeded B-spline pulses scaled to U_const)",
        "config": {"workload": L["name"], "precision": prec, "grid": "%dx%dx%d" % (g["nx"], g["ny"], g["nz"]),
                   "n_steps": L["n_steps"], "T": L["T"], "nstart": S, "qke_state_budget_gib": budget_gib,
                   "options": {k: L[k] for k in ("mu0", "xi", "outer", "max_iter", "gtol", "ctol")}},
        "mode_steps_per_s": mode_steps / (eval_ms * 1e-3),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "pipe_frac": QKE_ADJ_FP32_INSTR * mode_steps / (eval_ms * 1e-3)
                     / pk["fp32_lanes_per_s"],
                     "peak_source": pk["fp32_source"],
                     **measured_peak(pk, True, achieved),
                     "note": "%d FP32 flop (%d instructions) per mode-step from ncu SASS counts of the "
                             "kept-state adjoint; whole evaluation (synthesis, adjoint, chain rule) timed"
                             % (QKE_ADJ_FLOP, QKE_ADJ_FP32_INSTR)},
        "search": None if r is None else {
            "seconds": wall, "evals_total": int(r["evals"].sum()),
            "J_start": [float(v) for v in J0], "J_end": [float(v) for v in r["J"]],
            "C_end": [float(v) for v in r["C"]], "status": [int(v) for v in r["status"]],
            "outer": [int(v) for v in r["outer"]],
            "best_J": float(np.max(r["J"][r["status"] == 0])) if np.any(r["status"] == 0) else None},
        "clocks": clk}), flush=True)
    return 0


def large_main(args):
    """The large-scale configuration: population 1024, K = 16, T = 400 (20000 steps),
    grid 128 x 128 x 64, surrogate-screened DE (R = 8).  Scores the initial
    population and fits the network on those exact evaluations, then runs --steps
    generations (default 2).  With --branch B and --steps equal to the refit period
    (20), the run reaches the first scheduled refit and continues B generations two
    ways from the same state: with the network refitted on every pulse scored so far,
    and without.  The wall-clock of the configured 200 generations is extrapolated
    from the measured generation and refit times."""
    import torch
    import paper_1704_08919_gb300 as pp
    from paper_1704_08919_gb300 import screening as scr
    Lg = inputs.LARGE_SCALE
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    pp.lib()
    spec, grid = inputs.field_spec(Lg), Lg["grid"]
    K, D, NP, R = Lg["K"], 4 * Lg["K"], Lg["NP"], Lg["R"]
    G = args.steps
    prec, sch = args.precision, args.scheme
    lo, hi, per = (torch.tensor(x, device="cuda") for x in inputs.param_bounds(K))
    pop = torch.tensor(inputs.random_population(NP, K, seed=Lg["pop_seed"]), device="cuda")
    dt = spec["T"] / spec["n_steps"]
    modes = grid["nx"] * grid["ny"] * grid["nz"]
    clocks = ClockSampler(local)
    clocks.start()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    A, _, _ = pp.synth_field(pop, spec)
    fit, _ = pp.pair_number(A, dt, grid, precision=prec, scheme=sch)
    e1.record(st)
    torch.cuda.synchronize()
    init_ms = e0.elapsed_time(e1)
    del A
    lt = scr.LogTarget(fit)
    net = pp.Surrogate(D, 256, max_batch=R * NP)
    net.init(5)
    X = pp.mlp_features(pop, lo, hi)
    t = lt.targets(pp, fit)
    t0 = time.perf_counter()
    net.fit(X, t, 256, 200, 2e-3, 5e-5)
    torch.cuda.synchronize()
    fit_s = time.perf_counter() - t0
    seen_X, seen_N = [X], [fit.clone()]
    trial = torch.empty_like(pop)
    tfit = torch.empty_like(fit)

    def generations(net_g, pop_g, fit_g, g0, count, log):
        best, ms = [fit_g.max().item()], []
        for g in range(g0, g0 + count):
            e0.record(st)
            pp.de_screened_step(pop_g, fit_g, spec, grid, lo, hi, per, Lg["F"], Lg["CR"], Lg["de_seed"], g, R,
                                net_g, precision=prec, scheme=sch, trial_out=trial, trial_fit_out=tfit)
            e1.record(st)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            best.append(fit_g.max().item())
            if log:
                seen_X.append(pp.mlp_features(trial, lo, hi))
                seen_N.append(tfit.clone())
        return best, ms

    best, gen_ms = generations(net, pop, fit, 0, G, True)
    branch = None
    if args.branch > 0:
        # the first scheduled refit, then both continuations from the same state
        snap_pop, snap_fit, snap_w = pop.clone(), fit.clone(), net.get_params().clone()
        Xs = torch.cat(seen_X)
        ts = lt.targets(pp, torch.cat(seen_N))
        loss_before = scr.mean_loss(pp, net, Xs, ts)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        net.fit(Xs, ts, 256, args.refit_epochs, 2e-4, 2e-4, seed=G + 1)  # rows reshuffled every epoch
        torch.cuda.synchronize()
        refit_s = time.perf_counter() - t0
        loss_after = scr.mean_loss(pp, net, Xs, ts)
        best_r, ms_r = generations(net, pop, fit, G, args.branch, False)
        net_plain = pp.Surrogate(D, 256, max_batch=R * NP)
        net_plain.set_params(snap_w)
        best_p, ms_p = generations(net_plain, snap_pop, snap_fit, G, args.branch, False)
        net_plain.close()
        gen_ms += ms_r + ms_p
        calls = [NP * (G + 1 + k) for k in range(args.branch + 1)]
        branch = {"at_generation": G, "rows": int(Xs.shape[0]), "epochs": args.refit_epochs,
                  "refit_seconds": refit_s, "loss_before": loss_before, "loss_after": loss_after,
                  "exact_calls": calls, "best_N_with_refit": best_r, "best_N_without_refit": best_p}
        fit_s_refit = refit_s
    else:
        fit_s_refit = fit_s
    clk = clocks.stop()
    if pp.sync_status() != pp.PP_OK:
        raise RuntimeError("device status after the large-scale run")
    # accuracy: two scored trials of the last generation, this path against FP64 RK4
    idx = [0, 1]
    Ac, _, _ = pp.synth_field(trial[idx].contiguous(), spec)
    N64, _ = pp.pair_number(Ac, dt, grid, precision="fp64", scheme="rk4")
    rel = float((tfit[idx] / N64 - 1).abs().max().item())
    ms = statistics.mean(gen_ms)
    print(json.dumps({
        "metric": "candidate pulses scored/s (large-scale configuration, screened DE)",
        "value": NP / (ms * 1e-3), "unit": "candidates/s", "n_gpus": 1, "steps": len(gen_ms), "warmup": 0,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "none", "vs_baseline": None,
        "dtype": "f32" if prec != "fp64" else "f64", "data": "synthetic (seeded B-spline pulses)",
        "config": {"workload": Lg["name"], "precision": prec, "scheme": sch, "NP": NP, "K": K,
                   "T": Lg["T"], "n_steps": Lg["n_steps"], "grid": "128x128x64 over [-2.5,2.5]^2 x [0,2.5]",
                   "R": R, "generations_run": G, "branch_generations": args.branch,
                   "generations_configured": Lg["generations"]},
        "mode_steps_per_s": NP * modes * Lg["n_steps"] / (ms * 1e-3),
        "generation_ms": gen_ms, "initial_population_ms": init_ms, "surrogate_fit_s": fit_s,
        "best_N": best, "n_rel_err_vs_fp64_rk4_max": rel, "refit_branch": branch,
        "extrapolated_hours_for_configured_generations":
            (init_ms + ms * Lg["generations"]) / 3.6e6
            + fit_s_refit * (Lg["generations"] // Lg["refit_every"]) / 3600.0,
        "note": "%d generations to the branch point plus %d on each branch; the configured %d "
                "extrapolated from their mean time and %d refits at the measured refit time"
                % (G, args.branch, Lg["generations"], Lg["generations"] // Lg["refit_every"]),
        "clocks": clk}), flush=True)
    return 0


def measure_single(pp, torch, local, peaks, steps=10, warmup=3, tune=True, with_oracle=True):
    """The plain FP64 single-field solve (the rotating Gaussian of the parity case):
    GPU FP64 RK4 on all 16384 modes x 4000 steps, timed with CUDA events over
    `steps` solves after `warmup`; with_oracle: the FP64 oracle on the same
    potential (all modes), for the N and n(p) errors and the CPU time."""
    g = inputs.ROTATING_GAUSSIAN
    ns = g["n_steps"]
    dt = (g["t1"] - g["t0"]) / ns
    A = inputs.rotating_gaussian_potential(g, 2 * ns + 1)
    Ad = torch.tensor(A[None], device="cuda")
    tuned = None
    if tune:  # 16384 modes: the CTA size decides how many SMs get work
        chosen, cfg_ms, _ = pp.tune_pair_number(Ad, dt, g["grid"], precision="fp64", scheme="rk4")
        tuned = {"chosen": pp.launch_configs()[chosen], "ms": [round(x, 2) for x in cfg_ms]}
    for _ in range(warmup):
        pp.pair_number(Ad, dt, g["grid"], precision="fp64", scheme="rk4")
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(steps):
        N, n = pp.pair_number(Ad, dt, g["grid"], precision="fp64", scheme="rk4", want_n=True)
    e1.record(st)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / steps
    if pp.sync_status() != pp.PP_OK:
        raise RuntimeError("device status after the single-field solve")
    gr = g["grid"]
    modes = gr["nx"] * gr["ny"] * gr["nz"]
    flop = WORK[("fp64", "rk4")][0]
    achieved = flop * modes * ns / (ms * 1e-3) / 1e12
    rec = {"workload": g["name"], "precision": "fp64", "scheme": "rk4", "steps": steps, "warmup": warmup,
           "ms_per_solve": ms, "mode_steps_per_s": modes * ns / (ms * 1e-3), "N": N.item(),
           "roofline": {"bound": "alu", "kernel": "propagate_kernel<rk4, double>", "achieved": achieved,
                        "peak": peaks["fp64_tflops"], "unit": "TFLOP/s",
                        "frac": achieved / peaks["fp64_tflops"], "peak_source": peaks["fp64_source"],
                        **measured_peak(peaks, False, achieved),
                        "flop_per_mode_step": flop,
                        "note": "whole solve timed (table build, propagation, momentum sum)"},
           "launch_tuning": tuned, "clocks": clk,
           "l2": "not flushed: the solve is ALU-bound with a 0.5 MB working set"}
    if with_oracle:
        import oracle
        t0 = time.perf_counter()
        No, no = oracle.pair_number(A[None], ns, dt, g["grid"])
        cpu_s = time.perf_counter() - t0
        nn = n.cpu().numpy().reshape(-1)
        nov = no.reshape(-1)
        big = nov >= 1e-6 * nov.max()
        rec["N_oracle"] = float(No[0])
        rec["N_rel_err_vs_oracle"] = abs(N.item() / No[0] - 1)
        rec["n_max_rel_err_vs_oracle_where_n_ge_1e-6_max"] = float(np.abs(nn[big] / nov[big] - 1).max())
        rec["cpu_baseline"] = {"value": cpu_s * 1e3, "unit": "ms", "cores": oracle.num_threads(0),
                               "kind": "oracle", "sample": "the whole solve (all 16384 modes)"}
    return rec


def single_main(args):
    """--workload single: the config-1 solve as its own JSON line."""
    import torch
    import paper_1704_08919_gb300 as pp
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    pp.lib()
    rec = measure_single(pp, torch, local, device_peaks(local), steps=args.steps, warmup=args.warmup,
                         tune=not args.no_tune)
    ms = rec["ms_per_solve"]
    print(json.dumps(dict({
        "metric": "single-field FP64 solve time (rotating Gaussian, 16384 modes x 4000 RK4 steps)",
        "value": ms, "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": False, "scaling": "none", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (analytic field)", "config": {"workload": rec["workload"]}},
        **{k: v for k, v in rec.items() if k not in ("workload", "steps", "warmup")})), flush=True)
    return 0


def gemm_main(args):
    import torch
    import paper_1704_08919_gb300 as pp
    pp.lib()
    print(json.dumps({"metric": "pp_gemm_bf16 throughput", "gemm": gemm_measure(pp, torch)}),
          flush=True)
    return 0


def surrogate_main(args):
    """Surrogate-screened DE against plain DE on the de-batch solver settings: the
    network is trained on exact evaluations of random pulses, then both forms run
    from the same initial population; reports exact solver calls and wall-clock
    time to reach plain DE's best N, and the network's held-out error."""
    import torch
    import paper_1704_08919_gb300 as pp
    from paper_1704_08919_gb300 import screening as scr
    S = inputs.SURROGATE_DE
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    pp.lib()
    spec, grid = inputs.field_spec(CFG), CFG["grid"]
    K, D, NP = CFG["K"], 4 * CFG["K"], S["NP"]
    n_train = args.train or S["n_train"]
    G = args.generations or S["generations"]
    prec, sch = args.precision, args.scheme
    lo, hi, per = (torch.tensor(x, device="cuda") for x in inputs.param_bounds(K))
    clocks = ClockSampler(local)
    clocks.start()
    P_tr, N_tr, t_gen = scr.score_random(pp, n_train, spec, grid, S["train_seed"], precision=prec,
                                          scheme=sch)
    P_te, N_te, _ = scr.score_random(pp, S["n_heldout"], spec, grid, S["heldout_seed"],
                                     precision=prec, scheme=sch)
    lt = scr.LogTarget(N_tr)
    net = pp.Surrogate(D, S["hidden"], max_batch=max(S["R"] * NP, S["batch"], 1024))
    net.init(1)
    X_tr = pp.mlp_features(P_tr, lo, hi)
    t_tr = lt.targets(pp, N_tr)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = net.fit(X_tr, t_tr, S["batch"], S["epochs"], S["lr0"], S["lr1"])
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t0
    held = scr.held_out_error(pp, net, lt, P_te, N_te, lo, hi)
    de = dict(F=CFG["F"], CR=CFG["CR"], precision=prec, scheme=sch)
    modes = ["individual", "global"]
    per_seed = []
    for s_i in range(args.seeds):
        pop0 = torch.tensor(inputs.random_population(NP, K, seed=S["pop_seed"] + s_i), device="cuda")
        A0, _, _ = pp.synth_field(pop0, spec)
        fit0, _ = pp.pair_number(A0, spec["T"] / spec["n_steps"], grid, precision=prec, scheme=sch)
        seed = S["de_seed"] + s_i
        plain = scr.run_de(pp, pop0, fit0, spec, grid, G, seed, **de)
        target = plain["best"][-1]
        pc = scr.calls_to_reach(plain, target)
        rec = {"seed": seed, "plain": {"calls_to_best": pc, "best_N": target,
                                       "seconds_total": plain["seconds"],
                                       "seconds_to_best": plain["seconds"] * (pc // NP - 1) / G}}
        runs = {m: scr.run_de(pp, pop0, fit0, spec, grid, G, seed, net=net, R=S["R"], lt=lt,
                              mode=m, **de) for m in modes}
        if args.online:
            net_o = pp.Surrogate(D, S["hidden"], max_batch=net.max_batch)
            net_o.set_params(net.get_params())
            runs["individual_online"] = scr.run_de(pp, pop0, fit0, spec, grid, G, seed, net=net_o,
                                                   R=S["R"], lt=lt, online=(args.online, 4, 128, 2e-4),
                                                   **de)
        for m, r in runs.items():
            c = scr.calls_to_reach(r, target)
            rec[m] = {"calls_to_plain_best": c, "best_N": r["best"][-1],
                      "seconds_total": r["seconds"],
                      "seconds_to_plain_best": (r["seconds"] * (c // NP - 1) / G if c else None),
                      "gain_in_exact_calls": (pc / c) if c else 0.0}
        per_seed.append(rec)
    clk = clocks.stop()
    if pp.sync_status() != pp.PP_OK:
        raise RuntimeError("device status after the surrogate run")
    gains = {m: [r[m]["gain_in_exact_calls"] for r in per_seed] for m in per_seed[0] if m not in ("seed", "plain")}
    med = {m: statistics.median(v) for m, v in gains.items()}
    # exact calls saved per search (plain minus screened, to plain DE's best N) and the number of
    # searches after which the training evaluations have paid for themselves
    saved = {m: [r["plain"]["calls_to_best"] - r[m]["calls_to_plain_best"] for r in per_seed
                 if r[m]["calls_to_plain_best"]] for m in gains}
    break_even = {m: (n_train / statistics.median(v) if v and statistics.median(v) > 0 else None)
                  for m, v in saved.items()}
    print(json.dumps({
        "metric": "exact solver calls to reach plain-DE best N, plain / surrogate-screened "
                  "(median over seeds, %s screening)" % args.screen,
        "value": med[args.screen], "unit": "x", "n_gpus": 1, "steps": G, "warmup": 0,
        "higher_is_better": True, "scaling": "none", "vs_baseline": None,
        "dtype": "f32" if prec != "fp64" else "f64", "data": "synthetic (seeded B-spline pulses)",
        "config": {"workload": S["name"], "solver": workload_config(prec, NP, sch),
                   "R": S["R"], "n_train": n_train, "n_heldout": S["n_heldout"],
                   "epochs": S["epochs"], "batch": S["batch"], "generations": G,
                   "seeds": args.seeds},
        "gain_median": med, "gains": gains,
        "gain_range": {m: [min(v), max(v)] for m, v in gains.items()},
        "seeds_below_4x": {m: sum(1 for x in v if x < 4.0) for m, v in gains.items()},
        "exact_calls_saved_per_search": saved,
        "searches_to_repay_training": break_even,
        "training": {"pulses": n_train, "seconds_generate": t_gen, "seconds_fit": t_fit,
                     "final_epoch_loss": float(losses[-1].item())},
        "heldout": held, "per_seed": per_seed, "gemm": gemm_measure(pp, torch),
        "clocks": clk}), flush=True)
    return 0


def measure_de_batch_fp64(pp, torch, local, peaks, pop, fit, seed, gen, lo_t, hi_t, per_t, flush):
    """Config 2's FP64 arm: one DE generation of the 64-candidate batch through
    pp_de_step with FP64 RK4 propagation (the parity path), timed with CUDA events
    and the library's kernel timing; selection is against the population's current
    fitness.  The scored trials are rescored by the FP32-fast Magnus path for the
    FP64-vs-FP32 comparison."""
    spec, grid = inputs.field_spec(CFG), CFG["grid"]
    dt = CFG["T"] / CFG["n_steps"]
    NP = pop.shape[0]
    # warm-up: the FP64 kernel and its table on 4 candidates
    Aw, _, _ = pp.synth_field(pop[:4].contiguous(), spec)
    pp.pair_number(Aw, dt, grid, precision="fp64", scheme="rk4")
    trial = torch.empty_like(pop)
    tfit = torch.empty_like(fit)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    flush.zero_()
    pp.profile_begin()
    e0.record(stream)
    pp.de_step(pop, fit, spec, grid, lo_t, hi_t, per_t, CFG["F"], CFG["CR"], seed, gen, precision="fp64",
               scheme="rk4", trial_out=trial, trial_fit_out=tfit)
    e1.record(stream)
    torch.cuda.synchronize()
    kern_ms, launches = pp.profile_end()
    clk = clocks.stop()
    if pp.sync_status() != pp.PP_OK:
        raise RuntimeError("FP64 DE generation: device status")
    ms = e0.elapsed_time(e1)
    At, _, _ = pp.synth_field(trial, spec)
    Nf, _ = pp.pair_number(At, dt, grid, precision="fp32fast", scheme="magnus4")
    pp.sync_status()
    units = NP * units_per_candidate()
    flop = WORK[("fp64", "rk4")][0]
    per_launch = kern_ms / max(launches, 1)
    achieved = flop * units / (per_launch * 1e-3) / 1e12
    return {"workload": CFG["name"], "precision": "fp64", "scheme": "rk4", "generations": 1,
            "ms_per_generation": ms, "candidates_per_s": NP / (ms * 1e-3),
            "mode_steps_per_s": units / (ms * 1e-3),
            "fp32fast_magnus4_vs_fp64_rk4_max_rel_N_on_trials": (Nf / tfit - 1).abs().max().item(),
            "roofline": {"bound": "alu", "kernel": "propagate_kernel<rk4, double>", "achieved": achieved,
                         "peak": peaks["fp64_tflops"], "unit": "TFLOP/s",
                         "frac": achieved / peaks["fp64_tflops"], "peak_source": peaks["fp64_source"],
                         **measured_peak(peaks, False, achieved),
                         "flop_per_mode_step": flop, "launch_ms": per_launch,
                         "kernel_share_of_step": kern_ms / ms},
            "l2": "flushed before the generation (256 MiB write)",
            "note": "selection against the population's fitness from the FP32 run (within 1e-6 of FP64)",
            "clocks": clk, "gpu_launches": 7}


# ----------------------------------------------------------------------------- GPU leg


def main():
    args = parse()
    if args.impl == "reference":
        return reference_main(args)
    if args.workload == "uneven":
        return uneven_main(args)
    if args.workload == "surrogate":
        return surrogate_main(args)
    if args.workload == "gemm":
        return gemm_main(args)
    if args.workload == "localsearch":
        return localsearch_main(args)
    if args.workload == "large":
        return large_main(args)
    if args.workload == "single":
        return single_main(args)
    import torch
    import paper_1704_08919_gb300 as pp

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    pp.lib()
    stream = torch.cuda.current_stream()
    peaks = device_peaks(local)

    # One population of NP candidates per rank: at N = 1 the DE batch itself; at N > 1
    # one population of N * NP replicated on every rank, each rank scoring its NP
    # trials per generation and one allgather of the pair numbers (weak scaling).
    NP, K = args.ncand, CFG["K"]
    NP_total = NP * ws
    first, last = shard.shard_bounds(NP_total, ws, rank)
    spec = inputs.field_spec(CFG)
    grid = CFG["grid"]
    dt = CFG["T"] / CFG["n_steps"]
    lo, hi, per = inputs.param_bounds(K)
    pop_seed, seed = 1, 1000
    pop0 = inputs.random_population(NP_total, K, seed=pop_seed)
    lo_t, hi_t = torch.tensor(lo, device=dev), torch.tensor(hi, device=dev)
    per_t = torch.tensor(per, device=dev)
    pop = torch.tensor(pop0, device=dev)
    A, _, _ = pp.synth_field(pop[first:last].contiguous(), spec)
    tuned = None
    if not args.no_tune:
        chosen, cfg_ms, _ = pp.tune_pair_number(A, dt, grid, precision=args.precision,
                                                scheme=args.scheme)
        tuned = {"chosen": pp.launch_configs()[chosen], "ms": [round(x, 2) for x in cfg_ms],
                 "configs": pp.launch_configs()}
    fit_local, _ = pp.pair_number(A, dt, grid, precision=args.precision, scheme=args.scheme)
    gather = shard.allgather_fn(dist) if dist is not None else None
    fit = gather(fit_local, NP_total, ws) if gather else fit_local
    trial = torch.empty_like(pop)
    tfit = torch.empty_like(fit)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    if pp.sync_status() != pp.PP_OK:
        raise RuntimeError("initial scoring failed: %s" % pp.lib().pp_last_error().decode())
    sharded_steps = {}

    def generation(g, precision):
        """One DE generation of the population: pp_de_step at N = 1, the sharded
        generation (replicated proposal, local scoring, allgather, replicated
        selection) at N > 1."""
        if dist is None:
            pp.de_step(pop, fit, spec, grid, lo_t, hi_t, per_t, CFG["F"], CFG["CR"], seed, g,
                       precision=precision, trial_out=trial, trial_fit_out=tfit, scheme=args.scheme)
            return
        if precision not in sharded_steps:
            sharded_steps[precision] = shard.library_steps(pp, spec, grid, lo_t, hi_t, per_t, CFG["F"],
                                                           CFG["CR"], seed, precision, args.scheme)
        propose, score, select = sharded_steps[precision]
        shard.sharded_generation(propose, score, select, gather, pop, fit, g, rank, ws)

    gen = 0
    for _ in range(max(args.warmup, 0)):
        generation(gen, args.precision)
        gen += 1
    torch.cuda.synchronize()

    # ---- timed region: K generations, each bracketed by CUDA events, L2 flushed between
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    pp.profile_begin()
    t_wall = time.perf_counter()
    for s in range(args.steps):
        flush.zero_()
        starts[s].record(stream)
        generation(gen, args.precision)
        ends[s].record(stream)
        gen += 1
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    kern_ms, kern_launches = pp.profile_end()
    clk = clocks.stop()
    st = pp.sync_status()
    if st != pp.PP_OK:
        raise RuntimeError("device status %d after the timed region" % st)
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    replicas = None
    if dist is not None:
        # every rank must hold the same population and fitness after the sharded generations
        chk = float(torch.sum(pop).item() + torch.sum(fit).item())
        replicas = max_over_ranks(chk, dist, dev) == -max_over_ranks(-chk, dist, dev)
        if not replicas:
            raise RuntimeError("the ranks' populations diverged")
    ms_per_step = total_ms / args.steps
    cand_per_s = throughput(ws, NP, args.steps, total_ms)
    mode_steps_per_s = cand_per_s * units_per_candidate()

    # ---- live roofline of the propagation kernel
    per_launch_ms = kern_ms / max(kern_launches, 1)
    flop, inst = WORK[(args.precision, args.scheme)]
    units = (last - first) * units_per_candidate()
    achieved = flop * units / (per_launch_ms / 1000.0) / 1e12
    if args.precision in ("fp32", "fp32fast"):
        peak = peaks["fp32_tflops"]
        peak_src = peaks["fp32_source"]
        lanes = peaks["fp32_lanes_per_s"]
    else:
        peak = peaks["fp64_tflops"]
        peak_src = peaks["fp64_source"]
        lanes = peak * 1e12 / 2
    roofline = {"bound": "alu", "kernel": "propagate_kernel<%s, %s>" % (args.scheme, {
        "fp32": "float, compensated", "fp32fast": "float", "fp64": "double"}[args.precision]),
        "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
        "frac": achieved / peak, "peak_source": peak_src,
        **measured_peak(peaks, args.precision in ("fp32", "fp32fast"), achieved),
        "flop_per_mode_step": flop, "inst_per_mode_step": inst,
        "pipe_frac": inst * units / (per_launch_ms / 1000.0) / lanes,
        "launch_ms": per_launch_ms,
        "kernel_share_of_step": kern_ms / total_ms if ws == 1 else None,
        "traffic": (TRAFFIC_PER_CAND[(args.precision, args.scheme)] * NP
                    if (args.precision, args.scheme) in TRAFFIC_PER_CAND else None),
        "traffic_source": ("dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of this kernel "
                           "at 4 candidates (1.091 MB, nothing written), scaled by candidates: the "
                           "per-candidate step table is read from DRAM once, every other access hits L2"
                           if (args.precision, args.scheme) in TRAFFIC_PER_CAND else None)}

    # ---- accuracy at the bench config: N of the timed path vs FP64 RK4 (the oracle's
    # algorithm, parity-tested against it) on 4 candidates of the final population
    pcheck = pop[:4].clone()
    Acheck, _, _ = pp.synth_field(pcheck, spec)
    N32, _ = pp.pair_number(Acheck, dt, grid, precision=args.precision, scheme=args.scheme)
    N64, n64 = pp.pair_number(Acheck, dt, grid, precision="fp64", scheme="rk4", want_n=True)
    pp.sync_status()
    rel_err = (N32 / N64 - 1).abs().max().item()

    # ---- end to end through the public API with host buffers
    pop_h = torch.tensor(pop0, dtype=torch.float64).pin_memory()
    fit_h = fit.cpu().pin_memory()
    e2e_times = []
    for s in range(0 if args.no_e2e else args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pop.copy_(pop_h, non_blocking=True)
        fit.copy_(fit_h, non_blocking=True)
        generation(gen, args.precision)
        pop_h.copy_(pop, non_blocking=True)
        fit_h.copy_(fit, non_blocking=True)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
        gen += 1
    e2e_total = max_over_ranks(sum(e2e_times) if e2e_times else float("nan"), dist, dev)
    e2e_value = throughput(ws, NP, args.steps, 1000.0 * e2e_total)
    h2d = pop_h.numel() * 8 + fit_h.numel() * 8

    # ---- the compensated FP32 path on the same population, reported beside the main line
    alt = None
    if args.precision == "fp32fast" and args.alt_steps > 0:
        if not args.no_tune:
            pp.tune_pair_number(A, dt, grid, precision="fp32", scheme=args.scheme)
        for _ in range(2):
            generation(gen, "fp32")
            gen += 1
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.alt_steps)]
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            generation(gen, "fp32")
            b.record(stream)
            gen += 1
        torch.cuda.synchronize()
        alt_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), dist, dev)
        Nc, _ = pp.pair_number(Acheck, dt, grid, precision="fp32", scheme=args.scheme)
        pp.sync_status()
        alt = {"precision": "fp32 (compensated)",
               "value": throughput(ws, NP, args.alt_steps, alt_ms),
               "ms_per_step": alt_ms / args.alt_steps,
               "n_rel_err_vs_fp64_rk4_max": (Nc / N64 - 1).abs().max().item()}

    # ---- the FP64 oracle on one whole candidate (rank 0, N = 1 only): the metric's own
    # check (N of the timed path against the oracle's) and the CPU baseline.  The
    # oracle synthesises the candidate from its parameters itself.
    cpu = None
    oracle_check = None
    if rank == 0 and ws == 1 and not args.no_oracle_n:
        import oracle
        prm = pcheck[:1].cpu().numpy()
        Ao, _, _, orc = oracle.synth_field(prm, K, CFG["order"], CFG["w_min"], CFG["w_max"], CFG["T"],
                                           CFG["fluence"], CFG["n_steps"], want_E=False)
        t0 = time.perf_counter()
        No, no = oracle.pair_number(Ao, CFG["n_steps"], dt, grid)
        el = time.perf_counter() - t0
        cores = oracle.num_threads(0)
        n_gpu = n64[0].reshape(-1).cpu().numpy()
        nov = no.reshape(-1)
        big = nov >= 1e-6 * nov.max()
        oracle_check = {
            "candidate": "population row 0 after the timed generations (all %d modes x %d steps)"
                         % (units_per_candidate() // CFG["n_steps"], CFG["n_steps"]),
            "N_oracle": float(No[0]),
            "n_rel_err_vs_oracle": abs(N32[0].item() / No[0] - 1),
            "gpu_fp64_rk4_N_rel_err_vs_oracle": abs(N64[0].item() / No[0] - 1),
            "gpu_fp64_rk4_n_max_rel_err_where_n_ge_1e-6_max": float(np.abs(n_gpu[big] / nov[big] - 1).max()),
            "oracle_seconds": el, "oracle_cores": cores}
        if not args.no_cpu_baseline:
            cpu = {"value": 1.0 / el, "unit": "candidates/s", "cores": cores, "kind": "oracle",
                   "sample": "one whole candidate: %d modes x %d RK4 steps in FP64 (%.1f s); the "
                             "oracle's synthesis excluded" % (units_per_candidate() // CFG["n_steps"],
                                                              CFG["n_steps"], el),
                   "mode_steps_per_s": units_per_candidate() / el}
            A_host = Acheck.cpu().numpy()
            el1, _, _, _ = oracle_sample(A_host, 0, 256, seed=1, nthreads=1)
            cpu["one_core"] = {"mode_steps_per_s": 256 * CFG["n_steps"] / el1,
                               "value": 256 * CFG["n_steps"] / el1 / units_per_candidate(),
                               "sample": "256 strided modes x %d steps on one thread (%.2f s)" % (
                                   CFG["n_steps"], el1)}

    # ---- the other configurations, each with its own timing, clocks and roofline
    configs = None
    if rank == 0 and ws == 1 and not args.no_configs:
        configs = {"single_fp64": measure_single(pp, torch, local, peaks, tune=not args.no_tune),
                   "de_batch_fp64": measure_de_batch_fp64(pp, torch, local, peaks, pop, fit, seed, gen,
                                                          lo_t, hi_t, per_t, flush)}
        gen += 1
        configs["uneven"], _ = measure_uneven(pp, torch, local, peaks, 4, tune=not args.no_tune)

    if rel_err > 1e-4:
        raise RuntimeError("N error %.3e vs FP64 RK4 exceeds 1e-4: no valid measurement" % rel_err)
    if oracle_check and oracle_check["n_rel_err_vs_oracle"] > 1e-4:
        raise RuntimeError("N error %.3e vs the FP64 oracle exceeds 1e-4: no valid measurement"
                           % oracle_check["n_rel_err_vs_oracle"])
    if rank == 0:
        line = {
            "metric": "candidate pulses scored/s (DE batch, rel. N err <= 1e-4 vs FP64 oracle)",
            "value": cand_per_s, "unit": "candidates/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32",
            "scheme": args.scheme,
            "data": "synthetic (seeded B-spline pulses, uniform in bounds)",
            "config": dict(workload_config(args.precision, NP, args.scheme), **(
                {"population": NP_total,
                 "sharding": "one population of %d replicated on %d ranks; each rank scores its %d trials "
                             "per generation; one allgather of the %d pair numbers (NCCL) per generation"
                             % (NP_total, ws, NP, NP_total)} if ws > 1 else {})),
            "mode_steps_per_s": mode_steps_per_s,
            # a mode-step advances both spin channels of one momentum mode
            "mode_spin_steps_per_s": 2.0 * mode_steps_per_s,
            "n_rel_err_vs_fp64_rk4_max": rel_err,
            "n_rel_err_vs_oracle": oracle_check["n_rel_err_vs_oracle"] if oracle_check else None,
            "oracle_check": oracle_check,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "candidates/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": h2d},
            # per generation: proposal, spectrum, samples, table, propagation (+ its
            # wide-range twin for Magnus-4), partial sums, selection
            "gpu_launches": (8 if args.scheme == "magnus4" else 7) * args.steps,
            "replicas_identical": replicas,
            "launch_tuning": tuned,
            "alt_compensated": alt,
            "clocks": clk,
            "wall_s_timed": t_wall,
            "step_ms": step_ms,
            "peaks": {k: peaks[k] for k in ("sm_count", "sm_max_mhz", "fp32_tflops", "fp64_tflops",
                                            "fp32_measured_tflops", "fp64_measured_tflops")},
            "configs": configs,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
