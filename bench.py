"""Benchmark of the SPH timestep on the rotating square patch.

Default workload: 200^3 = 8,000,000 particles, FP32-mixed path, one step =
neighbour search + density/EOS + momentum/energy + Courant dt + update +
conserved sums.  Metric: pair interactions per second = sum_i |N(i)| x 2
pair phases (density, momentum) per step / time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mine|reference]

Prints one JSON line (rank 0).  Under torchrun each rank advances its own
replica of the patch (the path does not shard; replicas only) and the slowest
rank's time is used.  --impl reference times the FP64 CPU oracle, the
correctness authority, on host cores.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SPH pair-interactions/s & steps/s, 8M-particle patch, FP32-mixed vs FP64"
UNIT = "pair-interactions/s"
SMS = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
# FP32 operations per pair (FMA = 2, MUFU and min/max not counted), counted by
# hand from k_momentum_mixed and k_density_mixed.  Momentum: separation 9, r^2 5,
# r 2, q_i 2, w_j^2 and w_j q_j 3, F 7, v_ij 3, v.r 5, h sum 1, mu 6, Pi 7, g 1,
# (A_i + A_j + Pi) g 3, force terms 3, du term 5, sums 8 = 70
FLOPS_PER_PAIR_MOMENTUM = 70
FLOPS_PER_PAIR_DENSITY = 28
# the Sinc kernel (n = 6) in k_momentum_mixed: the Wendland count with its
# gradient shape (12) replaced by two sides of x = pi r w, S = sin x / x,
# S^5, g(x) and w^5 S^5 g (15 each) plus w_j^5 (3) and their sum (1)
FLOPS_PER_PAIR_MOMENTUM_SINC = 92
# the grad-h form: each side's gradient shape on its own (+2 for the Wendland
# kernel: w_j^5 and the sum; the Sinc count already has both) and the
# pressure terms 2 A_i f_i + 2 A_j f_j + Pi F and 2 A_i f_i + Pi F / 2 (+4)
FLOPS_PER_PAIR_MOMENTUM_GRADH = 76
FLOPS_PER_PAIR_MOMENTUM_SINC_GRADH = 96
# FP64 operations per pair of k_momentum_fp64 (mul/add each 1, sqrt and
# divisions not counted): 47 on every pair plus 17 for the viscosity of
# approaching pairs, taken on half of them
FLOPS_PER_PAIR_MOMENTUM_FP64 = 56
# Algorithmic bytes of the neighbour-list kernel (k_nb_thread): 4 B per list
# entry written, and per particle the row start (8 B), length (4 B) and own
# count (4 B) written plus its record (16 B), h (8 B), cell (4 B) and row hint
# (4 B) read once.
NB_BYTES_PER_ENTRY = 4
NB_BYTES_PER_PARTICLE = 48
# DRAM bytes (read + write) per list entry of one launch, from one-pass ncu
# captures of these kernels on the 200^3 patch itself (dram__bytes_read.sum +
# dram__bytes_write.sum divided by the launch's 8.54e8 list entries; see
# profiles/launches_square_patch_200cubed.md), scaled to the benchmark's
# launch by its entries.  None once the kernel has changed since; the
# momentum figure is that of its 2-lanes-per-particle instantiation, the
# search's that of both its 2- and 3-cell stencils (5.70 B each).
NB_DRAM_BYTES_PER_ENTRY = 5.70
MOMENTUM_DRAM_BYTES_PER_ENTRY = 7.88
MOMENTUM_DRAM_TPP = 2

WORKLOADS = {
    "c1": ("square patch 20^3 (8,000 particles), omega=5", 20),
    "c2": ("square patch 100^3 (1,000,000 particles), omega=5", 100),
    "c3": ("square patch 200^3 (8,000,000 particles), omega=5", 200),
    "c4": ("64 independent square patches, edges 10..60, omega 2..8 (seed 0), one launch per phase", None),
    "c5": ("irregular patch 159^3 (4,019,679 particles): jittered lattice, log-normal masses, "
           "neighbour counts 50-400", 159),
}


def rank_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def reduce_over_ranks(ms, pairs, device):
    """Replicas (one independent patch per rank, no data-path collective):
    the job's time is the slowest rank's, its pairs every rank's."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    p = torch.tensor([float(pairs)], dtype=torch.float64, device=device)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t.item()), float(p.item())


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": SM_MAX_MHZ}, "fallback"


class Clocks:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_kw(args):
    """The oracle's kernel and momentum form for the bench's options."""
    return {"kernel": args.kernel, "kernel_n": 6, "grad_h": bool(args.grad_h)}


def oracle_sample(args, threads, n_edge, warmup=3, nsteps=None, min_seconds=10.0, max_steps=None):
    """The FP64 oracle (as it stands) on the n_edge^3 square patch, stepped
    with the timestep of the benchmarked patch: the first Courant step
    C min(h/c) taken with the full-size patch's h (dt follows h), held fixed.
    The sample's steps then cover the same stretch of the flow as the
    full-size steps (with its own Courant step a smaller patch would run ahead
    in time, into states where the oracle's uniform grid, sized by the largest
    h, is slower).  After `warmup` untimed steps, times `nsteps` steps, or as
    many as fill `min_seconds` (at most `max_steps`).  Returns (pairs,
    seconds, steps, n_edge, dt)."""
    import numpy as np
    import oracle
    from paper_1905_03344_gb300 import inputs
    full = WORKLOADS[args.config][1] or 200
    n_edge = min(n_edge, full)
    f = inputs.square_patch(n_edge)
    gamma = inputs.GAMMA
    # c = sqrt(gamma P / rho) with P = (gamma - 1) rho u, and h = eta L / n
    cmax = float(np.sqrt(gamma * (gamma - 1.0) * f["u"]).max())
    dt = 0.2 * inputs.ETA / full / cmax
    sim = oracle.Sim(f, nthreads=threads, dt_fixed=dt, **oracle_kw(args))
    for _ in range(warmup):
        sim.step(1)
    t0 = time.perf_counter()
    pairs = 0
    k = 0
    while True:
        sim.step(1)
        pairs += sim.nnz
        k += 1
        el = time.perf_counter() - t0
        if nsteps is not None:
            if k >= nsteps:
                return pairs, el, k, n_edge, dt
        elif el >= min_seconds or (max_steps is not None and k >= max_steps):
            return pairs, el, k, n_edge, dt


def cpu_baseline_1thread(args, sample_n=40):
    """The same oracle steps on one host core, on the 40^3 patch."""
    pairs, dt, k, ne, step_dt = oracle_sample(args, 1, sample_n, min_seconds=5.0, max_steps=max(args.steps, 1))
    return {"value": 2.0 * pairs / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d full oracle steps on the %d^3 square patch (%d particles) after 3 warm-up steps, "
                      "dt = %.3g (the full-size patch's Courant step), one host core; %.1f s"
                      % (k, ne, ne ** 3, step_dt, dt)}


def cpu_baseline(args, sample_n=100):
    """The FP64 oracle (as it stands) on all host cores: full steps on the
    100^3 patch, the same rotating-patch workload at 1/8 of the particles."""
    threads = os.cpu_count() or 1
    pairs, dt, k, ne, step_dt = oracle_sample(args, threads, sample_n, max_steps=max(args.steps, 1))
    return {"value": 2.0 * pairs / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d full oracle steps (neighbours..update) on the %d^3 square patch (%d particles) "
                      "after 3 warm-up steps, dt = %.3g (the full-size patch's Courant step), OpenMP on "
                      "all host cores; %.1f s" % (k, ne, ne ** 3, step_dt, dt)}


def run_reference(args):
    rank, world, _ = rank_info()
    if rank != 0:
        return 0
    threads = os.cpu_count() or 1
    pairs, el, k, n_edge, step_dt = oracle_sample(args, threads, 50, warmup=args.warmup, nsteps=args.steps)
    val = 2.0 * pairs / el
    wl = WORKLOADS[args.config][0]
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl, "precision": "fp64 (CPU oracle)", "kernel": args.kernel,
                   "grad_h": bool(args.grad_h),
                   "sample": "%d^3 square patch per step" % n_edge},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "each step: one full FP64 oracle step on the %d^3 square patch "
                                   "(%d particles) with the %s workload's Courant step (dt = %.3g), "
                                   "so the steps span the same stretch of the flow"
                                   % (n_edge, n_edge ** 3, args.config, step_dt)},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--config", default="c3", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=-1,
                    help="steps of the end-to-end leg (-1: as many as the timed steps; 0: skip)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--kernel", default="wendland", choices=["wendland", "sinc"],
                    help="SPH kernel of Sec. 3 (Sinc with n = 6)")
    ap.add_argument("--pair-mode", default="auto", choices=["auto", "lists", "fused"],
                    help="pair sums over neighbour lists, list-free (the search inside the sums), "
                         "or whichever the autotuner finds faster")
    ap.add_argument("--adapt-h", type=int, choices=[0, 1], default=None,
                    help="h adaptation (default: on, off for c5, which is timed with h frozen)")
    ap.add_argument("--skin", type=float, default=0.0,
                    help="reuse the neighbour search across steps: search radius scaled by 1 + skin, "
                         "exact lists filtered from it every step (0: search every step)")
    ap.add_argument("--mode-steps", type=int, default=10,
                    help="steps timed for the pair mode not chosen (0: skip)")
    ap.add_argument("--grad-h", action="store_true",
                    help="the grad-h momentum and energy form (Omega factors)")
    ap.add_argument("--cell-factor", type=float, default=0.0,
                    help="fixed cell factor (implies --no-autotune); 0 = tuned")
    ap.add_argument("--tpp", type=int, default=0,
                    help="fixed lanes per particle of the pair sums (implies --no-autotune); 0 = tuned")
    ap.add_argument("--pair-bins", type=int, default=0,
                    help="row-length bins of the pair sums, list words per lane (8..256; -1: never; "
                         "0: the autotuner decides)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.cell_factor or args.tpp:
        args.no_autotune = True
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank, world, local = rank_info()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_1905_03344_gb300 import binding, build, inputs
    build.build()
    wl, n_edge = WORKLOADS[args.config]
    offsets = None
    if args.config == "c4":
        f, offsets, _, _ = inputs.batch_patches(64, seed=0)
    elif args.config == "c5":
        f = inputs.irregular_patch(159)
    else:
        f = inputs.square_patch(n_edge)
    adapt = args.adapt_h if args.adapt_h is not None else (0 if args.config == "c5" else 1)
    n = len(f["x"])
    stream = torch.cuda.current_stream()
    dfields = {k: torch.tensor(v, dtype=torch.float64, device=dev) for k, v in f.items()}

    def make(precision, graph=False, **over):
        kw = {"kernel": args.kernel, "kernel_n": 6, "grad_h": int(args.grad_h), "pair_mode": args.pair_mode,
              "list_skin": args.skin, "adapt_h": adapt}
        if args.cell_factor:
            kw["cell_factor"] = args.cell_factor
        if args.tpp:
            kw["threads_per_particle"] = args.tpp
        if args.pair_bins:
            kw["pair_bins"] = args.pair_bins
        kw.update(over)
        sim = binding.SPH(n, precision=precision, stream=stream.cuda_stream, use_graph=int(graph),
                          max_pairs=int(160 * n), max_patches=64 if offsets is not None else 1, **kw)
        sim.set_particles(dfields)
        if offsets is not None:
            sim.set_patches(offsets)
        return sim

    # FMA rate of this GPU in the path's precision (0.3 s, before anything is timed)
    fma_peak = binding.sph_fma_peak("fp64" if args.precision == "fp64" else "mixed",
                                    stream=stream.cuda_stream) / 1e12

    sim = make(args.precision, True)
    for _ in range(args.warmup):
        sim.step(1)
    if not args.no_autotune:
        # tune on the warmed-up state (h adapted); the physical state is unchanged
        sim.autotune()
        sim.step(1)
    tpp, cf = binding.sph_get_tuning(sim.ctx)
    tpp_den = binding.sph_get_density_tpp(sim.ctx)
    bins_den, bins_mom = sim.pair_bins()
    mode = sim.pair_mode()
    torch.cuda.synchronize()
    # the state at the start of the timed steps, on the host: the graph
    # replay and the end-to-end leg below run the same stretch of steps from it
    e2e_blob = torch.empty(sim.state_bytes(), dtype=torch.uint8).pin_memory()
    sim.get_state(e2e_blob)
    sim.pair_count(reset=True)
    # the timed region runs the phases with CUDA events between them (per-kernel
    # durations for the roofline); the graph is bypassed while profiling
    sim.profile(True)
    sim.profile()      # reset accumulators
    clocks = Clocks(local)
    l0 = sim.launches()
    rb0 = sim.list_rebuilds()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        sim.step(1)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    ms_total = e0.elapsed_time(e1)
    launches = sim.launches() - l0
    rebuilds = sim.list_rebuilds() - rb0
    pairs = sim.pair_count(reset=True)
    prof = sim.profile()
    cf_end = binding.sph_get_tuning(sim.ctx)[1]
    sim.profile(False)

    # the same stretch of steps replayed from captured CUDA graphs: back to
    # the state at the start of the timed region, three untimed steps (the
    # first after a restore is launched directly, the next two capture the
    # graph of each buffer parity), then K replayed steps
    sim.set_state(e2e_blob)
    for _ in range(3):
        sim.step(1)
    torch.cuda.synchronize()
    sim.pair_count(reset=True)
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(args.steps):
        sim.step(1)
    g1.record(stream)
    torch.cuda.synchronize()
    ms_graph = g0.elapsed_time(g1)
    pairs_graph = sim.pair_count(reset=True)
    if world > 1:
        ms_total, pairs_all = reduce_over_ranks(ms_total, pairs, dev)
    else:
        pairs_all = float(pairs)
    sec = ms_total / 1e3
    value = 2.0 * pairs_all / sec
    steps_per_s = args.steps / sec
    pairs_per_step = pairs / args.steps

    peaks, peak_src = measured_peaks()
    sm_max = peaks.get("sm_max_mhz") or SM_MAX_MHZ
    fp32_peak = SMS * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    mom_ms = prof["momentum"][0] / max(args.steps, 1)
    flops_pair = {(False, False): FLOPS_PER_PAIR_MOMENTUM, (True, False): FLOPS_PER_PAIR_MOMENTUM_SINC,
                  (False, True): FLOPS_PER_PAIR_MOMENTUM_GRADH,
                  (True, True): FLOPS_PER_PAIR_MOMENTUM_SINC_GRADH}[(args.kernel == "sinc", args.grad_h)]
    prec_tag = "mixed" if args.precision == "mixed" else "fp64"
    pair_peak = fp32_peak
    pair_peak_src = "derived: %d SMs x %d FP32 lanes x 2 x %.0f MHz (max SM clock)" % (SMS, FP32_LANES_PER_SM, sm_max)
    if args.precision == "fp64":
        # the FP64 pair sums run on the FP64 pipe: their own operation count
        # (the Wendland form; no count is kept for the others) against the
        # measured FP64 FMA rate
        flops_pair = FLOPS_PER_PAIR_MOMENTUM_FP64 if args.kernel == "wendland" and not args.grad_h else None
        pair_peak = fma_peak
        pair_peak_src = "measured: sph_fma_peak FP64 FMA chains"
    mom_tf = flops_pair * pairs_per_step / (mom_ms / 1e3) / 1e12 if flops_pair else None
    if mode == "lists":
        # dominant kernel: the neighbour-list search (k_nb_thread), HBM roofline
        # on its algorithmic bytes
        nb_ms = prof["nb"][0] / max(args.steps, 1)
        nb_bytes = NB_BYTES_PER_ENTRY * pairs_per_step + NB_BYTES_PER_PARTICLE * n
        nb_gbs = nb_bytes / (nb_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": "k_nb_thread", "achieved": nb_gbs, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": nb_gbs / peaks["hbm_gbs"],
                "traffic": (NB_DRAM_BYTES_PER_ENTRY * pairs_per_step) if NB_DRAM_BYTES_PER_ENTRY else None,
                "algorithmic_bytes": nb_bytes, "ms_per_launch": nb_ms,
                "peak_source": "%s hbm_gbs (MEASURED_PEAKS.json)" % peak_src,
                "share_of_step": prof["nb"][0] / ms_total}
    else:
        # list-free: the momentum pass (search + pair sums) dominates; its pair
        # arithmetic against the FP32 peak (the search is not counted)
        roof = {"bound": "alu", "kernel": "k_fused_momentum_" + prec_tag, "achieved": mom_tf,
                "peak": pair_peak, "unit": "TFLOP/s", "frac": mom_tf and mom_tf / pair_peak, "traffic": None,
                "flops_per_pair": flops_pair, "ms_per_launch": mom_ms, "peak_source": pair_peak_src,
                "share_of_step": prof["momentum"][0] / ms_total}
    # the pair sums: FP32 pipe (mixed) against the derived FP32 peak, FP64
    # pipe (FP64 path) against the measured FP64 FMA rate
    roof_mom = {"bound": "alu", "kernel": ("k_momentum_" if mode == "lists" else "k_fused_momentum_") + prec_tag,
                "achieved": mom_tf, "peak": pair_peak, "unit": "TFLOP/s", "frac": mom_tf and mom_tf / pair_peak,
                # the DRAM figure is the standard Wendland variant's
                "traffic": (MOMENTUM_DRAM_BYTES_PER_ENTRY * pairs_per_step)
                if MOMENTUM_DRAM_BYTES_PER_ENTRY and args.kernel == "wendland" and not args.grad_h
                and mode == "lists" and args.precision == "mixed" and tpp == MOMENTUM_DRAM_TPP else None,
                "peak_source": pair_peak_src,
                "peak_fma_measured": fma_peak, "frac_of_fma_measured": mom_tf and mom_tf / fma_peak,
                "flops_per_pair": flops_pair, "ms_per_launch": mom_ms,
                "share_of_step": prof["momentum"][0] / ms_total}
    if clk.get("sm_mhz") and mom_tf and args.precision == "mixed":
        roof_mom["frac_at_sampled_clock"] = mom_tf / (fp32_peak * clk["sm_mhz"] / sm_max)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32-mixed (f32 pair sums + Kahan, f64 positions/integration/reductions)"
        if args.precision == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": wl, "particles": n, "precision": args.precision, "kernel": args.kernel,
                   "adapt_h": bool(adapt),
                   "grad_h": bool(args.grad_h),
                   "parallelism": "replicas x%d" % world if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (%.1f GB of particle fields and neighbour lists)"
                         % ((n * 13 * 8 * 2 + pairs_per_step * 4) / 1e9),
                   "threads_per_particle": tpp, "threads_per_particle_density": tpp_den,
                   "row_length_bins": {"density_words_per_lane": bins_den, "momentum_words_per_lane": bins_mom,
                                       "note": "0: uniform lanes per particle"},
                   "cell_factor": cf, "cell_factor_end": cf_end, "pair_mode": mode,
                   "list_skin": args.skin, "searches_in_timed_steps": rebuilds if args.skin > 0 else args.steps,
                   "timed": "K steps with CUDA events between phases (no graph)"},
        "steps_per_s": steps_per_s, "pairs_per_step": pairs_per_step,
        "gpu_launches": launches, "clocks": clk,
        "phase_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "roofline": roof, "roofline_pair_sum": roof_mom,
        "graph_replay": {"value": 2.0 * pairs_graph / (ms_graph / 1e3), "unit": UNIT,
                         "ms_per_step": ms_graph / args.steps, "steps_per_s": 1e3 * args.steps / ms_graph,
                         "steps": args.steps,
                         "stretch": "the timed region's steps, from its saved start state, shifted by 3"},
    }

    # the other pair mode at the same cell factor (and lanes per particle)
    if args.mode_steps > 0 and world == 1:
        other = "fused" if mode == "lists" else "lists"
        # a second context beside the tuned one (both fit in HBM)
        so = make(args.precision, pair_mode=other, cell_factor=cf, threads_per_particle=tpp)
        for _ in range(args.warmup):
            so.step(1)
        torch.cuda.synchronize()
        so.pair_count(reset=True)
        so.profile(True)
        so.profile()
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for _ in range(args.mode_steps):
            so.step(1)
        b1.record(stream)
        torch.cuda.synchronize()
        mso = b0.elapsed_time(b1) / args.mode_steps
        po = so.pair_count(reset=True) / args.mode_steps
        profo = so.profile()
        so.profile(False)
        so.close()
        line["other_pair_mode"] = {"pair_mode": other, "value": 2.0 * po / (mso / 1e3), "unit": UNIT,
                                   "ms_per_step": mso, "steps": args.mode_steps, "cell_factor": cf,
                                   "threads_per_particle": tpp,
                                   "phase_ms_per_step": {k: v[0] / args.mode_steps for k, v in profo.items()}}

    # FP64 GPU path on the same patch
    if args.fp64_steps > 0 and args.precision == "mixed":
        sim.close()
        s64 = make("fp64")
        for _ in range(args.warmup):
            s64.step(1)
        if not args.no_autotune:
            s64.autotune()
        torch.cuda.synchronize()
        s64.pair_count(reset=True)
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(args.fp64_steps):
            s64.step(1)
        a1.record(stream)
        torch.cuda.synchronize()
        ms64 = a0.elapsed_time(a1) / args.fp64_steps
        p64 = s64.pair_count(reset=True) / args.fp64_steps
        line["fp64_path"] = {"value": 2.0 * p64 / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64,
                             "steps_per_s": 1e3 / ms64, "steps": args.fp64_steps}
        # the FP64 path's momentum sum against the FP64 FMA rate
        s64.profile(True)
        s64.profile()
        s64.step(1)
        torch.cuda.synchronize()
        prof64 = s64.profile()
        s64.profile(False)
        fma64 = binding.sph_fma_peak("fp64", stream=stream.cuda_stream) / 1e12
        mom64_ms = prof64["momentum"][0]
        mom64_tf = FLOPS_PER_PAIR_MOMENTUM_FP64 * p64 / (mom64_ms / 1e3) / 1e12
        line["fp64_path"]["roofline_pair_sum"] = {
            "bound": "alu", "kernel": "k_momentum_fp64", "achieved": mom64_tf, "peak": fma64, "unit": "TFLOP/s",
            "frac": mom64_tf / fma64, "peak_source": "measured: sph_fma_peak FP64 FMA chains",
            "flops_per_pair": FLOPS_PER_PAIR_MOMENTUM_FP64, "ms_per_launch": mom64_ms}
        line["mixed_over_fp64"] = line["ms_per_step"] and ms64 / line["ms_per_step"]
        s64.close()
        sim = make(args.precision)
        for _ in range(args.warmup):
            sim.step(1)
        if not args.no_autotune:
            sim.autotune()

    # end to end through the C ABI with host (pinned) buffers: every step
    # uploads the whole time state from host memory (sph_set_state: fields,
    # permutation, dt state), takes one step and reads the whole new state
    # back (sph_get_state), which the next step uploads.  Starting from the
    # state saved at the start of the timed region, these are the same steps
    # as the timed ones (all K of them by default).
    if args.e2e_steps != 0:
        ne2e = args.steps if args.e2e_steps < 0 else args.e2e_steps
        nbytes = e2e_blob.numel()
        sim.set_state(e2e_blob)
        sim.step(1)                 # untimed: the launch shape's graph and rows for this order
        sim.set_state(e2e_blob)
        sim.pair_count(reset=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ne2e):
            sim.set_state(e2e_blob)
            sim.step(1)
            sim.get_state(e2e_blob)
        el = time.perf_counter() - t0
        pe = sim.pair_count(reset=True)
        line["e2e"] = {"value": 2.0 * pe / el, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                       "d2h_bytes_per_step": nbytes, "steps": ne2e, "ms_per_step": 1e3 * el / ne2e,
                       "call": "per step: sph_set_state(pinned host state) + sph_step(1) + "
                               "sph_get_state(pinned host state): all 13 particle fields, the "
                               "permutation and the dt state in and out; the timed region's steps"}
    sim.close()

    # the oracle baseline is of the square patch (c1-c3)
    if rank == 0 and world == 1 and not args.no_cpu and args.config in ("c1", "c2", "c3"):
        line["cpu_baseline"] = cpu_baseline(args)
        line["cpu_baseline_1core"] = cpu_baseline_1thread(args)
        try:
            cpu = [l.split(":", 1)[1].strip() for l in open("/proc/cpuinfo") if l.lower().startswith(("model name", "cpu part"))]
        except OSError:
            cpu = []
        line["cpu_baseline"]["host"] = {"nproc": os.cpu_count(), "cpu": cpu[0] if cpu else "unknown"}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
