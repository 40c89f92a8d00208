"""Benchmark: M-rPIE pattern-updates/s on the 256x256, 5-mode Fermat-spiral
scan (10^4 positions, 2800x2800 object), one GPU per rank.

A step is one full iteration over all positions through the C ABI
(libpty.so).  Prints ONE JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                    [--impl ours|reference] [--no-cpu-baseline]

--impl reference times the FP64 CPU oracle (the only baseline that exists
for this method) on a bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rPIE pattern-updates/s at 256^2 with 5 modes"
UNIT = "pattern-updates/s"


def workloads():
    from paper_2205_04295_b300 import synth
    return {
        "spiral_256": lambda: synth.spiral_256(),
        "spiral_256_n2000": lambda: synth.spiral_256(n=2000),
        # 2000 positions over the 10^4-position spiral's extent: groups of its size
        "spiral_256_n2000_spread5": lambda: synth.spiral_256(n=2000, spread=5.0),
        "plain_64": lambda: synth.plain_rpie_64(),
        "refine_128": lambda: synth.refine_128(),
        "sweep_256": lambda: synth.sweep_256(),
    }


def algorithmic(W, M):
    """Algorithmic flops and HBM bytes of one pattern update (no registration).

    flops: 2M unitary 2-D DFTs at 5 n log2 n each (n = W^2) plus about
    (30 M + 20) W^2 for the exit waves, constraint and both updates.
    bytes: the pattern (2 B/px) + reading and writing the crop (8 + 8 B/px);
    probe traffic is shared by a whole group and far-field waves stay on chip.
    """
    import math
    n = W * W
    fft = 5.0 * n * math.log2(n)
    return 2 * M * fft + (30 * M + 20) * n, 18.0 * n


def per_pass_flops(W, M):
    """Algorithmic flops per pattern update of each pass (and of the fused
    patch kernel, which does all three)."""
    import math
    lw = math.log2(W)
    row = 5.0 * W * W * lw          # W row DFTs of length W
    f = {"rows_fwd": M * row + 6 * M * W * W,
         "cols": 2 * M * row + (4 * M + 10) * W * W,
         "rows_inv": M * row + (24 * M + 10) * W * W}
    f["patch"] = f["rows_fwd"] + f["cols"] + f["rows_inv"]
    return f


# DRAM bytes per pattern update of each pass, warm L2: ncu
# dram__bytes_read.sum + dram__bytes_write.sum with --cache-control none on
# `bench.py` (the 256^2 / 5-mode spiral of 10^4 positions; launches 81-120 of the
# three passes and the probe update: groups 20-29, 674 patches).  A group's
# far field (about 67 patches x 2.62 MB) is larger than L2, so most of it
# goes to HBM and back between the passes.  Valid for the pass kernels as
# profiled; a launch's traffic is this times its patches.
DRAM_PER_PATCH = {(256, 5): {"rows_fwd": 2.648e6, "cols": 4.018e6, "rows_inv": 3.741e6}}


def fp32_peak_tflops():
    """148 SMs x 128 FP32 lanes x 2 flop (FMA) x 2032 MHz maximum SM clock."""
    return 148 * 128 * 2 * 2.032e9 / 1e12


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out, _ = self.p.communicate()

    def summary(self):
        rows = [r.split(",") for r in (self.out or "").strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for i, nm in enumerate(names):
                if r[5 + i].strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


def dist_setup(n_gpus, backend=None):
    """Rank, world size and local rank from the launcher's environment; for a
    world > 1 the process group (nccl on GPUs, gloo otherwise).  Replicas
    only: the group carries the barrier and the max-over-ranks of the timing,
    never data of the reconstruction."""
    import torch
    import torch.distributed as dist
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def batch_shard(costs, rank, world):
    """Problems of the batched workload that `rank` runs: longest processing
    time first onto the least-loaded rank (ties to the lower rank), so every
    rank gets a near-equal share of the work and each problem runs on exactly
    one rank.  `costs` is any per-problem work estimate."""
    load = [0.0] * world
    mine = []
    for p in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += costs[p]
        if r == rank:
            mine.append(p)
    return sorted(mine)


def problem_cost(wl):
    """Work of one M-rPIE iteration of a problem, in flops (2M 2-D DFTs per patch)."""
    import math
    return wl.N * wl.M * wl.W * wl.W * math.log2(wl.W * wl.W)


def replica_rate(units_per_rank, seconds_per_rank, world):
    """Whole-job throughput of `world` independent replicas: all units over
    the slowest rank's time (weak scaling)."""
    return world * units_per_rank / max_over_ranks(seconds_per_rank, world)


# ------------------------------------------------------------------ oracle
def oracle_sample(wl, d_host, budget_s):
    """Time the FP64 oracle on whole groups of the workload until the budget
    is spent; returns (pattern-updates/s, patches, seconds, groups)."""
    import numpy as np
    from oracle import grouping, model, rpie
    groups = grouping.greedy_groups(d_host["pos"].astype(np.float64), wl.W)
    st = rpie.State.create(d_host["O0"], d_host["P0"], d_host["pos"])
    corners = model.crop_corners(d_host["pos"])
    prm = rpie.RPIEParams()
    done, t0, ng = 0, time.perf_counter(), 0
    for g in groups:
        rpie.rpie_group(st.O, st.P, d_host["I"], corners, g, prm)
        done += len(g)
        ng += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return done / dt, done, dt, ng


def host_inputs_for_groups(wl, n_groups):
    """Host inputs with the counts of the first n_groups simulated on the CPU."""
    import numpy as np
    from oracle import grouping
    from paper_2205_04295_b300 import synth
    groups = grouping.greedy_groups(wl.pos.astype(np.float64), wl.W)
    sel = np.concatenate(groups[:n_groups])
    rng = np.random.Generator(np.random.PCG64(wl.seed))
    O = synth.make_object(wl.Hy, wl.Hx, rng)
    P = synth.make_probe(wl.W, wl.M, wl.photons, wl.occupancy)
    cnt, _ = synth.simulate_counts(O, P, wl.pos_true[sel], wl.seed)
    I = np.zeros((wl.N, wl.W, wl.W), np.uint16)
    I[sel] = cnt.numpy().astype(np.uint16)
    return {"I": I, "pos": wl.pos.astype(np.float32), "O0": np.ones((wl.Hy, wl.Hx), np.complex64),
            "P0": synth.initial_probe(P)}


def _oracle_worker(d, groups, budget_s, start, q):
    """One process of the all-core oracle figure: its own copy of the state,
    whole groups of the selected patterns in order (cycling), timed after every
    process is ready."""
    single_thread_env()
    from oracle import rpie
    st = rpie.State.create(d["O0"], d["P0"], d["pos"])
    prm = rpie.RPIEParams()
    start.wait()
    done, t0, i = 0, time.perf_counter(), 0
    while time.perf_counter() - t0 < budget_s:
        g = groups[i % len(groups)]
        rpie.rpie_group(st.O, st.P, d["I"], d["corners"], g, prm)
        done += len(g)
        i += 1
    q.put((done, time.perf_counter() - t0))


def oracle_all_cores(wl, nproc, budget_s, n_groups=8):
    """Aggregate oracle throughput of `nproc` concurrent FP64 processes, each
    running the oracle unchanged on its own copy of the state over the first
    n_groups whole groups (a bound on what splitting the work across processes
    could reach: the groups of one iteration depend on each other)."""
    import multiprocessing as mp
    import numpy as np
    from oracle import grouping, model
    d = host_inputs_for_groups(wl, n_groups)
    groups = grouping.greedy_groups(d["pos"].astype(np.float64), wl.W)[:n_groups]
    sel = np.concatenate(groups)
    local = np.empty(wl.N, np.int64)
    local[sel] = np.arange(len(sel))
    dd = {"I": d["I"][sel], "corners": model.crop_corners(d["pos"])[sel], "pos": d["pos"],
          "O0": d["O0"], "P0": d["P0"]}
    lg = [local[g] for g in groups]
    ctx = mp.get_context("spawn")
    start, q = ctx.Barrier(nproc), ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(dd, lg, budget_s, start, q)) for _ in range(nproc)]
    for p in ps:
        p.start()
    res = [q.get() for _ in ps]
    for p in ps:
        p.join()
    patches = sum(r[0] for r in res)
    return {"value": sum(r[0] / r[1] for r in res), "unit": UNIT, "cores": nproc, "kind": "oracle",
            "sample": "%d concurrent FP64 processes, each on its own copy of the state over the "
                      "first %d groups (%d patches in all, %.1f s each)"
                      % (nproc, n_groups, patches, budget_s)}


def single_thread_env():
    for v in ("OMP_NUM_THREADS", "MKL_NUM_THREADS", "OPENBLAS_NUM_THREADS"):
        os.environ.setdefault(v, "1")


def run_reference(args, wl):
    """--impl reference: the FP64 oracle on the host cores."""
    single_thread_env()
    d = host_inputs_for_groups(wl, 12)
    per_step = max(2.0, 20.0 / max(1, args.steps))
    for _ in range(min(args.warmup, 1)):
        oracle_sample(wl, d, 0.5)
    rates, patches, secs = [], 0, 0.0
    for _ in range(args.steps):
        r, n, dt, ng = oracle_sample(wl, d, per_step)
        rates.append(r)
        patches += n
        secs += dt
    value = patches / secs
    sample = ("first whole groups of the greedy schedule per step (%d patches in %.1f s over %d steps)"
              % (patches, secs, args.steps))
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * wl.N / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": wl.name, "W": wl.W, "M": wl.M, "N": wl.N, "object": [wl.Hy, wl.Hx]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            **({"cpu_all_cores": oracle_all_cores(wl, args.oracle_procs, per_step)}
               if args.oracle_procs > 0 else {})}


# --------------------------------------------------------------------- ours
def run_ours(args, wl, rank, world, local):
    import numpy as np
    import torch
    from paper_2205_04295_b300 import pty, synth

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    d = synth.build(wl, device=dev)
    I_dev = synth.counts_u16(d["I"])
    pos_dev = torch.from_numpy(d["pos"]).to(dev)
    O0_dev = torch.from_numpy(d["O0"]).to(dev)
    P0_dev = torch.from_numpy(d["P0"]).to(dev)
    prm = pty.rpie_params()

    prob = pty.Problem(wl.W, wl.M, wl.N, wl.Hy, wl.Hx, stream=stream)
    prob.set_data(I_dev, pos_dev, O0_dev, P0_dev)
    from paper_2205_04295_b300 import autotune
    tiling = autotune.apply(prob)
    n_groups = len(prob.groups())

    # ---- device-resident timing (inputs already in HBM)
    for _ in range(args.warmup):
        prob.run(1, prm, errors=False)
    prob.profile(1)
    prob.run(1, prm, errors=False)
    prob.stats(reset=True)
    prob.profile(0)
    torch.cuda.synchronize()
    barrier(world)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        start.record(stream)
        prob.run(args.steps, prm, errors=False)
        stop.record(stream)
        torch.cuda.synchronize()
    ms = start.elapsed_time(stop)
    barrier(world)
    st = prob.stats(reset=True)
    value = replica_rate(wl.N * args.steps, ms / 1e3, world)
    ms = max_over_ranks(ms, world)
    launches = sum(st["launches"].values())

    # ---- the same step with XCORR_A registration and the Adam position step on
    rp = pty.refine_params(upsample=20, lr=0.5, start_iter=0)
    prob.refine(1, prm, rp, errors=False)
    torch.cuda.synchronize()
    rsteps = max(1, min(args.steps, 3))
    start.record(stream)
    prob.refine(rsteps, prm, rp, errors=False)
    stop.record(stream)
    torch.cuda.synchronize()
    refine_ms = max_over_ranks(start.elapsed_time(stop) / rsteps, world)
    prob.set_positions(pos_dev)

    # ---- the unfused torch + cuFFT form of the same schedule (comparison)
    from paper_2205_04295_b300.unfused import UnfusedRPIE
    unf = UnfusedRPIE(O0_dev, P0_dev, I_dev.to(torch.int32), pos_dev, wl.W)
    unf.iteration()
    torch.cuda.synchronize()
    start.record(stream)
    unf.iteration()
    stop.record(stream)
    torch.cuda.synchronize()
    unfused_ms = max_over_ranks(start.elapsed_time(stop), world)
    del unf

    # ---- per-kernel durations, CUDA events on the library's stream
    prob.stats(reset=True)  # counts of this one iteration only
    prob.profile(1)
    prob.run(1, prm, errors=False)
    kst = prob.stats(reset=True)
    prob.profile(0)
    pf = per_pass_flops(wl.W, wl.M)
    kinds = [k for k in ("rows_fwd", "cols", "rows_inv", "patch", "probe", "reduce")
             if kst["launches"][k]]
    total_ms = sum(kst["ms"][k] for k in kinds)
    dom = max(kinds, key=lambda k: kst["ms"][k])
    n_dom = kst["launches"][dom]
    avg_ms = kst["ms"][dom] / n_dom
    flops_launch = pf.get(dom, 0.0) * wl.N / n_dom
    peak = fp32_peak_tflops()
    achieved = flops_launch / (avg_ms / 1e3) / 1e12
    per_patch = DRAM_PER_PATCH.get((wl.W, wl.M), {}).get(dom)
    traffic = per_patch * wl.N / n_dom if per_patch else None
    flops, bytes_ = algorithmic(wl.W, wl.M)
    hbm = measured_peaks().get("hbm_gbs", 6400.0)

    # ---- gradient step: loss + dL/dO, dL/dP, dL/dpos (fused adjoint)
    O_t = torch.from_numpy(d["O_true"]).to(dev)
    for _ in range(max(1, args.warmup)):
        prob.loss_grad(O_t, P0_dev, pos_dev)
    gsteps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    barrier(world)
    start.record(stream)
    for _ in range(gsteps):
        prob.loss_grad(O_t, P0_dev, pos_dev)
    stop.record(stream)
    torch.cuda.synchronize()
    grad_ms = max_over_ranks(start.elapsed_time(stop) / gsteps, world)

    # ---- end to end through the C ABI with pinned host buffers
    I_h = I_dev.to(torch.int32).cpu().to(torch.uint16).pin_memory() if hasattr(torch, "uint16") else None
    pos_h = pos_dev.cpu().pin_memory()
    O0_h = O0_dev.cpu().pin_memory()
    P0_h = P0_dev.cpu().pin_memory()
    O_out = torch.empty_like(O0_h).pin_memory()
    P_out = torch.empty_like(P0_h).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        prob.set_data(I_h, pos_h, O0_h, P0_h, overlap=True)  # upload overlaps the passes
        prob.run(1, prm, errors=False)
        pty.check(pty.lib().pty_get_object(prob.h, O_out.data_ptr(), pty.MEM_HOST))
        pty.check(pty.lib().pty_get_probe(prob.h, P_out.data_ptr(), pty.MEM_HOST))
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    h2d = I_h.numel() * 2 + pos_h.numel() * 4 + O0_h.numel() * 8 + P0_h.numel() * 8
    d2h = O_out.numel() * 8 + P_out.numel() * 8

    # ---- probe-mode orthogonalisation (between iterations; synchronises)
    prob.orthogonalize_probe()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(5):
        prob.orthogonalize_probe()
    ortho_ms = (time.perf_counter() - t0) / 5 * 1e3

    batch = run_batch_measure(args, dev, rank, world) if not args.no_batch else None
    # measured FP32 FMA throughput, beside the nominal peak (after the timed work)
    ffma = pty.measure_fp32_peak()

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": wl.name, "W": wl.W, "M": wl.M, "N": wl.N,
                      "object": [wl.Hy, wl.Hx], "groups": n_groups, "tiling": tiling,
                      "schedule": "greedy disjoint groups, index order",
                      "l2": "no flush: every step streams the %.2f GB pattern stack (> 126 MB L2)"
                            % (wl.N * wl.W * wl.W * 2 / 1e9),
                      "parallelism": "replicas" if world > 1 else "single"},
           "hbm_frac_step": value / world * bytes_ / (hbm * 1e9),
           "fp32_frac_step": value / world * flops / (peak * 1e12),
           "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak,
                        "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                        "traffic_unit": "DRAM bytes per launch (warm L2, scaled from ncu)",
                        # the same launch's HBM rate at that traffic, against the
                        # measured copy bandwidth
                        "traffic_gbs": traffic / (avg_ms / 1e3) / 1e9 if traffic else None,
                        "traffic_frac_of_hbm": traffic / (avg_ms / 1e3) / 1e9 / hbm if traffic else None,
                        "peak_source": "148 SM x 128 FP32 lanes x 2 x 2032 MHz",
                        "peak_measured": ffma, "frac_of_measured": achieved / ffma if ffma else None,
                        "peak_measured_source": "FMA-chain kernel (pty_measure_fp32_peak)",
                        "share": kst["ms"][dom] / total_ms},
           # every pass against the same FP32 roof: each one's algorithmic flops
           # per pattern update x N / its summed event time
           "frac_by_kernel": {k: pf[k] * wl.N / (kst["ms"][k] / 1e3) / 1e12 / peak
                              for k in kinds if k in pf and kst["ms"][k] > 0},
           "kernel_ms": {k: kst["ms"][k] for k in kinds},
           "kernel_launches": {k: kst["launches"][k] for k in kinds},
           "gpu_launches": launches,
           "grad": {"ms_per_step": grad_ms, "unit": "ms",
                    "what": "loss and dL/dO, dL/dP, dL/dpos over all positions, bilinear crops"},
           "batch": batch,
           "unfused_cufft": {"value": world * wl.N / (unfused_ms / 1e3), "unit": UNIT,
                             "ms_per_step": unfused_ms,
                             "what": "same schedule as stock torch ops + cuFFT (comparison form)"},
           "refine": {"value": world * wl.N / (refine_ms / 1e3), "unit": UNIT, "ms_per_step": refine_ms,
                      "what": "same step with XCORR_A registration (U = 20) and one Adam step per position"},
           "orthogonalize_ms": ortho_ms,
           "e2e": {"value": world * wl.N * e2e_steps / e2e_s, "unit": UNIT,
                   "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
           "clocks": clk.summary()}
    prob.close()
    return out


def run_batch_measure(args, dev, rank=0, world=1, n_iter=50):
    """The 64-problem uneven batch (W in {64,96,128,192}, N 50..900, M 1..3),
    50 M-rPIE iterations each, in one persistent graph-captured launch per
    rank: aggregate pattern-updates/s.  With several ranks the problems are
    split between them (batch_shard; independent problems: no data-path
    collective, the timing takes the slowest rank), so the total work is
    fixed as ranks are added.  The task granularity and the position-group
    schedule (a cap on the group size) come from the autotuner's table."""
    import torch
    from paper_2205_04295_b300 import autotune, pty, synth
    all_wls = [synth.batch_problem(p) for p in range(64)]
    mine = batch_shard([problem_cost(w) for w in all_wls], rank, world)
    wls = [all_wls[p] for p in mine]
    tuned = autotune.batch_schedule()
    b = pty.Batch([(w.W, w.M, w.N, w.Hy, w.Hx) for w in wls])
    if tuned:
        b.schedule(**tuned["schedule"])
    for w, p in zip(wls, b.problems):
        d = synth.build(w, device=dev)
        p.set_data(synth.counts_u16(d["I"]), torch.from_numpy(d["pos"]).to(dev),
                   torch.from_numpy(d["O0"]).to(dev), torch.from_numpy(d["P0"]).to(dev))
    prm = pty.rpie_params(max_group=tuned["max_group"] if tuned else 0)
    b.run(1, prm)
    torch.cuda.synchronize()
    barrier(world)
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    b.run(n_iter, prm)
    e.record()
    torch.cuda.synchronize()
    ms = max_over_ranks(a.elapsed_time(e), world)
    n = sum(w.N for w in all_wls) * n_iter
    b.close()
    # the same problems one after another, each through pty_run_iterations
    # with its own tuned per-pass launches
    seq_ms = max_over_ranks(run_sequential(wls, dev, n_iter, prm), world)
    return {"problems": 64, "iterations": n_iter, "pattern_updates": n, "ms": ms,
            "value": n / (ms / 1e3), "unit": UNIT, "launches": 1, "ranks": world,
            "scaling": "strong" if world > 1 else None,
            "schedule": tuned,
            "sequential": {"ms": seq_ms, "value": n / (seq_ms / 1e3), "unit": UNIT,
                           "what": "the same problems one after another, pty_run_iterations each"},
            "what": "one persistent cooperative launch (a CUDA graph) per rank for all its "
                    "problems and iterations"}


def run_sequential(wls, dev, n_iter, prm):
    """Milliseconds for the problems run one after another (device time)."""
    import torch
    from paper_2205_04295_b300 import autotune, pty, synth
    probs = []
    for w in wls:
        d = synth.build(w, device=dev)
        q = pty.Problem(w.W, w.M, w.N, w.Hy, w.Hx)
        autotune.apply(q)
        q.set_data(synth.counts_u16(d["I"]), torch.from_numpy(d["pos"]).to(dev),
                   torch.from_numpy(d["O0"]).to(dev), torch.from_numpy(d["P0"]).to(dev))
        q.run(1, prm, errors=False)
        probs.append(q)
    torch.cuda.synchronize()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for q in probs:
        q.run(n_iter, prm, errors=False)
    e.record()
    torch.cuda.synchronize()
    for q in probs:
        q.close()
    return a.elapsed_time(e)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="spiral_256")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--oracle-procs", type=int, default=0,
                    help="with --impl reference: also time this many concurrent oracle processes")
    args = ap.parse_args()
    wl = workloads()[args.workload]()

    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        if rank != 0:
            return
        print(json.dumps(run_reference(args, wl)), flush=True)
        return

    rank, world, local = dist_setup(args.gpus)
    out = run_ours(args, wl, rank, world, local)
    if rank == 0 and not args.no_cpu_baseline:
        single_thread_env()
        d = host_inputs_for_groups(wl, 8)
        r, n, dt, ng = oracle_sample(wl, d, args.cpu_seconds)
        out["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": "%d patches = first %d greedy groups, one FP64 process"
                                         % (n, ng)}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
