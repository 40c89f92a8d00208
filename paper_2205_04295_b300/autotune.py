"""Project autotuner for the launch geometry of the M-rPIE passes.

For a (W, M) class it searches, in stages, the tiling of one problem:
  1. CB, columns per CTA of the column pass;
  2. R x ppc, rows and patches per CTA of the two row passes;
  3. the far-field scratch budget (the chunk of a group held in L2);
  4. for W <= 128, the fused single-kernel patch path with S = 1, 2, 4, 8
     CTAs per patch, kept where it beats the three passes;
timing one full iteration per candidate with CUDA events on the library's
stream (results never depend on the tiling beyond the summation order of the
probe sums).  For the batched form it searches the task granularity (how many
tasks a pass of one chunk is split into).  Winners are cached in JSON
(``tuning.json`` beside this file) keyed "W x M".

    python -m paper_2205_04295_b300.autotune [--classes 256x5,64x1,...] [--out FILE]
"""
import argparse
import json
import os

from . import pty

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")
LANES = {32: 8, 64: 8, 96: 12, 128: 16, 192: 16, 256: 16}


def _pow2(lo, hi):
    v = lo
    while v <= hi:
        yield v
        v *= 2


def candidates(W, M):
    L = LANES[W]
    Rs = [r for r in _pow2(1, 16) if W % r == 0 and M * r * L <= 256]
    CBs = [c for c in _pow2(2, 16) if (W // 2) % c == 0 and M * c * L <= 384]
    # patches per CTA: not only powers of two, so that a group's grid can end
    # on a nearly full wave of CTAs
    return (Rs, [1, 2, 3, 4, 5, 6, 8, 10, 12, 16], CBs, [48 << 20, 96 << 20, 144 << 20, 192 << 20],
            [1, 2, 3, 4])


def time_iteration(prob, params, reps=2):
    """Milliseconds of one iteration (median of reps, after one warm-up)."""
    import torch
    prob.run(1, params, errors=False)
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(prob.stream)
        prob.run(1, params, errors=False)
        b.record(prob.stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    ts.sort()
    return ts[len(ts) // 2]


def tune_problem(prob, params=None, reps=2):
    """Staged search on one problem (its data already set).  Returns a dict
    with the best tiling, its time and every trial."""
    params = params or pty.rpie_params()
    Rs, ppcs, CBs, budgets, ppcbs = candidates(prob.W, prob.M)
    best = dict(prob.tiling())
    best["scratch_bytes"] = max(budgets)  # the largest chunk first: fewest launches
    trials = []

    def trial(**t):
        cfg = dict(best)
        cfg.update(t)
        prob.set_tiling(cfg["R"], cfg["ppc"], cfg["CB"], cfg["scratch_bytes"], cfg["ppcb"],
                        cfg.get("fused", 0))
        ms = time_iteration(prob, params, reps)
        trials.append(dict(cfg, ms=ms))
        return ms, cfg

    for stage in (
        [dict(CB=c, ppcb=q) for c in CBs for q in ppcbs],
        [dict(R=r, ppc=q) for r in Rs for q in ppcs],
        [dict(scratch_bytes=b) for b in budgets],
    ):
        results = [trial(**t) for t in stage]
        ms, cfg = min(results, key=lambda x: x[0])
        best = cfg
        best_ms = ms
    best, best_ms = _fused_stage(prob, best, best_ms, trial)
    _set(prob, best)
    return {"tiling": best, "ms": best_ms, "trials": trials}


def _set(prob, t):
    prob.set_tiling(t["R"], t["ppc"], t["CB"], t["scratch_bytes"], t.get("ppcb", 0),
                    t.get("fused", 0))


def _fused_stage(prob, best, best_ms, trial):
    """Stage 4: the fused patch kernel (W <= 128) on top of the best
    three-pass tiling (whose scratch budget it keeps for registration
    chunks); slab counts the shared memory does not hold are skipped."""
    if prob.W > 128:
        return best, best_ms
    for S in (1, 2, 4, 8):
        try:
            ms, cfg = trial(fused=S)
        except pty.PtyError:
            continue
        if ms < best_ms:
            best, best_ms = cfg, ms
    return best, best_ms


def tune_fused(prob, params=None, reps=2, base=None):
    """Stage 4 alone, starting from `base` (a three-pass tiling; default the
    problem's current one)."""
    params = params or pty.rpie_params()
    trials = []
    base = dict(base or prob.tiling())
    base["fused"] = 0

    def trial(**t):
        cfg = dict(base)
        cfg.update(t)
        _set(prob, cfg)
        ms = time_iteration(prob, params, reps)
        trials.append(dict(cfg, ms=ms))
        return ms, cfg

    ms0, _ = trial()
    best, best_ms = _fused_stage(prob, base, ms0, trial)
    _set(prob, best)
    return {"tiling": best, "ms": best_ms, "trials": trials}


def tune_batch(batch, n_iter=1, params=None, caps=(0, 32, 16, 8)):
    """Task granularity and position-group schedule of the batched form.

    Stage 1 times the task splits with unlimited groups; stage 2 times caps
    on the number of positions per disjoint group (0 = the greedy groups as
    they come; a cap makes more, smaller groups: more dependency steps, but
    finer tasks for the persistent kernel to balance).  A different cap is a
    different schedule of the same method (the oracle takes the same
    ``max_group``), so parity tests run with the chosen cap on both sides.
    The problems' state advances with every trial; only times are compared.
    Returns {"schedule": splits, "max_group": cap, "s": seconds, "trials": [...]}."""
    import time
    import torch
    params = params or pty.rpie_params()
    trials = []

    def timed(cap):
        p = pty.rpie_params(params.alpha_O, params.alpha_P, params.beta, params.gamma,
                            params.eps, params.reg_eps, cap, bool(params.update_probe))
        batch.run(n_iter, p)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        batch.run(n_iter, p)
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    best = None
    for sr, sc, sp in ((1, 1, 1), (2, 1, 2), (4, 2, 4), (8, 2, 4), (8, 4, 8), (16, 8, 8)):
        sched = dict(split_rows=sr, split_cols=sc, split_probe=sp)
        batch.schedule(**sched)
        dt = timed(0)
        trials.append(dict(sched, max_group=0, s=dt))
        if best is None or dt < best[0]:
            best = (dt, sched, 0)
    batch.schedule(**best[1])
    for cap in caps:
        if cap == 0:
            continue
        dt = timed(cap)
        trials.append(dict(best[1], max_group=cap, s=dt))
        if dt < best[0]:
            best = (dt, best[1], cap)
    return {"schedule": best[1], "max_group": best[2], "s": best[0], "trials": trials}


def batch_schedule(table=None):
    """The cached batched-form choice ({"schedule": ..., "max_group": ...}), or None."""
    table = load() if table is None else table
    return table.get("batch")


def load(path=CACHE):
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return {}


def save(table, path=CACHE):
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)


def apply(prob, table=None):
    """Apply the cached tiling of prob's (W, M) class, if any; returns it."""
    table = load() if table is None else table
    ent = table.get("%dx%d" % (prob.W, prob.M))
    if ent:
        t = ent["tiling"]
        _set(prob, t)
        return t
    return None


def _workload(W, M):
    from . import synth
    if (W, M) == (64, 1):
        return synth.plain_rpie_64()  # the 10 x 10 raster of the plain workload
    if (W, M) == (128, 3):
        return synth.refine_128()  # the 40 x 40 jittered raster of the refinement workload
    if W == 256 and M == 4:
        return synth.sweep_256()  # the 40 000-position raster: its group sizes
    if W == 256:
        return synth.spiral_256()  # the full 10^4-position scan: its group sizes
    n = 14 if W <= 96 else 10
    return synth.tiny(W=W, M=M, ny=n, nx=n, step=W / 8.0, seed=900 + W + M, photons=1e6,
                      jitter=2.0)


def main():
    import torch
    from . import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--classes", default="256x5,256x4,64x1,64x2,64x3,96x1,96x2,96x3,128x1,"
                                        "128x2,128x3,192x1,192x2,192x3")
    ap.add_argument("--out", default=CACHE)
    ap.add_argument("--fused-only", action="store_true",
                    help="only stage 4 (the fused patch kernel) on top of each cached tiling")
    ap.add_argument("--batch", action="store_true",
                    help="also tune the 64-problem batched workload (task splits, group cap)")
    args = ap.parse_args()
    table = load(args.out)
    for cls in filter(None, args.classes.split(",")):
        W, M = (int(v) for v in cls.split("x"))
        wl = _workload(W, M)
        d = synth.build(wl, device="cuda")
        prob = pty.Problem(wl.W, wl.M, wl.N, wl.Hy, wl.Hx)
        prob.set_data(synth.counts_u16(d["I"]), torch.from_numpy(d["pos"]).cuda(),
                      torch.from_numpy(d["O0"]).cuda(), torch.from_numpy(d["P0"]).cuda())
        if args.fused_only and cls in table:
            res = tune_fused(prob, base=table[cls]["tiling"])
            res["trials"] = table[cls].get("trials", []) + res["trials"]
        else:
            res = tune_problem(prob)
        res["workload"] = wl.name
        table[cls] = res
        print(cls, res["tiling"], "%.3f ms" % res["ms"], flush=True)
        prob.close()
    if args.batch:
        wls = [synth.batch_problem(p) for p in range(64)]
        b = pty.Batch([(w.W, w.M, w.N, w.Hy, w.Hx) for w in wls])
        for w, p in zip(wls, b.problems):
            d = synth.build(w, device="cuda")
            p.set_data(synth.counts_u16(d["I"]), torch.from_numpy(d["pos"]).cuda(),
                       torch.from_numpy(d["O0"]).cuda(), torch.from_numpy(d["P0"]).cuda())
        res = tune_batch(b, n_iter=2)
        res["workload"] = "64-problem uneven batch"
        table["batch"] = res
        print("batch", res["schedule"], "max_group", res["max_group"], "%.3f s" % res["s"], flush=True)
        b.close()
    save(table, args.out)


if __name__ == "__main__":
    main()
