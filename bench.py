"""Benchmark: randomized rounding of a sum of 20 TT-tensors (N = 50, I = 100,
rank 10 each, sketch rank 30, tolerance 1e-8) on GB300, one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one full call of the rounding (device sketch drawn from the seed,
right-to-left partial contractions, left-to-right sketch / QR / projection,
tolerance truncation) on inputs resident in HBM. Inputs plus sketch (112 MB)
fit in L2, so L2 is flushed (a 256 MB write) before every timed step, outside
the timed events. Multi-GPU runs are independent replicas (weak scaling): each
rank rounds its own sum; value = all ranks' work / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TT-round time & TFLOP/s (sum of 20 TTs, N=50): rand vs det, mixed vs FP64"
DTYPE_MIXED = ("f64-emulated: bf16 digit products on tcgen05 with exact integer sums (2 digits = 14 bits in the "
               "Algorithm 3 contractions, 8 digits = 56 bits in core updates / sketches / projections), f64 QR / "
               "SVD / truncation")
WORKLOAD = dict(workload="sum of K=20 TT-tensors, N=50, I_n=100, rank 10 each (formal rank 200), "
                         "sketch rank 30, tol 1e-8, Gaussian cores (Definition 3.1 scaling)",
                K=20, N=50, I=100, R=10, ell=30, tol=1e-8)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="auto", choices=["auto", "fp64", "mixed"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    p.add_argument("--no-det", action="store_true", help="skip the deterministic comparison")
    p.add_argument("--no-extra", action="store_true", help="skip the single-TT and adjoint legs")
    p.add_argument("--legs", default="mixed,fp64,twosided,det",
                   help="--config large: comma list of the legs to run (mixed, fp64, twosided, det)")
    p.add_argument("--config", default="sum", choices=["sum", "batched", "large"],
                   help="sum: 20 TTs, N=50 (default); batched: 256 uneven sums in one graph; "
                        "large: 30 TTs, N=30, I=256, rank 20")
    return p.parse_args()


def max_over_ranks(x, world, dist, device):
    """The largest of every rank's value (timings: the job ends with its slowest replica)."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(rank):
    """Rank r rounds its own sum, drawn from seed 1 + r (replicas, no shared data)."""
    return 1 + int(rank)


def replica_tflops(flops_per_replica, ms, world):
    """Whole-job throughput of `world` independent replicas finishing within `ms`."""
    return world * flops_per_replica / (ms * 1e-3) / 1e12


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def fp64_alu_peak_tflops(sm_mhz):
    # 152 SMs x 2 FP64 FMA per clock per SM x 2 flops (GB300 FP64 units)
    return 152 * 2 * 2 * sm_mhz * 1e6 / 1e12


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.proc = None
        self.index = index
        self.path = os.path.join(ROOT, ".bench", f"clocks_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        try:
            rows = [l.split(",") for l in open(self.path) if l.strip()]
        except Exception:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        mx = float(rows[0][2])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": reasons, "samples": len(rows)}


def load_workload(seed):
    import synth
    return synth.workload_sum_literal(seed, K=WORKLOAD["K"], N=WORKLOAD["N"], I=WORKLOAD["I"], R=WORKLOAD["R"])


def ranks_of(Ys):
    return [[1] + [int(c.shape[2]) for c in Y] for Y in Ys]


ORACLE_SEED = 7          # sketch seed of the oracle leg (the GPU legs re-run once with it)


def _oracle_rounding(Ys, seed=ORACLE_SEED):
    import oracle
    dims = [c.shape[1] for c in Ys[0]]
    ell = [1] + [WORKLOAD["ell"]] * (len(dims) - 1) + [1]
    sk = oracle.gaussian_sketch_philox(seed, dims, ell)
    X = oracle.round_sum_randorth(Ys, sk)
    return oracle.truncate_left_orthogonal(X, WORKLOAD["tol"])


def oracle_one_thread_seconds():
    """One oracle rounding of the workload in a child process limited to one
    BLAS / OpenMP thread (the thread count is fixed when NumPy loads)."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    p = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample"], capture_output=True, text=True,
                       env=env, timeout=900)
    if p.returncode != 0:
        return None
    return json.loads(p.stdout.strip().splitlines()[-1])["seconds"]


def oracle_leg(Ys, gpu_results, det_result, reps=2):
    """The oracle as it stands (NumPy FP64) on the host cores: the cpu_baseline
    (whole workload, all cores, best of `reps`, plus one rounding on one thread)
    and, against its result on the same sketch (Philox, seed ORACLE_SEED), the
    relative Frobenius error of every GPU leg. gpu_results: name -> host cores of
    the GPU rounding with that sketch seed; det_result: host cores of the
    deterministic rounding. Rounding errors ||X - sum_j Y_j|| / ||sum_j Y_j||
    come from inner products (exact algebra; about 1e-8 relative resolution)."""
    import numpy as np
    import oracle
    from paper_2110_04393_gb300.costs import flops_sum_randorth
    dims = [c.shape[1] for c in Ys[0]]
    ell = [1] + [WORKLOAD["ell"]] * (len(dims) - 1) + [1]
    ts = []
    Xo = None
    for _ in range(reps):
        t0 = time.perf_counter()
        Xo = _oracle_rounding(Ys)
        ts.append(time.perf_counter() - t0)
    t = min(ts)
    fl = flops_sum_randorth(dims, ranks_of(Ys), ell)
    threads = os.environ.get("OPENBLAS_NUM_THREADS") or os.environ.get("OMP_NUM_THREADS") or str(os.cpu_count())
    t1 = oracle_one_thread_seconds()
    base = {"value": fl / t / 1e12, "unit": "TFLOP/s", "cores": int(threads), "kind": "oracle",
            "sample": f"whole workload (sum-rounding + truncation, host-drawn sketch), best of {reps}",
            "seconds_per_rounding": t,
            "one_thread": ({"value": fl / t1 / 1e12, "unit": "TFLOP/s", "cores": 1, "seconds_per_rounding": t1,
                            "sample": "one rounding of the whole workload, BLAS limited to one thread"}
                           if t1 else None)}
    K = len(Ys)
    G = np.array([[oracle.inner(Ys[a], Ys[b]) for b in range(K)] for a in range(K)])
    yy = float(G.sum())

    def rounding_error(X):
        xy = sum(oracle.inner(X, Y) for Y in Ys)
        return float(np.sqrt(max(yy - 2.0 * xy + oracle.inner(X, X), 0.0) / yy))

    e_o = rounding_error(Xo)
    nrm_o = oracle.norm(Xo)
    err = {"sketch_seed": ORACLE_SEED, "oracle_rounding_error": e_o,
           "method": "distance to the oracle's result by orthogonalizing the difference TT; rounding errors "
                     "from inner products"}
    for name, X in gpu_results.items():
        e = rounding_error(X)
        err[name] = {"rel_diff_vs_oracle_result": oracle.diff_norm(X, Xo) / nrm_o, "rounding_error": e,
                     "ratio_to_oracle_error": e / e_o if e_o > 0 else None,
                     "ranks_equal_oracle": oracle.ranks_of(X) == oracle.ranks_of(Xo)}
    if det_result is not None:
        e_d = rounding_error(det_result)
        err["det_fp64"] = {"rounding_error": e_d, "resolved": e_d > 1e-7,
                           "resolution": "inner-product errors below about 1e-7 read as 0",
                           "note": "deterministic TT-SVD rounding to the same tolerance (the sum is generically "
                                   "of full rank 200, so its error is at the tolerance while the rank-30 "
                                   "randomized rounding's is O(1))"}
    return base, err


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2110_04393_gb300.costs import flops_sum_randorth
    Ys = load_workload(1)
    dims = [c.shape[1] for c in Ys[0]]
    ell = [1] + [WORKLOAD["ell"]] * (len(dims) - 1) + [1]
    fl = flops_sum_randorth(dims, ranks_of(Ys), ell)

    def step(seed):
        sk = oracle.gaussian_sketch_philox(seed, dims, ell)
        X = oracle.round_sum_randorth(Ys, sk)
        return oracle.truncate_left_orthogonal(X, WORKLOAD["tol"])

    for w in range(a.warmup):
        step(100 + w)
    t0 = time.perf_counter()
    for s in range(a.steps):
        step(s)
    t = (time.perf_counter() - t0) / a.steps
    val = fl / t / 1e12
    threads = os.environ.get("OPENBLAS_NUM_THREADS") or os.environ.get("OMP_NUM_THREADS") or str(os.cpu_count())
    cfg = {k: v for k, v in WORKLOAD.items()}
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": a.gpus,
                      "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
                      "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": int(threads), "kind": "oracle",
                                       "sample": "whole workload per step (sketch drawn on the host)"},
                      "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
          flush=True)


def _event_ms(torch, fn, reps=10, warm=3):
    """Median of `reps` CUDA-event timings of fn() after `warm` untimed calls."""
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def leg_single_tt(tt, torch, dev):
    """Section 4.1 shape (config 1): Y of rank 10 plus 1e-6 E of rank 30, N = 10,
    I = 50; Randomize-then-Orthogonalize with sketch rank 15 (captured plan and
    eager call), the fixed-rank truncation to 10, and the deterministic rounding
    to rank 10. Latencies in microseconds (inputs resident, warm)."""
    import synth
    Ys = synth.workload_single(1, N=10, I=50, R=10, R_pert=30, eps=1e-6)
    Yd = [[torch.from_numpy(c).to(dev) for c in Y] for Y in Ys]
    dims = [50] * 10
    ell = [1] + [15] * 9 + [1]
    plan = tt.SumRoundingPlan(dims, ranks_of(Ys), ell, tol=0.0, precision="fp64", device=dev)
    X = plan(Yd, seed=1)
    out = {"workload": "N=10, I=50, Y rank 10 + 1e-6 E rank 30 (formal rank 40), sketch rank 15, truncation to 10",
           "rand_plan_us": 1e3 * _event_ms(torch, lambda: plan(Yd, seed=1)),
           "rand_eager_us": 1e3 * _event_ms(torch, lambda: tt.tt_round_sum_rand(Yd, ell, seed=1)),
           "truncate_to_10_us": 1e3 * _event_ms(torch, lambda: tt.tt_truncate_lorth(X, max_rank=10)),
           "det_rank10_us": 1e3 * _event_ms(torch, lambda: tt.tt_round_det(Yd, max_rank=10), reps=5)}
    plan.close()
    return out


def leg_adjoint_f32(tt, torch, dev):
    """Config 4: fixed-sketch RandOrth of a TT with N = 16, I = 32, rank 64 to
    l = 16 with float32 storage: forward and hand-written adjoint (FP32-class
    products, FP64 QR steps), beside the float64 path. Milliseconds."""
    import synth
    N, I, R, ell = 16, 32, 64, 16
    dims = [I] * N
    Y = synth.gaussian_tt(synth.rng_for(140, 0), dims, [1] + [R] * (N - 1) + [1])
    el = tt.clamp_ranks(dims, [1] + [ell] * (N - 1) + [1])
    Om = synth.gaussian_tt(synth.rng_for(140, 1), dims, el)
    res = {"workload": "N=16, I=32, rank 64 rounded to l=16, fixed sketch; loss gradient w.r.t. all input cores"}
    for name, dt in (("f32", torch.float32), ("f64", torch.float64)):
        Yd = [torch.from_numpy(c).to(dev, dt) for c in Y]
        Od = [torch.from_numpy(c).to(dev, dt) for c in Om]
        X = tt.tt_round_rand(Yd, el, sketch=Od, tol=0.0)
        Xb = [torch.ones_like(c) for c in X]
        res[name + "_forward_ms"] = _event_ms(torch, lambda: tt.tt_round_rand(Yd, el, sketch=Od, tol=0.0))
        res[name + "_backward_ms"] = _event_ms(torch, lambda: tt.tt_round_rand_backward(Yd, el, Od, Xb))
    return res


def timed_plan(tt, torch, plan, Yd, steps, warmup, flush, stream, world, dist):
    """Warm-up and timed replays of a captured plan. Returns (ms per step,
    per-kind profile, kernel launches, output ranks); the profile holds the
    event pairs captured in the graph when it was captured with profiling on."""
    for w in range(warmup):
        plan(Yd, seed=1000 + w)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    tt.prof_reset()
    times = []
    out_ranks = None
    for s in range(steps):
        flush.fill_(s & 0xFF)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        X = plan(Yd, seed=s)
        e1.record(stream)
        out_ranks = [int(X[0].shape[0])] + [int(c.shape[2]) for c in X]
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    kinds = {k: tt.prof_read_kind(k) for k in (0, 1)}
    launches = tt.prof_read()[3]
    return statistics.median(times), kinds, launches, out_ranks


def run_ours(a):
    import torch
    import torch.distributed as dist
    import paper_2110_04393_gb300 as tt
    from paper_2110_04393_gb300.costs import flops_sum_randorth, bytes_sum_randorth

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    Ys = load_workload(replica_seed(rank))
    dims = [c.shape[1] for c in Ys[0]]
    N = len(dims)
    ell = [1] + [WORKLOAD["ell"]] * (N - 1) + [1]
    tol = WORKLOAD["tol"]
    flops = flops_sum_randorth(dims, ranks_of(Ys), ell)
    nbytes = bytes_sum_randorth(dims, ranks_of(Ys), ell)
    Yd = [[torch.from_numpy(c).to(dev) for c in Y] for Y in Ys]
    precs = ["mixed", "fp64"] if a.precision == "auto" else [a.precision]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    # Each precision is planned and captured into a CUDA graph once (profiling
    # on, so the timed launches' event pairs are graph nodes); every step
    # replays it on the resident inputs with a fresh sketch seed.
    # The timed steps replay graphs captured without profiling; the kernel-class
    # durations of the roofline come from a second capture of the same schedule
    # with event nodes around every timed launch, replayed as many steps right
    # after (those event nodes slow a replay a little, so they are kept out of
    # the headline time).
    res_prec, prof_prec, plans = {}, {}, {}
    with Clocks(local) as clk:
        for prec in precs:
            tt.prof_enable(False)
            plans[prec] = tt.SumRoundingPlan(dims, ranks_of(Ys), ell, tol=tol, precision=prec, device=dev)
            res_prec[prec] = timed_plan(tt, torch, plans[prec], Yd, a.steps, a.warmup, flush, stream, world, dist)
            tt.prof_enable(True)
            pp = tt.SumRoundingPlan(dims, ranks_of(Ys), ell, tol=tol, precision=prec, device=dev)
            prof_prec[prec] = timed_plan(tt, torch, pp, Yd, a.steps, 1, flush, stream, world, dist)
            tt.prof_enable(False)
            pp.close()
    prim = precs[0]
    t_ms, _, launches, out_ranks = res_prec[prim]
    tp_ms, kinds, _, _ = prof_prec[prim]
    launches = plans[prim].launches * a.steps          # kernels launched by the timed replays
    t_ms = max_over_ranks(t_ms, world, dist, dev)
    if world > 1:
        dist.barrier()

    # end to end through the public API with host buffers (pinned): one packed
    # host-to-device copy of the summands, the replay, one device-to-host copy
    # of the rounded cores, all inside the timed region
    plan = plans[prim]
    e2e_times = []
    h2d = d2h = 0
    if not a.no_e2e:
        h_in = plan.pack_host(Ys)
        _, _, in_total, out_total = plan.host_layout()
        h_out = torch.empty(out_total, dtype=torch.float64, pin_memory=True)
        h2d, d2h = in_total * 8, out_total * 8
    for s in range(0 if a.no_e2e else max(2, a.steps // 2) + 1):
        flush.fill_(s & 0xFF)                 # L2 flushed like the device-resident steps
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hX = plan.run_host(h_in, seed=s, out=h_out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if s > 0:
            e2e_times.append(e0.elapsed_time(e1))
    e2e_ms = max_over_ranks(statistics.median(e2e_times) if e2e_times else float("nan"), world, dist, dev)

    # the same rounding without a captured plan (planning and launches per call)
    ws = torch.empty(1 << 30, dtype=torch.uint8, device=dev)
    eager = []
    for s in range(3):
        flush.fill_(s & 0xFF)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tt.tt_round_sum_rand(Yd, ell, seed=s, tol=tol, precision=prim, workspace=ws)
        e1.record(stream)
        torch.cuda.synchronize()
        eager.append(e0.elapsed_time(e1))
    eager_ms = min(eager)

    # deterministic comparison (Algorithms 1 + 2 on the formed sum), same inputs and tolerance
    # one more (untimed) rounding per precision with the oracle leg's sketch
    # seed, copied to the host for the error comparison of the oracle leg
    err_inputs = {}
    if world == 1 and not a.no_cpu_baseline:
        for prec in precs:
            Xp = plans[prec](Yd, seed=ORACLE_SEED)
            torch.cuda.synchronize()
            err_inputs["rand_" + prec] = [c.cpu().numpy() for c in Xp]
    det = None
    det_host = None
    if not a.no_det:
        from paper_2110_04393_gb300.costs import flops_det
        Xd = tt.tt_round_det(Yd, tol=tol)          # warm-up
        dts = []
        for s in range(2):
            flush.fill_(s & 0xFF)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            Xd = tt.tt_round_det(Yd, tol=tol)
            e1.record(stream)
            torch.cuda.synchronize()
            dts.append(e0.elapsed_time(e1))
        dr = [int(Xd[0].shape[0])] + [int(c.shape[2]) for c in Xd]
        det_host = [c.cpu().numpy() for c in Xd]
        S = [1] + [sum(R[n] for R in ranks_of(Ys)) for n in range(1, N)] + [1]
        S[1] = min(S[1], dims[0])
        for n in range(N - 1, 0, -1):
            S[n] = min(S[n], dims[n] * S[n + 1])
        dfl = flops_det(dims, S, dr)
        dms = min(dts)
        det = {"ms_per_step": dms, "tflops_alg": dfl / (dms * 1e-3) / 1e12, "gflop_alg": dfl / 1e9,
               "output_ranks_max": max(dr), "rand_speedup": dms / t_ms}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    P = peaks()
    clocks = clk.summary()
    # FP64 roofline denominator: the FMA rate measured live on this GPU (best of
    # three launches of a register-only FMA loop); the unit-count figure stays
    # beside it for context
    fp64_derived = fp64_alu_peak_tflops(P.get("sm_max_mhz", 2070.0))
    try:
        fp64_peak = max(tt.probe_fp64_rate(1 << 14) for _ in range(3))
        fp64_note = (f"FP64 FMA rate measured (of measured): tt_probe_fp64_rate, best of 3 launches, "
                     f"{fp64_peak:.3f} TFLOP/s; derived 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz = "
                     f"{fp64_derived:.3f}; flops algorithmic (FP64-equivalent)")
    except Exception as e:                  # the probe failed: the derived figure, said so
        fp64_peak = fp64_derived
        fp64_note = (f"FP64 ALU peak derived (of derived; the probe failed: {e}): 152 SMs x 2 DFMA/clk x "
                     "2 flop x 2070 MHz; flops algorithmic (FP64-equivalent)")
    traffic = {}
    try:
        traffic = json.load(open(os.path.join(ROOT, "profiles", "traffic_per_launch.json")))
    except Exception:
        pass

    def kind_line(k, ms, fl, n):
        name, kern = {0: ("contraction groups (Algorithm 3 sweep, core updates, sketches, projections)",
                          "contraction group (tc_exponent + tc_split + gemm_tc)"),
                      1: ("cqr_coop_kernel (one-launch Cholesky-QR chain of the sketch and truncation QRs)",
                          "cqr_coop_kernel")}[k]
        achieved = fl / (ms * 1e-3) / 1e12 if ms > 0 else None
        tr = traffic.get(f"{prim}:{k}", {})
        return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": (achieved / fp64_peak) if achieved else None,
                # counters taken on another kernel than the one timed now are not reported
                "traffic": tr.get("bytes_per_launch") if tr.get("kernel") == kern else None,
                "peak_note": fp64_note,
                "launches": n, "ms_per_step": ms / a.steps, "share_of_step": ms / (tp_ms * a.steps),
                "measured_on": "profiled replays of the same schedule (event nodes around every timed launch), "
                               f"{tp_ms:.2f} ms per step"}

    lines = {k: kind_line(k, *kinds[k]) for k in (0, 1)}
    dom = max((0, 1), key=lambda k: kinds[k][0])
    variants = {}
    for prec in precs:
        tm, kd, _, _ = res_prec[prec]
        variants["rand_" + prec] = {"ms_per_step": tm, "tflops_alg": flops / (tm * 1e-3) / 1e12,
                                    "graph_replay": True}
    variants["rand_" + prim + "_eager"] = {"ms_per_step": eager_ms, "tflops_alg": flops / (eager_ms * 1e-3) / 1e12}
    variants["det_fp64"] = det
    if world == 1 and not a.no_extra:
        variants["single_tt_cfg1"] = leg_single_tt(tt, torch, dev)
        variants["adjoint_cfg4"] = leg_adjoint_f32(tt, torch, dev)
    res = {
        "metric": METRIC,
        "value": replica_tflops(flops, t_ms, world),
        "unit": "TFLOP/s",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": t_ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": DTYPE_MIXED if prim == "mixed" else "f64",
        "data": "synthetic",
        "config": dict(WORKLOAD, precision=prim, l2="flushed before every timed step (256 MB write)",
                       parallelism=f"replicas x{world}", algorithmic_gflop_per_step=flops / 1e9,
                       algorithmic_mb_per_step=nbytes / 1e6, output_ranks_max=max(out_ranks),
                       execution="captured CUDA graph per precision, replayed per step"),
        "e2e": {"value": replica_tflops(flops, e2e_ms, world), "unit": "TFLOP/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "l2": "flushed before every step (256 MB write, outside the timed region)"},
        "gpu_launches": launches,
        "roofline": lines[dom],
        "roofline_other": lines[1 - dom],
        "clocks": clocks,
        "variants": variants,
    }
    if world == 1 and not a.no_cpu_baseline:
        res["cpu_baseline"], res["error_vs_oracle"] = oracle_leg(Ys, err_inputs, det_host)
    print(json.dumps(res), flush=True)
    for pl in plans.values():
        pl.close()
    if world > 1:
        dist.destroy_process_group()


BATCHED = dict(workload="256 independent sums in one CUDA graph: N=20, I_n=64, K ~ U[2,30] summands of rank "
                        "~ U[4,16] (formal ranks 8-480), target = sketch rank ~ U[8,32], fixed rank, mixed precision",
               B=256, N=20, I=64)


def batched_problems(seed=1):
    import numpy as np
    rng = np.random.default_rng(seed)
    N, I = BATCHED["N"], BATCHED["I"]
    probs = []
    for b in range(BATCHED["B"]):
        K = int(rng.integers(2, 31))
        Rs = [int(x) for x in rng.integers(4, 17, size=K)]
        ell = int(rng.integers(8, 33))
        probs.append(dict(dims=[I] * N, summand_ranks=[[1] + [r] * (N - 1) + [1] for r in Rs],
                          ells=[1] + [ell] * (N - 1) + [1], tol=0.0))
    return probs


def run_batched(a):
    """Config 3: one graph of 256 roundings, chain width chosen by the autotuner."""
    import torch
    import paper_2110_04393_gb300 as tt
    from paper_2110_04393_gb300.costs import flops_sum_randorth
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    dev = torch.device("cuda", 0)
    probs = batched_problems(1)
    g = torch.Generator(device=dev)
    g.manual_seed(2)
    batch = []
    for pr in probs:
        I = pr["dims"]
        Ys = []
        for R in pr["summand_ranks"]:
            Ys.append([torch.randn((R[n], I[n], R[n + 1]), dtype=torch.float64, device=dev, generator=g)
                       / (R[n] * I[n] * R[n + 1]) ** 0.5 for n in range(len(I))])
        batch.append(Ys)
    flops = sum(flops_sum_randorth(pr["dims"], pr["summand_ranks"], tt.clamp_ranks(pr["dims"], pr["ells"]))
                for pr in probs)
    in_bytes = sum(c.numel() * 8 for Ys in batch for Y in Ys for c in Y)
    t0 = time.perf_counter()
    (width, qr_ctas), tune = tt.tune_batch_schedule(probs, batch, precision="mixed", widths=(1, 2, 4),
                                                    qr_ctas=(4, 8, 16), reps=1,
                                                    cache_path=os.path.join(ROOT, ".bench", "batch_tuning.json"))
    t_tune = time.perf_counter() - t0
    t0 = time.perf_counter()
    plan = tt.BatchRoundingPlan(probs, precision="mixed", width=width, qr_ctas=qr_ctas)
    t_plan = time.perf_counter() - t0
    for w in range(a.warmup):
        plan(batch, seeds=[1000 * w + b for b in range(len(probs))])
    torch.cuda.synchronize()
    times = []
    with Clocks(0) as clk:
        for s in range(a.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            plan(batch, seeds=[s * 7919 + b for b in range(len(probs))])
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    t_ms = statistics.median(times)
    P = peaks()
    hbm = P.get("hbm_gbs") or P.get("hbm_GBps") or 6784.5
    gbs = 2 * in_bytes / (t_ms * 1e-3) / 1e9
    print(json.dumps({
        "metric": METRIC + " [batched config]", "value": flops / (t_ms * 1e-3) / 1e12, "unit": "TFLOP/s",
        "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": t_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 (mixed: emulated FP64 tensor-core contractions)",
        "data": "synthetic", "config": dict(BATCHED, inputs_gb=in_bytes / 1e9, l2="inputs larger than L2",
                                            algorithmic_gflop=flops / 1e9),
        "schedule": {"fused": plan.fused, "width": width, "qr_ctas": qr_ctas,
                     "tuning_ms": {f"width={w},qr_ctas={q}": v for (w, q), v in tune.items()},
                     "tuning_s": t_tune, "plan_s": t_plan, "launches_per_step": plan.launches},
        "input_read_gbs": gbs, "input_read_frac_of_hbm": gbs / hbm, "clocks": clk.summary()}), flush=True)
    plan.close()


LARGE = dict(workload="sum of K=30 TT-tensors, N=30, I_n=256, rank 20 each (formal rank 600), sketch rank 70 "
                      "(Two-Sided 70 / 105), tol 1e-6, Gaussian cores (Definition 3.1 scaling, drawn on the device)",
             K=30, N=30, I=256, R=20, ell=70, rho=105, tol=1e-6)


def run_large(a):
    """The large sum: Randomize-then-Orthogonalize through captured plans in
    both precisions, Two-Sided (fixed ranks) and the deterministic rounding of
    the formed sum (about 22 GB of cores), on the same device-resident inputs
    (0.74 GB, larger than L2, so no flush)."""
    import torch
    import paper_2110_04393_gb300 as tt
    from paper_2110_04393_gb300.costs import flops_sum_randorth, flops_det
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    dev = torch.device("cuda", 0)
    K, N, I, R = LARGE["K"], LARGE["N"], LARGE["I"], LARGE["R"]
    dims = [I] * N
    rk = [1] + [R] * (N - 1) + [1]
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    Yd = [[torch.randn((rk[n], I, rk[n + 1]), dtype=torch.float64, device=dev, generator=g)
           / (rk[n] * I * rk[n + 1]) ** 0.5 for n in range(N)] for _ in range(K)]
    ranks = [rk] * K
    ell = tt.clamp_ranks(dims, [1] + [LARGE["ell"]] * (N - 1) + [1])
    rho = tt.clamp_ranks(dims, [1] + [LARGE["rho"]] * (N - 1) + [1])
    tol = LARGE["tol"]
    flops = flops_sum_randorth(dims, ranks, ell)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps, warm):
        for w in range(warm):
            fn(1000 + w)
        torch.cuda.synchronize()
        ts = []
        for s in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn(s)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts), out

    variants = {}
    legs = set(a.legs.split(","))
    with Clocks(0) as clk:
        for prec in [p for p in ("mixed", "fp64") if p in legs]:
            plan = tt.SumRoundingPlan(dims, ranks, ell, tol=tol, precision=prec, device=dev)
            ms, X = timed(lambda s: plan(Yd, seed=s), a.steps, a.warmup)
            variants["rand_" + prec] = {"ms_per_step": ms, "tflops_alg": flops / (ms * 1e-3) / 1e12,
                                        "output_ranks_max": max(int(c.shape[2]) for c in X), "graph_replay": True,
                                        "launches_per_step": plan.launches}
            plan.close()
        if "twosided" in legs:
            for prec in ("mixed", "fp64"):
                ms, X = timed(lambda s: tt.tt_round_twosided(Yd, ell, rhos=rho, seed=s, precision=prec), 2, 1)
                variants["twosided_" + prec] = {"ms_per_step": ms, "eager": True}
        if "det" in legs and not a.no_det:
            ms, Xd = timed(lambda s: tt.tt_round_det(Yd, tol=tol), 1, 0)
            dr = [int(Xd[0].shape[0])] + [int(c.shape[2]) for c in Xd]
            S = [1] + [K * R] * (N - 1) + [1]
            S[1] = min(S[1], dims[0])
            for n in range(N - 1, 0, -1):
                S[n] = min(S[n], dims[n] * S[n + 1])
            dfl = flops_det(dims, S, dr)
            variants["det_fp64"] = {"ms_per_step": ms, "tflops_alg": dfl / (ms * 1e-3) / 1e12,
                                    "gflop_alg": dfl / 1e9, "output_ranks_max": max(dr)}
            if "rand_mixed" in variants:
                variants["det_fp64"]["rand_mixed_speedup"] = ms / variants["rand_mixed"]["ms_per_step"]
    head = variants.get("rand_mixed") or variants.get("rand_fp64")
    t = head["ms_per_step"] if head else float("nan")
    print(json.dumps({"metric": METRIC.replace("sum of 20 TTs, N=50", "sum of 30 TTs, N=30, I=256"),
                      "value": flops / (t * 1e-3) / 1e12 if head else None, "unit": "TFLOP/s", "n_gpus": 1, "steps": a.steps,
                      "warmup": a.warmup, "ms_per_step": t if head else None, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": dict(LARGE, precision="mixed", l2="inputs (0.74 GB) exceed L2",
                                     algorithmic_gflop_per_step=flops / 1e9,
                                     execution="captured CUDA graph per precision, replayed per step"),
                      "clocks": clk.summary(), "variants": variants}), flush=True)


def main():
    a = parse()
    if a.oracle_sample:
        Ys = load_workload(replica_seed(0))
        t0 = time.perf_counter()
        _oracle_rounding(Ys)
        print(json.dumps({"seconds": time.perf_counter() - t0}))
        return
    if a.impl == "reference":
        run_reference(a)
    elif a.config == "batched":
        run_batched(a)
    elif a.config == "large":
        run_large(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
