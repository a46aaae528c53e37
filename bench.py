"""Benchmark of the FastKroneckerRegression hot path on GB300.

One step = one complete Alg. 2 solve through the C ABI: leverage scores and CDFs, Philox
sampling, grouping, gather of b, Richardson iterations until the (1+eps)-aware stopping
rule holds (the proof of Thm 4.5 with Lemma 4.2), and the FP64 final check of the sampled
objective. The default workload is the largest single-GPU configuration: N = 3, A(n)
1024 x 64 Gaussian with 10% of the rows scaled by 20 (high-leverage outliers), b a
rank-(64,64,64) Tucker tensor plus 1% relative noise stored dense (1024^3 FP32, 4 GB),
eps = 0.05, s = ceil(4 R ln R / eps) = 261,654,300 draws, FP32 contractions. Inputs are
generated on the device from a seed (synthetic; the paper's data are not used).

`value` times solves on inputs resident in HBM; `e2e` times the same C-ABI call with
page-locked host buffers (host <-> device traffic inside the timed region). Every timed solve
is certified afterwards: f(x) <= (1 + eps) OPT, with f(x) the library's FP64 full objective
and OPT the oracle's FP64 closed form (x* = (A(1)^+ (x) ... (x) A(N)^+) b), computed once on
the host.

Multi-GPU: the path is run as independent replicas (one solve per rank, no data exchange;
weak scaling).
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "kron_n3_1024x64_outliers": dict(I=[1024, 1024, 1024], R=[64, 64, 64], dist="outliers", noise_rel=0.01,
                                     b_kind="tucker", tucker_rank=[64, 64, 64], eps=0.05, lam=0.0, seed=2210,
                                     solve_seed=1),
    "kron_n3_512x32_lognormal": dict(I=[512, 512, 512], R=[32, 32, 32], dist="lognormal_rows", noise_rel=0.05,
                                     b_kind="kron", tucker_rank=None, eps=0.1, lam=0.0, seed=2209, solve_seed=1),
}
METRIC = "sampled rows/s (draws of one time-to-(1+eps) solve per second)"
PEAKS_FALLBACK = dict(hbm_gbs=6800.0, bf16_tflops=1900.0)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"], samples=0)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return dict(sm_mhz=float(np.median(sm)) if sm else None, sm_max_mhz=max(mx) if mx else None,
                    reasons=sorted(reasons), samples=len(sm))


def make_inputs(w, seed, device):
    """The workload's factors and right-hand side (FP32, on `device`), from the seeded
    device generator (the numpy generator when no CUDA device is present)."""
    import torch

    from workloads import kron_problem, kron_problem_device

    if device != "cpu":
        p = kron_problem_device(w["I"], w["R"], dist=w["dist"], seed=seed, noise_rel=w["noise_rel"], device=device,
                                b_kind=w["b_kind"], tucker_rank=w["tucker_rank"])
        return p["As"], p["b"]
    p = kron_problem(w["I"], w["R"], dist=w["dist"], seed=seed, noise_rel=w["noise_rel"], b_kind=w["b_kind"],
                     tucker_rank=w["tucker_rank"])
    return ([torch.from_numpy(np.ascontiguousarray(A, dtype=np.float32)) for A in p["As"]],
            torch.from_numpy(np.ascontiguousarray(p["b"], dtype=np.float32)))


def dist_setup(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if args.impl != "reference" else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def _reduce(v, world, op):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(v, world):
    import torch.distributed as dist

    return _reduce(v, world, dist.ReduceOp.MAX if world > 1 else None)


def whole_job_rate(units, seconds, world):
    """Replicas run side by side: the units every rank processed over the slowest rank's time.
    Returns (rate, slowest seconds)."""
    import torch.distributed as dist

    total = _reduce(float(units), world, dist.ReduceOp.SUM if world > 1 else None)
    slowest = _reduce(float(seconds), world, dist.ReduceOp.MAX if world > 1 else None)
    return total / slowest, slowest


# ---------------------------------------------------------------------------- CPU oracle legs

def oracle_opt(As64, b64, lam):
    """OPT = f(x*) with the oracle's FP64 closed form (once per run, on the host)."""
    from oracle import kron as ko

    t0 = time.perf_counter()
    opt = ko.objective(As64, b64, ko.closed_form_ridge(As64, b64, lam), lam)
    return opt, time.perf_counter() - t0


def oracle_rows_per_s(w, As64, b32, iters, frac, call_id=0):
    """Times the oracle's Alg. 2 pipeline (tables, sampling, grouping, gather and `iters`
    FP64 Richardson iterations) on a bounded fraction of the workload's draws; returns
    (draws / second, draws, seconds)."""
    from oracle import kron as ko

    R = int(np.prod(w["R"]))
    s = max(1, int(ko.sample_count(R, w["eps"]) * frac))
    t0 = time.perf_counter()
    levs = [ko.leverage_scores(A) for A in As64]
    cdfs = [ko.cdf_table(l) for l in levs]
    probs = [ko.probabilities(l) for l in levs]
    smp = ko.draw_sample(As64, s, w["solve_seed"], call_id, cdfs=cdfs, probs=probs)
    b_s = b32[smp.keys].astype(np.float64)
    ko.richardson(As64, b_s, smp, w["lam"], w["eps"], tol=0.0, max_iter=max(1, iters))
    dt = time.perf_counter() - t0
    return s / dt, s, dt


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle as it stands, on a bounded sample per step."""
    if rank != 0:
        return
    import torch

    from oracle import kron as ko

    w = WORKLOADS[args.workload]
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    As, b = make_inputs(w, w["seed"], dev)
    As64 = [A.cpu().double().numpy() for A in As]
    b32 = b.cpu().numpy()
    del As, b
    if dev != "cpu":
        torch.cuda.empty_cache()
    frac, iters = args.ref_fraction, args.ref_iters
    for k in range(args.warmup):
        oracle_rows_per_s(w, As64, b32, 1, frac / 10.0, call_id=1000 + k)
    vals, secs = [], []
    for k in range(args.steps):
        v, s, dt = oracle_rows_per_s(w, As64, b32, iters, frac, call_id=k)
        vals.append(v)
        secs.append(dt)
    value = float(np.mean(vals))
    cores = os.cpu_count()
    s_full = ko.sample_count(int(np.prod(w["R"])), w["eps"])
    sample = "%.3g of the workload's %d draws per step (%d draws), %d FP64 Richardson iteration(s)" % (
        frac, s_full, s, iters)
    line = dict(impl="reference", metric=METRIC, value=value, unit="rows/s", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1000.0 * float(np.mean(secs)), higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=args.workload, I=w["I"], R=w["R"], eps=w["eps"]),
                cpu_baseline=dict(value=value, unit="rows/s", cores=cores, kind="oracle", sample=sample),
                e2e=dict(value=value, unit="rows/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- GPU leg

def kernel_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` from the committed ncu capture at this workload
    (profiles/traffic.json), or None once the kernel's source differs from the captured one."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
        src = open(os.path.join(ROOT, rec["source"]), "rb").read()
    except (OSError, KeyError, ValueError):
        return None, None
    if hashlib.sha1(src).hexdigest() != rec["source_sha1"] or rec["workload"] != workload:
        return None, None
    return rec["dram_bytes_per_launch"], rec.get("note")


def sketch_stats(kr, As_d, b_d, s, seed, call_id, IT):
    """Distinct rows and non-empty cells of the sketch of solve `call_id`."""
    tab = kr.kron_leverage(As_d)
    sk = kr.kron_sketch(As_d, tab["cdf"], tab["prob"], b_d, s, seed, call_id)
    keys = sk.export()[0]
    sk.free()
    distinct = int(keys.numel())
    cells = int(torch_unique_count(keys // IT))
    return distinct, cells


def torch_unique_count(t):
    import torch

    return torch.unique_consecutive(t).numel()


TUCKER_WORKLOADS = {
    # Tucker ALS: 256^3 tensor of multilinear rank (16,16,16) + 1% noise, lambda = 1e-3, 10 sweeps
    "tucker_256x256x256_r16": dict(I=[256, 256, 256], R=[16, 16, 16], Rt=[16, 16, 16], noise_rel=0.01,
                                   decay=False, lam=1e-3, eps=0.1, sweeps=10, seed=11),
    # the cardiac MRI tensor's shape and rank (App. D), synthetic: Tucker tensor of twice the rank
    # with a decaying core spectrum + 10% noise, 5 sweeps
    "cardiac_mri_256x256x14x20": dict(I=[256, 256, 14, 20], R=[8, 8, 4, 4], Rt=[16, 16, 8, 8], noise_rel=0.1,
                                      decay=True, lam=1e-3, eps=0.1, sweeps=5, seed=31),
}


def run_tucker(name):
    """Sampled (Alg. 1 with Alg. 3 factor steps and Alg. 2 core steps) and exact (KronMatMul)
    TuckerALS sweeps from the same start: milliseconds per sweep (host clock around the
    synchronous calls, inputs resident) and the RRE after every sweep."""
    import torch

    import paper_2209_04876_gb300 as kr
    from workloads import tucker_tensor_device

    w = TUCKER_WORKLOADS[name]
    I, R = w["I"], w["R"]
    X = tucker_tensor_device(I, w["Rt"], seed=w["seed"], noise_rel=w["noise_rel"],
                             decay_rank=R if w["decay"] else None)

    def start():
        g = torch.Generator(device="cuda")
        g.manual_seed(w["seed"] + 1)
        As = [torch.linalg.qr(torch.randn(i, r, generator=g, device="cuda"))[0].contiguous() for i, r in zip(I, R)]
        return As, kr.kron_matmul(As, X.reshape(-1), trans=[1] * len(As))

    out = dict(I=I, R=R, lam=w["lam"], eps=w["eps"], sweeps=w["sweeps"], timing="host clock, synchronous calls")
    As, G = start()
    kr.tucker_als_exact_sweep(X, As, G, w["lam"], sweeps=1)  # warm-up
    As, G = start()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rre_e = kr.tucker_als_exact_sweep(X, As, G, w["lam"], sweeps=w["sweeps"])
    torch.cuda.synchronize()
    out["exact"] = dict(ms_per_sweep=1e3 * (time.perf_counter() - t0) / w["sweeps"], rre=rre_e)
    N = len(I)
    opts = dict(eps=w["eps"], seed=5, tol=1e-7, max_iter=300, stop_rule=kr.STOP_EPS)
    As, G = start()
    kr.tucker_als_sweep(X, As, G, w["lam"], sweeps=1, call_id=50, **opts)  # warm-up
    As, G = start()
    rre_s, t = [], 0.0
    for k in range(w["sweeps"]):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        kr.tucker_als_sweep(X, As, G, w["lam"], sweeps=1, call_id=100 + k * (N + 1), **opts)
        torch.cuda.synchronize()
        t += time.perf_counter() - t0
        rre_s.append(kr.tucker_rre(X, As, G))
    out["sampled"] = dict(ms_per_sweep=1e3 * t / w["sweeps"], rre=rre_s, stop_rule="(1+eps)-aware")
    out["rre_ratio_last"] = rre_s[-1] / rre_e[-1]
    # the same sweeps (same Philox streams) in one call: sweeps 2.. run as one CUDA graph
    As, G = start()
    torch.cuda.synchronize()
    g0 = kr.graph_count()
    t0 = time.perf_counter()
    kr.tucker_als_sweep(X, As, G, w["lam"], sweeps=w["sweeps"], call_id=100, **opts)
    torch.cuda.synchronize()
    out["sampled_one_call"] = dict(ms_per_sweep=1e3 * (time.perf_counter() - t0) / w["sweeps"],
                                   rre_last=kr.tucker_rre(X, As, G), graphs=kr.graph_count() - g0,
                                   form="sweep 1 from the host, sweeps 2.. as one CUDA graph")
    del X, As, G
    torch.cuda.empty_cache()
    return out


def run_gpu(args, rank, world, local):
    import torch

    import paper_2209_04876_gb300 as kr

    torch.cuda.set_device(local)
    w = WORKLOADS[args.workload]
    As_d, b_d = make_inputs(w, w["seed"] + rank, "cuda")
    torch.cuda.synchronize()
    eps, lam = w["eps"], w["lam"]
    solve = kr.kron_ridge if lam > 0 else kr.kron_regress
    lam_kw = dict(lam=lam) if lam > 0 else {}
    opts = dict(eps=eps, seed=w["solve_seed"], stop_rule=kr.STOP_EPS, max_iter=200, **lam_kw)
    opts_step = dict(eps=eps, seed=w["solve_seed"], tol=1e-7, max_iter=200, **lam_kw)
    # OPT from the oracle's FP64 closed form, once, on the host
    As64 = [A.cpu().double().numpy() for A in As_d]
    b32 = b_d.cpu().numpy()
    opt, opt_s = oracle_opt(As64, b32.astype(np.float64), lam)
    log("oracle OPT %.6e in %.1f s" % (opt, opt_s))
    for k in range(args.warmup):
        solve(As_d, b_d, call_id=1000 + k, **opts)
    torch.cuda.synchronize()
    # timed region: K solves on resident inputs (b is 4 GB: larger than L2 on every pass)
    kr.timing_enable(False)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    l0 = kr.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    reps, xs = [], []
    for k in range(args.steps):
        x, rep = solve(As_d, b_d, call_id=k, **opts)
        reps.append(rep)
        xs.append(x)
    ev1.record()
    torch.cuda.synchronize()
    barrier(world)
    launches = kr.launch_count() - l0
    elapsed_ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    s = reps[0]["s"]
    value, elapsed_s = whole_job_rate(args.steps * s, elapsed_ms / 1000.0, world)
    elapsed_ms = 1000.0 * elapsed_s
    # certify every timed solve against the oracle's OPT
    ratios = [kr.kron_objective(As_d, b_d, x, lam) / opt for x in xs]
    certified = all(r <= 1.0 + eps for r in ratios)
    del xs
    # the same solves with the relative-step rule (tol 1e-7), for the stopping-rule comparison
    n_step = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    step_reps = [solve(As_d, b_d, call_id=k, **opts_step)[1] for k in range(n_step)]
    e1.record()
    torch.cuda.synchronize()
    step_ms = e0.elapsed_time(e1) / n_step
    # kernel time shares and the dominant kernel's launch time: one more solve with
    # per-launch event pairs on the library's stream
    kr.timing_reset()
    kr.timing_enable(True)
    x, rep_t = solve(As_d, b_d, call_id=args.steps, **opts)
    tim = kr.timing_read()
    kr.timing_enable(False)
    # end to end through the same C-ABI call with page-locked host buffers
    As_h = [A.cpu().pin_memory() for A in As_d]
    b_h = b_d.cpu().pin_memory()
    solve(As_h, b_h, call_id=0, host_io=True, **opts)
    barrier(world)
    t0 = time.perf_counter()
    for k in range(args.steps):
        xh, rep_h = solve(As_h, b_h, call_id=k, host_io=True, **opts)
    e2e, e2e_s = whole_job_rate(args.steps * s, time.perf_counter() - t0, world)
    h2d = int(4 * rep_h["distinct"] + sum(A.numel() * 4 for A in As_h))
    d2h = int(xh.numel() * 4)
    # the same calls with all of b copied in (the library's path for b outside page-locked memory)
    kr.set_option(kr.OPT_HOST_GATHER, 0)
    solve(As_h, b_h, call_id=0, host_io=True, **opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        solve(As_h, b_h, call_id=k, host_io=True, **opts)
    e2e_copy = whole_job_rate(args.steps * s, time.perf_counter() - t0, world)[0]
    kr.set_option(kr.OPT_HOST_GATHER, 1)
    del As_h, b_h
    if rank != 0:
        return
    # Roofline of the dominant kernel of a solve, by the library's per-kind launch timing:
    # k_draw_keys (the draws, a3, with the dense grouping's per-key counts and key bitmap, a4,
    # in the same launch) or k_slab (the fused sampled products a6-a8, one launch per
    # Richardson iteration plus the final check); the other one is reported beside it.
    # Algorithmic bytes per launch, per the method's own accounting: a3 writes 4 N + 4 B per
    # draw (indices, weight) and a4 reads about three 12-byte passes per draw and writes 8 B
    # per distinct row; a6-a8 move 10 B per distinct sampled row (last-mode index, weight, b~)
    # and 2 R_N 4 B per non-empty cell (its Y row read and W row written).
    peaks, peak_kind = load_peaks()
    hbm = float(peaks["hbm_gbs"])
    peak_source = "%s copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" % peak_kind
    I, R = w["I"], w["R"]
    N = len(I)
    RT, R2 = R[-1], R[-2]
    distinct, cells = sketch_stats(kr, As_d, b_d, rep_t["s"], w["solve_seed"], args.steps, I[-1])
    alg_bytes = distinct * 10 + cells * 2 * RT * 4
    P = int(np.prod(I[:-2]))
    fused_bytes = distinct * 8 + cells * 16 + 2 * P * R2 * RT * 4
    alg_flops = distinct * 4 * RT + cells * 4 * R2 * RT
    ms_r, n_r = tim["slab"]
    t_launch = ms_r / n_r / 1000.0
    gbs = alg_bytes / t_launch / 1e9
    traffic, traffic_note = kernel_traffic("k_slab", args.workload)
    slab_roof = dict(bound="hbm", achieved=gbs, peak=hbm, unit="GB/s", frac=gbs / hbm, peak_source=peak_source,
                     traffic=traffic,
                     kernel="k_slab (fused sampled products a6-a8: last-two-mode products, residual, transpose)",
                     alg_bytes_per_launch=alg_bytes,
                     bytes_rule="10 B per distinct sampled row + 2 R_N 4 B per non-empty cell",
                     distinct_rows=distinct, nonempty_cells=cells, launches=n_r, avg_launch_ms=ms_r / n_r,
                     fused_kernel_bytes_per_launch=fused_bytes, fused_kernel_gbs=fused_bytes / t_launch / 1e9,
                     flops_per_launch=alg_flops, tflops=alg_flops / t_launch / 1e12)
    if traffic_note:
        slab_roof["traffic_note"] = traffic_note
    ms_d, n_d = tim["sample"]
    s_draws = int(rep_t["s"])
    draw_bytes = s_draws * (4 * N + 4 + 36) + distinct * 8
    t_draw = ms_d / max(n_d, 1) / 1000.0
    dtraffic, dnote = kernel_traffic("k_draw_keys", args.workload)
    draw_roof = dict(bound="hbm", achieved=draw_bytes / t_draw / 1e9, peak=hbm, unit="GB/s",
                     frac=draw_bytes / t_draw / 1e9 / hbm, peak_source=peak_source, traffic=dtraffic,
                     kernel="k_draw_keys (Philox draws from the product distribution, inverse CDF, dense "
                            "per-key counts and the key bitmap: a3 + a4 in one launch)",
                     alg_bytes_per_launch=draw_bytes,
                     bytes_rule="per draw 4 N + 4 B (a3: indices and weight) + 36 B (a4: three 12-byte passes); "
                                "8 B per distinct row",
                     draws=s_draws, distinct_rows=distinct, launches=n_d, avg_launch_ms=ms_d / max(n_d, 1),
                     draws_per_s=s_draws / t_draw)
    if dnote:
        draw_roof["traffic_note"] = dnote
    if ms_d >= ms_r:
        roof = dict(draw_roof, secondary=slab_roof)
    else:
        roof = dict(slab_roof, secondary=draw_roof)
    total_timed = sum(v[0] for v in tim.values())
    shares = {k: (round(v[0] / total_timed, 4) if total_timed else None) for k, v in tim.items()}
    mean = lambda rs, key: float(np.mean([r[key] for r in rs]))
    iters = mean(reps, "iters")
    t_iter = np.mean([r["t_ms"]["iterate"] for r in reps]) / 1000.0
    line = dict(
        metric=METRIC, value=value, unit="rows/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
        ms_per_step=elapsed_ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32",
        data="synthetic (seeded device generator: outlier factors, Tucker right-hand side + noise)",
        config=dict(workload=args.workload, I=I, R=R, eps=eps, lam=lam, s=s, parallelism="replicas",
                    stop_rule="(1+eps)-aware (theta = 0.01)",
                    l2="inputs larger than L2 (b = %d MB)" % (b32.nbytes >> 20)),
        time_to_solve_ms=elapsed_ms / args.steps, iters=iters, distinct=mean(reps, "distinct"),
        iter_rows_per_s=mean(reps, "distinct") * iters / t_iter if t_iter > 0 else None,
        approx_ratio_max=max(ratios), certified_1_plus_eps=certified, opt=opt, opt_source="oracle FP64 closed form",
        step_rule=dict(tol=1e-7, ms_per_solve=step_ms, iters=mean(step_reps, "iters")),
        roofline=dict(roof, kernel_time_shares=shares),
        e2e=dict(value=e2e, unit="rows/s", h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h,
                 b_read="in place at the sampled rows (page-locked host b mapped into the device's address space)",
                 copy_all_b=dict(value=e2e_copy, unit="rows/s",
                                 h2d_bytes_per_step=int(b32.nbytes + sum(A.numel() * 4 for A in As_d)))),
        gpu_launches=int(launches),
        clocks=dict(sm_mhz=clk["sm_mhz"], sm_max_mhz=clk["sm_max_mhz"], reasons=clk["reasons"], samples=clk["samples"]),
        phases_ms={k: float(np.mean([r["t_ms"][k] for r in reps])) for k in reps[0]["t_ms"]},
    )
    if not args.no_tucker:
        line["tucker"] = {name: run_tucker(name) for name in TUCKER_WORKLOADS}
    if not args.no_batched:
        line["batched_ridge"] = run_batched()
    if not args.no_cpu_baseline:
        it_c = max(1, min(int(round(iters)), args.cpu_iters))
        v, s_c, dt = oracle_rows_per_s(w, As64, b32, it_c, args.cpu_fraction)
        line["cpu_baseline"] = dict(
            value=v, unit="rows/s", cores=os.cpu_count(), kind="oracle",
            sample="%d of the %d draws (%.3g), full tables, grouping, gather and %d FP64 Richardson iteration(s)"
                   % (s_c, s, args.cpu_fraction, it_c), seconds=dt)
    print(json.dumps(line), flush=True)


def run_batched(problems=64, seed=4):
    """The batched-ridge workload: 64 independent N = 3 ridge problems (lambda = 1e-3, eps =
    0.1), I_n uniform in [64, 1024], R_n uniform in [4, 32], Gaussian factors, b = K x + 1%
    noise. Milliseconds per batch (host clock around synchronous calls, best of 3) for the 64
    single solves one after another, the worker-context batch, the fused batch (one CUDA graph
    for all Richardson loops) and the fused batch with the tile-budget autotuner, whose
    choices are recorded."""
    import torch

    import paper_2209_04876_gb300 as kr
    from workloads import kron_problem_device

    rng = np.random.default_rng(seed)
    probs, shapes = [], []
    for k in range(problems):
        I = [int(v) for v in rng.integers(64, 1025, size=3)]
        R = [int(v) for v in rng.integers(4, 33, size=3)]
        p = kron_problem_device(I, R, dist="gauss", seed=500 + k, noise_rel=0.01, b_kind="kron")
        probs.append((p["As"], p["b"]))
        shapes.append((I, R))
    torch.cuda.synchronize()
    lam, kw = 1e-3, dict(eps=0.1, seed=3, tol=1e-7, max_iter=300)

    def seq():
        return [kr.kron_ridge(As, b, lam, call_id=10 + p, **kw)[0] for p, (As, b) in enumerate(probs)]

    def batch():
        return kr.kron_ridge_batched(probs, lam, call_id=10, **kw)[0]

    out = dict(problems=problems, lam=lam, eps=0.1, timing="host clock, synchronous calls, best of 3")
    ref = None
    for name, fn, mode, tune in (("sequential", seq, 0, 0), ("workers", batch, 0, 0), ("fused", batch, 1, 0),
                                 ("fused_autotune", batch, 1, 1)):
        kr.set_option(kr.OPT_BATCH_MODE, mode)
        kr.set_option(kr.OPT_AUTOTUNE, tune)
        xs = fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            xs = fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        out[name + "_ms"] = 1e3 * min(ts)
        if ref is None:
            ref = xs
        elif not tune:
            out[name + "_bit_identical"] = all(torch.equal(a, b) for a, b in zip(xs, ref))
    kr.set_option(kr.OPT_BATCH_MODE, 0)
    kr.set_option(kr.OPT_AUTOTUNE, 0)
    for name in ("workers", "fused", "fused_autotune"):
        out[name + "_speedup"] = out["sequential_ms"] / out[name + "_ms"]
    out["autotune_choices"] = [dict(key=list(e["key"]), budget=e["budget"]) for e in kr.autotune_report()]
    del probs
    torch.cuda.empty_cache()
    return out


PROFILE_CASES = ("kron_rmatvec_512x512x1024_r64", "kron_n3_1024x1024x256_r64_outliers")


def run_case(name):
    """Small cases for ncu captures (a few GB on the device): three K^T z products at
    512 x 512 x 1024 with R = 64 (the tensor-core mode product), or three solves of the
    1024 x 1024 x 256, R = 64 outlier problem with a quarter of the sample count (the slab
    pass at the large workload's cell structure)."""
    import torch

    import paper_2209_04876_gb300 as kr
    from workloads import kron_problem_device

    torch.cuda.set_device(0)
    if name == "kron_rmatvec_512x512x1024_r64":
        I, R = [512, 512, 1024], [64, 64, 64]
        g = torch.Generator(device="cuda")
        g.manual_seed(1)
        As = [torch.randn(i, r, generator=g, device="cuda") for i, r in zip(I, R)]
        z = torch.randn(int(np.prod(I)), generator=g, device="cuda")
        for _ in range(3):
            y = kr.kron_matmul(As, z, trans=[1, 1, 1])
        torch.cuda.synchronize()
        print(name, "max|y| %.6g" % float(y.abs().max()))
    else:
        p = kron_problem_device([1024, 1024, 256], [64, 64, 64], dist="outliers", seed=2210, noise_rel=0.01,
                                b_kind="tucker", tucker_rank=[64, 64, 64])
        s = kr.kron_sample_count(64 ** 3, 0.05) // 4
        for k in range(3):
            _, rep = kr.kron_regress(p["As"], p["b"], eps=0.05, seed=1, call_id=k, num_samples=s,
                                     stop_rule=kr.STOP_EPS, max_iter=200)
            print(name, "iters", rep["iters"], "distinct", rep["distinct"])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=110)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="kron_n3_1024x64_outliers", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-fraction", type=float, default=0.1)
    ap.add_argument("--cpu-iters", type=int, default=2)
    ap.add_argument("--ref-fraction", type=float, default=0.001)
    ap.add_argument("--ref-iters", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tucker", action="store_true", help="skip the TuckerALS sweep timings")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-ridge timings")
    ap.add_argument("--case", choices=PROFILE_CASES, help="run one small profiling case and exit")
    args = ap.parse_args()
    if args.case:
        run_case(args.case)
        return
    rank, world, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
