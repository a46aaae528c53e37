"""Benchmark of the FastKroneckerRegression hot path on GB300.

One step = one complete Alg. 2 solve through the C ABI (leverage scores and CDFs,
Philox sampling, grouping, gather of b, Richardson iterations to the stopping
rule, FP64 final check) of the N=3 workload with 512 x 32 factors (rows scaled by
log-normal(sigma=1) weights), b = K x_true + 5% relative noise of length 512^3,
eps = 0.1, s = ceil(4 R ln R / eps) = 13,627,829 draws, FP32 contractions.
Inputs are resident in HBM for `value`; `e2e` passes host buffers through the same
C-ABI call (copies inside the timed region). Every solve is certified afterwards:
f(x) <= (1 + eps) OPT, with OPT from the exact KronMatMul solution computed by the
library.

Multi-GPU: the path is run as independent replicas (one solve per rank, no data
exchange; weak scaling).
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="kron_n3_512x32_lognormal", I=[512, 512, 512], R=[32, 32, 32], dist="lognormal_rows",
                noise_rel=0.05, eps=0.1, lam=0.0, seed=2209, solve_seed=1, call_id=0)
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
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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


def make_inputs(seed):
    from workloads import kron_problem

    w = WORKLOAD
    prob = kron_problem(w["I"], w["R"], dist=w["dist"], seed=seed, noise_rel=w["noise_rel"])
    As = [np.ascontiguousarray(A, dtype=np.float32) for A in prob["As"]]
    b = np.ascontiguousarray(prob["b"], dtype=np.float32)
    return As, b


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


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------- CPU oracle legs

def oracle_rows_per_s(As, b, gpu_iters, frac, call_id=0):
    """Times the oracle's Alg. 2 pipeline (tables, sampling, grouping, gather and
    `gpu_iters` Richardson iterations) on a bounded fraction of the workload's draws."""
    from oracle import kron as ko

    w = WORKLOAD
    R = int(np.prod(w["R"]))
    s_full = ko.sample_count(R, w["eps"])
    s = max(1, int(s_full * frac))
    As64 = [A.astype(np.float64) for A in As]
    t0 = time.perf_counter()
    levs = [ko.leverage_scores(A) for A in As64]
    cdfs = [ko.cdf_table(l) for l in levs]
    probs = [ko.probabilities(l) for l in levs]
    smp = ko.draw_sample(As64, s, w["solve_seed"], call_id, cdfs=cdfs, probs=probs)
    b_s = b[smp.keys].astype(np.float64)
    ko.richardson(As64, b_s, smp, w["lam"], w["eps"], tol=0.0, max_iter=max(1, gpu_iters))
    dt = time.perf_counter() - t0
    return s / dt, s, dt


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle as it stands, on a bounded sample per step."""
    if rank != 0:
        return
    As, b = make_inputs(WORKLOAD["seed"])
    frac = args.ref_fraction
    iters = args.ref_iters
    for _ in range(args.warmup):
        oracle_rows_per_s(As, b, 1, frac / 10.0)
    vals, secs = [], []
    for k in range(args.steps):
        v, s, dt = oracle_rows_per_s(As, b, iters, frac, call_id=k)
        vals.append(v)
        secs.append(dt)
    value = float(np.mean(vals))
    cores = os.cpu_count()
    from oracle import kron as ko

    s_full = ko.sample_count(int(np.prod(WORKLOAD["R"])), WORKLOAD["eps"])
    sample = "%.3g of the workload's %d draws per step (%d draws), %d Richardson iterations" % (
        frac, s_full, s, iters)
    line = dict(impl="reference", metric=METRIC, value=value, unit="rows/s", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1000.0 * float(np.mean(secs)), higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=WORKLOAD["name"], I=WORKLOAD["I"], R=WORKLOAD["R"], eps=WORKLOAD["eps"]),
                cpu_baseline=dict(value=value, unit="rows/s", cores=cores, kind="oracle", sample=sample),
                e2e=dict(value=value, unit="rows/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- GPU leg

def exact_opt(kr, As_d, b_d):
    """OPT = f(x*) with x* = (A1^+ (x) ... (x) AN^+) b = (x)(A^T A)^-1 . (x)A^T b via the library."""
    import torch

    KtB = kr.kron_matmul(As_d, b_d, trans=[1] * len(As_d))
    xstar = kr.kron_precond(As_d, KtB, 0.0)
    torch.cuda.synchronize()
    return kr.kron_objective(As_d, b_d, xstar, 0.0)


def slab_traffic():
    """DRAM bytes per k_slab launch from the committed ncu capture (profiles/traffic.json), or None
    once the kernel source differs from the captured one."""
    here = os.path.dirname(os.path.abspath(__file__))
    try:
        rec = json.load(open(os.path.join(here, "profiles", "traffic.json")))["k_slab"]
        src = open(os.path.join(here, rec["source"]), "rb").read()
    except (OSError, KeyError, ValueError):
        return None
    if hashlib.sha1(src).hexdigest() != rec["source_sha1"] or rec["workload"] != WORKLOAD["name"]:
        return None
    return rec["dram_bytes_per_launch"]


def nonempty_cells(kr, As_d, b_d, s, seed, call_id, IT):
    """Cells holding at least one sampled row in the sketch of solve `call_id`."""
    tab = kr.kron_leverage(As_d)
    sk = kr.kron_sketch(As_d, tab["cdf"], tab["prob"], b_d, s, seed, call_id)
    keys = sk.export()[0]
    sk.free()
    return int(np.unique(keys.cpu().numpy() // IT).shape[0])


def run_gpu(args, rank, world, local):
    import torch

    import paper_2209_04876_gb300 as kr

    torch.cuda.set_device(local)
    w = WORKLOAD
    As, b = make_inputs(w["seed"] + rank)
    As_d = [torch.from_numpy(A).cuda() for A in As]
    b_d = torch.from_numpy(b).cuda()
    opts = dict(eps=w["eps"], seed=w["solve_seed"], tol=1e-7, max_iter=200)
    torch.cuda.synchronize()
    opt = exact_opt(kr, As_d, b_d)
    # warm-up
    for k in range(args.warmup):
        kr.kron_regress(As_d, b_d, call_id=1000 + k, **opts)
    torch.cuda.synchronize()
    # timed region: K solves on resident inputs
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
        x, rep = kr.kron_regress(As_d, b_d, call_id=k, **opts)
        reps.append(rep)
        xs.append(x)
    ev1.record()
    torch.cuda.synchronize()
    barrier(world)
    launches = kr.launch_count() - l0
    elapsed_ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    elapsed_ms = max_over_ranks(elapsed_ms, world)
    s = reps[0]["s"]
    value = world * args.steps * s / (elapsed_ms / 1000.0)
    # certify every timed solve: f(x) <= (1 + eps) OPT
    ratios = [kr.kron_objective(As_d, b_d, x, 0.0) / opt for x in xs]
    certified = all(r <= 1.0 + w["eps"] for r in ratios)
    # dominant-kernel timing: one more solve with per-launch events on the library stream
    kr.timing_reset()
    kr.timing_enable(True)
    x, rep_t = kr.kron_regress(As_d, b_d, call_id=args.steps, **opts)
    tim = kr.timing_read()
    kr.timing_enable(False)
    # end to end through the same C-ABI call with host buffers (pinned)
    As_h = [torch.from_numpy(A).pin_memory() for A in As]
    b_h = torch.from_numpy(b).pin_memory()
    kr.kron_regress(As_h, b_h, call_id=0, host_io=True, **opts)
    barrier(world)
    t0 = time.perf_counter()
    for k in range(args.steps):
        xh, _ = kr.kron_regress(As_h, b_h, call_id=k, host_io=True, **opts)
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, world)
    e2e = world * args.steps * s / e2e_s
    # the same calls with all of b copied in (the library's path for b outside page-locked memory)
    kr.set_option(kr.OPT_HOST_GATHER, 0)
    kr.kron_regress(As_h, b_h, call_id=0, host_io=True, **opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        xc, rep_c = kr.kron_regress(As_h, b_h, call_id=k, host_io=True, **opts)
    e2e_copy = world * args.steps * s / max_over_ranks(time.perf_counter() - t0, world)
    kr.set_option(kr.OPT_HOST_GATHER, 1)
    # the timed calls read b (page-locked) in place at the sampled rows: 4 B per distinct row
    _, rep_h = kr.kron_regress(As_h, b_h, call_id=args.steps - 1, host_io=True, **opts)
    h2d = int(4 * rep_h["distinct"] + sum(A.nbytes for A in As))
    d2h = int(xh.numel() * 4)
    if rank != 0:
        return
    # roofline of the dominant kernel
    peaks, peak_kind = load_peaks()
    hbm = float(peaks["hbm_gbs"])
    I, R = w["I"], w["R"]
    ncell = int(np.prod(I[:-1]))
    RT, R2 = R[-1], R[-2]
    distinct = rep_t["distinct"]
    if tim["slab"][1]:
        # fused slab pass: per distinct row 8 B and 4 R_N flops (dot + axpy); per non-empty
        # cell a 16 B descriptor and 4 R_{N-1} R_N flops (its Y row and its share of Z);
        # X1 read and Z written once (P x R_{N-1} x R_N floats each)
        nact = nonempty_cells(kr, As_d, b_d, rep_t["s"], w["solve_seed"], args.steps, I[-1])
        P = int(np.prod(I[:-2]))
        alg_bytes = distinct * 8 + nact * 16 + 2 * P * R2 * RT * 4
        alg_flops = distinct * 4 * RT + nact * 4 * R2 * RT
        ms_r, n_r = tim["slab"]
        kname = "k_slab (fused last-two-mode products + sampled residual, a6-a8)"
    else:
        # per-cell residual pass: per distinct row 8 B, per cell 8 R_N + 12 B
        nact = None
        alg_bytes = distinct * 8 + ncell * (8 * RT + 12)
        alg_flops = distinct * 4 * RT
        ms_r, n_r = tim["resid"]
        kname = "k_resid (sampled residual + transpose, a7+a8)"
    t_launch = ms_r / n_r / 1000.0 if n_r else None
    gbs = alg_bytes / t_launch / 1e9 if n_r else None
    tflops = alg_flops / t_launch / 1e12 if n_r else None
    # FP32 FMA roof: 152 SMs x 128 lanes x 2 flops x the maximum SM clock
    alu_peak = 152 * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    if n_r and tflops / alu_peak > gbs / hbm:
        roof = dict(bound="alu", achieved=tflops, peak=alu_peak, unit="TFLOP/s", frac=tflops / alu_peak,
                    peak_source="FP32 FMA: 152 SMs x 128 lanes x 2 x %.0f MHz" % float(peaks.get("sm_max_mhz", 2070.0)),
                    hbm_gbs=gbs, hbm_frac=gbs / hbm)
    else:
        roof = dict(bound="hbm", achieved=gbs, peak=hbm, unit="GB/s", frac=(gbs / hbm if gbs else None),
                    peak_source=peak_kind, alu_tflops=tflops, alu_frac=(tflops / alu_peak if tflops else None))
    roof.update(kernel=kname, traffic=slab_traffic() if tim["slab"][1] else None, alg_bytes_per_launch=alg_bytes,
                alg_flops_per_launch=alg_flops, nonempty_cells=nact, avg_launch_ms=(ms_r / n_r if n_r else None))
    total_timed = sum(v[0] for v in tim.values())
    shares = {k: (round(v[0] / total_timed, 4) if total_timed else None) for k, v in tim.items()}
    mean = lambda key: float(np.mean([r[key] for r in reps]))
    line = dict(
        metric=METRIC, value=value, unit="rows/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
        ms_per_step=elapsed_ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32",
        data="synthetic",
        config=dict(workload=w["name"], I=w["I"], R=w["R"], eps=w["eps"], s=s, parallelism="replicas",
                    l2="inputs larger than L2 (b = %d MB)" % (b.nbytes >> 20)),
        time_to_solve_ms=elapsed_ms / args.steps,
        iters=mean("iters"), distinct=mean("distinct"),
        iter_rows_per_s=mean("distinct") * mean("iters") / (mean("iters") and np.mean([r["t_ms"]["iterate"] for r in reps]) / 1000.0),
        approx_ratio_max=max(ratios), certified_1_plus_eps=certified,
        roofline=dict(roof, kernel_time_shares=shares),
        e2e=dict(value=e2e, unit="rows/s", h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h,
                 b_read="in place at the sampled rows (page-locked host b mapped into the device's address space)",
                 copy_all_b=dict(value=e2e_copy, unit="rows/s", h2d_bytes_per_step=int(b.nbytes + sum(A.nbytes for A in As)))),
        gpu_launches=int(launches),
        clocks=dict(sm_mhz=clk["sm_mhz"], sm_max_mhz=clk["sm_max_mhz"], reasons=clk["reasons"]),
        phases_ms={k: float(np.mean([r["t_ms"][k] for r in reps])) for k in reps[0]["t_ms"]},
    )
    if not args.no_cpu_baseline:
        v, s_c, dt = oracle_rows_per_s(As, b, int(round(mean("iters"))), args.cpu_fraction)
        line["cpu_baseline"] = dict(
            value=v, unit="rows/s", cores=os.cpu_count(), kind="oracle",
            sample="%d of the %d draws (%.3g), full tables, grouping, gather and %d FP64 Richardson iterations"
                   % (s_c, s, args.cpu_fraction, int(round(mean("iters")))), seconds=dt)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-fraction", type=float, default=0.1)
    ap.add_argument("--ref-fraction", type=float, default=0.01)
    ap.add_argument("--ref-iters", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
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
