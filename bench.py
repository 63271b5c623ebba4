"""Throughput of the AeroSketch update path (persistent setting) on GB300.

One step = one call of sketch_update on a block of rows of the synthetic
stream (d = 4096, l = 1024, rank-200 power-law signal plus noise), i.e. every
row of the block goes through Algorithm 8 + Algorithm 4: threshold, insert,
FD shrink when the buffer is full, power-iteration gate, simultaneous
iteration, snapshot and residual.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  Under torchrun (N > 1) every rank runs an independent
sketch of its own stream (a single stream does not shard: each row's gate
depends on the whole prefix), rank 0 prints, value = rows of all ranks / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "rows/s of sketch_update at the stated cov-err (persistent AeroSketch)"
WORKLOADS = {
    "tight_d4096_l1024": dict(d=4096, ell=1024, r=200, spectrum="powerlaw", n=1_000_000),
    "small_d256_l32": dict(d=256, ell=32, r=20, spectrum="geometric", n=10_000),
}
FP32_SIMT_LANES_PER_SM = 128   # FP32 FMA lanes per SM
N_SM = 152
FP64_NOMINAL_TFLOPS = 1.25
# FP32 instructions of one df64 multiply-add (df_fma: TwoProduct 2, TwoSum 6,
# three corrections 3, FastTwoSum renormalisation 3, one add 1): the df64
# eigensolver's peak is the FP32 issue rate x 2 flop / this count
DF64_FP32_OPS_PER_FMA = 15
# DRAM traffic per launch from one ncu capture of the kernel as it stands
# (launch 781 of batch_tc in `python bench.py --steps 1 --warmup 3 --forms
# bf16x6 --no-cpu-baseline --no-err --no-e2e`, kpad = 1792; summary under
# profiles/), as the ratio of the measured dram__bytes_read.sum +
# dram__bytes_write.sum to that launch's algorithmic bytes (G's two BF16
# levels read once, 4 kpad^2).  A launch's traffic grows with kpad^2 like its
# algorithmic bytes, so the line's traffic is this ratio times the mean
# algorithmic bytes of the timed launches.  Set to None when the kernel changes.
TRAFFIC_RATIO = {"batch_tc": (13.152e6 + 0.199424e6) / (4.0 * 1792 ** 2)}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows: list[list[str]] = []
        self._stop = threading.Event()
        self._t = threading.Thread(target=self._run, daemon=True)

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.rows.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self) -> dict:
        sm = [float(r[0]) for r in self.rows if r and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if len(r) > 3 + k and r[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _max_over_ranks(x: float, ws: int, device) -> float:
    """The largest of the ranks' values (all ranks get it); x itself when ws == 1."""
    if ws <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def _job_rows_per_s(ws: int, steps: int, rows_per_step: int, slowest_s: float) -> float:
    """Whole-job throughput: every rank sketches its own stream of steps x
    rows_per_step rows (weak scaling), timed by the slowest rank."""
    return ws * steps * rows_per_step / slowest_s


def reference_arm(args) -> None:
    """The oracle (plain FP64 NumPy), timed on the host cores, on a bounded
    sample of the same workload: the stream is first brought to a full-size
    state by exact FD (theta = inf, no iterations), then each step times the
    oracle's AeroSketch update on `ref_rows` rows from that state."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import numpy as np

    from oracle.aerosketch import AeroSketch
    from synth import low_rank_noisy, spectrum
    w = WORKLOADS[args.workload]
    d, ell = w["d"], w["ell"]
    pre = 2 * ell + ell // 2
    per = args.ref_rows
    A = low_rank_noisy(pre + (args.warmup + args.steps) * per, d, w["r"], spectrum(w["spectrum"], w["r"]))
    A64 = A.astype(np.float64)
    fd = AeroSketch(d, ell, theta_mode="fixed", theta_fixed=float("inf")).run(A64[:pre])
    o = AeroSketch(d, ell)
    o.load_state(fd.C, fd.r, float(np.sum(A64[:pre] * A64[:pre])), pre)
    t_steps = []
    for k in range(args.warmup + args.steps):
        blk = A64[pre + k * per: pre + (k + 1) * per]
        t0 = time.perf_counter()
        o.run(blk)
        t1 = time.perf_counter()
        if k >= args.warmup:
            t_steps.append(t1 - t0)
    tot = sum(t_steps)
    value = args.steps * per / tot
    cores = os.cpu_count()
    sample = f"{per} rows/step of the d={d}, l={ell} stream after a {pre}-row exact-FD prefill"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "d": d, "ell": ell, "rows_per_step": per},
        "cpu_baseline": {"value": value, "unit": "rows/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


PRECISIONS = {"fp32": 0, "bf16": 1, "bf16x3": 2, "bf16x6": 3}
DTYPES = {f: {"fp32": "f32 products", "bf16": "bf16 tensor products (f32 acc)",
              "bf16x3": "2-level split-bf16 tensor products (f32 acc)",
              "bf16x6": "3-level split-bf16 tensor products (f32 acc)"}[f]
          + "; f64 orthonormalisation and Rayleigh-Ritz; df64 (~48-bit) eigensolver" for f in PRECISIONS}

_ORACLE_CHILD = r"""
import sys, time, numpy as np
sys.path.insert(0, sys.argv[1])
from oracle.aerosketch import AeroSketch
z = np.load(sys.argv[2])
o = AeroSketch(int(z["d"]), int(z["ell"]), stream_id=int(z["sid"]))
o.load_state(z["C0"].astype(np.float64), int(z["r0"]), float(z["fro2"]), int(z["rows"]))
blk = z["blk"].astype(np.float64)
t0 = time.perf_counter()
o.run(blk)
print(len(blk) / (time.perf_counter() - t0))
"""


def _oracle_rate(C0, r0, fro2, rows, blk, d, ell, sid, threads=None) -> float:
    """rows/s of the oracle (plain FP64 NumPy) on `blk` from the GPU's exact
    state; threads = 1 runs it in a child process with BLAS on one thread."""
    import numpy as np
    if threads is None:
        from oracle.aerosketch import AeroSketch
        o = AeroSketch(d, ell, stream_id=sid)
        o.load_state(C0.astype(np.float64), r0, fro2, rows)
        b64 = blk.astype(np.float64)
        t0 = time.perf_counter()
        o.run(b64)
        return len(b64) / (time.perf_counter() - t0)
    import tempfile
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "state.npz")
        np.savez(path, C0=C0, r0=r0, fro2=fro2, rows=rows, blk=blk, d=d, ell=ell, sid=sid)
        env = dict(os.environ)
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
            env[k] = str(threads)
        out = subprocess.run([sys.executable, "-c", _ORACLE_CHILD, ROOT, path], env=env, capture_output=True,
                             text=True, timeout=600)
        if out.returncode != 0:
            raise RuntimeError(out.stderr[-2000:])
        return float(out.stdout.strip().splitlines()[-1])


# Kernel classes timed with CUDA events inside the timed region: the candidates
# for the roofline line (the dominant single-kernel class).  Bracketing every
# class there costs host time on every block (two event records per class);
# the full class profile comes from PROFILE_STEPS further steps with every
# class timed.
TIMED_CLASSES = ["batch_tc", "batch_persist", "eig_tridiag", "eig_backtransform"]
PROFILE_STEPS = 2


def _run_form(p, torch, args, A_dev, d, ell, B, K, W, rank, local, ws, prec, want_state=False):
    """Warm up W steps, time K steps (L2 flushed between steps), then PROFILE_STEPS
    more steps with every kernel class timed; returns timings, counters, the
    timed-region profile of TIMED_CLASSES, the full class profile and
    (optionally) the state at the start of the timed region."""
    dev = A_dev.device
    stream = torch.cuda.Stream(device=dev)
    s = p.Sketch(d, ell, prec=prec, profile=True, stream=stream, stream_id=rank)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    for k in range(W):
        s.update(A_dev[k * B:(k + 1) * B])
    torch.cuda.synchronize()
    state = None
    if want_state:
        C0, r0 = s.buffer()
        state = (C0, r0, s.stats())
    st0 = s.stats()
    s.profile_select(TIMED_CLASSES)
    s.profile_reset()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    evs = []
    with ClockSampler(local) as clk:
        for k in range(W, W + K):
            with torch.cuda.stream(stream):
                flush.fill_(float(k))
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            s.update(A_dev[k * B:(k + 1) * B])
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    t_ms = _max_over_ranks(sum(step_ms), ws, dev)
    st1 = s.stats()
    prof = s.profile()
    s.profile_select(None)
    s.profile_reset()
    for k in range(W + K, W + K + PROFILE_STEPS):
        s.update(A_dev[k * B:(k + 1) * B])
    torch.cuda.synchronize()
    return dict(sketch=s, t_ms=t_ms, step_ms=step_ms, st0=st0, st1=st1, prof=prof, prof_full=s.profile(),
                st_end=s.stats(), clocks=clk.summary(),
                state=state)


ROOF_KINDS = {"batch_persist": "fp32", "batch_tc": "tensor", "eig_tridiag": "df64", "eig_backtransform": "df64",
              "ingest": "hbm"}


def roofline(prof: list, peaks: dict, peak_src: str) -> dict:
    """The roofline object of the dominant single-kernel class in a kernel-class
    profile (fd_rebuild_gemm, gram_rows_gemm, event_row_fp64 and eig_fp64 span
    several kernels and are listed in "profile" only).  `achieved` is the
    class's algorithmic work over its event-measured time; `traffic` the
    measured DRAM-to-algorithmic ratio times the mean algorithmic bytes per
    launch."""
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = N_SM * FP32_SIMT_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    single = [x for x in prof if x["name"] in ROOF_KINDS and (x["flops"] > 0 or x["bytes"] > 0)]
    top = max(single, key=lambda x: x["total_ms"])
    kind = ROOF_KINDS[top["name"]]
    if kind == "hbm":
        ach = top["bytes"] / (top["total_ms"] / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s"}
        src = f"{peak_src} copy bandwidth"
    elif kind == "tensor":
        # algorithmic flops: the power iterations of the rows whose gate the batch
        # decided and the k = 2 simultaneous iterations of the gated rows that used
        # it (2 m_t^2 per column product).  The kernel issues more: every row of the
        # block (rows after the first state-changing row are fed again), and three
        # split-BF16 passes of each product; issued_flops counts the rows, once.
        ach = top["flops"] / (top["total_ms"] / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": ach, "peak": peaks["bf16_tflops_sustained"], "unit": "TFLOP/s"}
        src = f"{peak_src} cuBLAS bf16 GEMM, sustained (the kernel runs inside a long step)"
    elif kind == "fp32":
        ach = top["flops"] / (top["total_ms"] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s"}
        src = (f"FP32 SIMT = {N_SM} SMs x {FP32_SIMT_LANES_PER_SM} FMA lanes x 2 flop x {sm_mhz:.0f} MHz "
               "(max SM clock of the measured peaks file)")
    else:
        ach = top["flops"] / (top["total_ms"] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": fp32_peak / DF64_FP32_OPS_PER_FMA, "unit": "TFLOP/s"}
        src = (f"df64 on the FP32 pipes: the FP32 SIMT peak ({fp32_peak:.1f} TFLOP/s) / "
               f"{DF64_FP32_OPS_PER_FMA} FP32 operations per df64 multiply-add")
    ratio = TRAFFIC_RATIO.get(top["name"])
    traffic = ratio * top["bytes"] / max(1, top["launches"]) if ratio is not None and top["bytes"] > 0 else None
    roof.update({"frac": roof["achieved"] / roof["peak"], "traffic": traffic,
                 "kernel": top["name"],
                 "launches": top["launches"], "avg_launch_us": 1000 * top["total_ms"] / max(1, top["launches"]),
                 "peak_source": src})
    if top.get("issued_flops", 0.0) > top["flops"] > 0.0:
        roof["issued_flops_per_launch"] = top["issued_flops"] / max(1, top["launches"])
        roof["algorithmic_flops_per_launch"] = top["flops"] / max(1, top["launches"])
        roof["issued_frac"] = top["issued_flops"] / (top["total_ms"] / 1e3) / 1e12 / roof["peak"]
    return roof


def our_arm(args) -> None:
    import numpy as np
    import torch

    import paper_2601_02019_gb300 as p
    from synth import low_rank_noisy, spectrum

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = WORKLOADS[args.workload]
    d, ell, B = w["d"], w["ell"], args.rows_per_step
    K, W = args.steps, args.warmup
    ntot = (W + K + PROFILE_STEPS) * B
    A = low_rank_noisy(ntot, d, w["r"], spectrum(w["spectrum"], w["r"]), stream=rank)
    A_dev = torch.from_numpy(A).to(dev)
    forms = [f for f in args.forms.split(",") if f]
    head = args.prec
    if head not in forms:
        forms.append(head)
    runs = {}
    for f in forms:
        runs[f] = _run_form(p, torch, args, A_dev, d, ell, B, K, W, rank, local, ws, PRECISIONS[f],
                            want_state=(f == head))
    hr = runs[head]
    value = _job_rows_per_s(ws, K, B, hr["t_ms"] / 1000.0)

    peaks, peak_src = _peaks()
    prof = hr["prof"]
    prof_full = hr["prof_full"]
    tot_prof = sum(x["total_ms"] for x in prof_full if x["name"] != "eig_fp64") or 1.0
    roof = roofline(prof, peaks, peak_src)

    # end to end through the C ABI from pinned host memory (host->device copy
    # inside the timed region, device->host read of the counters each step)
    e2e = None
    if not args.no_e2e:
        A_pin = torch.from_numpy(A).pin_memory()
        s2 = p.Sketch(d, ell, prec=PRECISIONS[head], stream_id=rank)
        for k in range(W):
            s2.update(A_pin[k * B:(k + 1) * B].numpy())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(W, W + K):
            s2.update(A_pin[k * B:(k + 1) * B].numpy())
            s2.stats()
        e2e_s = _max_over_ranks(time.perf_counter() - t0, ws, dev)
        e2e = {"value": _job_rows_per_s(ws, K, B, e2e_s), "unit": "rows/s", "h2d_bytes_per_step": B * d * 4,
               "d2h_bytes_per_step": 112}

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            C0, r0, st0 = hr["state"]
            S = args.cpu_rows
            blk = A[W * B: W * B + S]
            rate = _oracle_rate(C0, r0, st0["fro2"], st0["rows"], blk, d, ell, rank, threads=None)
            cpu = {"value": rate, "unit": "rows/s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"first {S} rows of the timed region, from the GPU's exact state at its start"}
            if args.cpu_rows_1core > 0:
                S1 = min(S, args.cpu_rows_1core)
                rate1 = _oracle_rate(C0, r0, st0["fro2"], st0["rows"], blk[:S1], d, ell, rank, threads=1)
                cpu["single_core"] = {"value": rate1, "unit": "rows/s", "cores": 1,
                                      "sample": f"first {S1} rows of the same sample, BLAS on one thread "
                                                "(the paper's single-core setting)"}
        forms_out = {}
        errs = {}
        if not args.no_err:
            from oracle.metric import cov_err, gram
            AtA = gram(A)
        for f, r in runs.items():
            fo = {"rows_per_s": ws * K * B / (r["t_ms"] / 1000.0), "ms_per_step": r["t_ms"] / K,
                  "shrinks": r["st1"]["shrinks"] - r["st0"]["shrinks"], "dumps": r["st1"]["dumps"] - r["st0"]["dumps"],
                  "gpu_launches": int(r["st1"]["kernel_launches"] - r["st0"]["kernel_launches"])}
            if not args.no_err:
                errs[f] = cov_err(A, r["sketch"].query(), AtA)
                fo["cov_err"] = errs[f]
            forms_out[f] = fo
        if errs and "fp32" in errs:
            for f in forms_out:
                forms_out[f]["cov_err_rel_to_fp32"] = abs(errs[f] - errs["fp32"]) / errs["fp32"]
        out = {
            "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": ws, "steps": K, "warmup": W,
            "ms_per_step": hr["t_ms"] / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32 products", "bf16": "bf16 tensor products (f32 acc)",
                      "bf16x3": "2-level split-bf16 tensor products (f32 acc)",
                      "bf16x6": "3-level split-bf16 tensor products (f32 acc)"}[head]
                     + "; f64 orthonormalisation and Rayleigh-Ritz; df64 (~48-bit) eigensolver",
            "data": "synthetic",
            "config": {"workload": args.workload, "d": d, "ell": ell, "rows_per_step": B, "precision": head,
                       "timed_rows": f"{W * B}..{(W + K) * B - 1} of the stream (after {W * B} warm-up rows)",
                       "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{ws}"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": forms_out[head]["gpu_launches"],
            "clocks": hr["clocks"],
            "profile": [{"kernel": x["name"], "launches": x["launches"], "ms": round(x["total_ms"], 3),
                         "share": round(x["total_ms"] / tot_prof, 4)} for x in prof_full],
            "profile_note": (f"the {PROFILE_STEPS} steps after the timed region with every kernel class timed "
                             "(inside the timed region only " + ", ".join(TIMED_CLASSES) + " are); share of "
                             "the summed class times; eig_fp64 is the sum of the three eig_* phases"),
            "forms": forms_out,
            "accuracy": ({"cov_err": errs.get(head), "bound_eps": 2.0 / ell, "rows": int(hr["st_end"]["rows"])}
                         if errs else None),
        }
        print(json.dumps(out))
    if ws > 1:
        torch.distributed.destroy_process_group()


# ---- the survey's next rows: P5 sites (Algorithm 10) and the sliding window
# (Algorithm 6), each measured on its own line with its own workload --------
EXTRA = {
    # C3 reduced to 16 sites so a run takes minutes: d = 512, l = 64, shared
    # rank 50 (sigma_i = 10 * 0.85^i) plus a rank-5 site part (5 * 0.85^i)
    "p5_d512_l64_m16": dict(d=512, ell=64, m=16, rows_per_site=256),
    # C3 at its stated 512 sites (d = 512, l = 64; the same rows), 64 rows per
    # site per synchronous round, a bounded number of rounds of the 2*10^4
    "p5_d512_l64_m512": dict(d=512, ell=64, m=512, rows_per_site=64),
    # C2 with the window reduced to 16384 rows (the timed steps then run with
    # a full window): d = 1024, l = 128, rows as the d = 256 workload
    "sliding_d1024_l128_N16384": dict(d=1024, ell=128, N=16384, rows_per_step=4096),
    # C2 at its stated window N = 10^5 (d = 1024, l = 128, rows as the d = 256
    # workload), the basis rotated by a Givens sweep every 250,000 rows: a
    # segment of the 2*10^6-row stream that fills the window with rows of the
    # old basis and times the steps right after the rotation at row 250,000
    "sliding_d1024_l128_N100000_drift": dict(d=1024, ell=128, N=100_000, rows_per_step=4096, drift=250_000),
    # C4: 2000 sessions (d = round8(exp U[ln 256, ln 8192]), l in {32..512}
    # clamped to d/2), batches of round(exp U[0, ln 4096]) rows for uniformly
    # chosen sessions; a saturation phase measures capacity, then Poisson
    # arrivals at three fractions of it give the latency percentiles
    "serve_c4_s2000": dict(sessions=2000, requests=2000, loads=(0.5, 0.8, 0.95), pool_rows=4096, dmax=8192),
    # many sketches in one launch: the C3 rows of 16 sites fed through
    # sketch_update_grouped (each sketch on its own worker thread, the launch
    # combiner grouping their batched iterations), beside sketch_update_many
    # (each sketch independent on a worker thread)
    "group_d512_l64_m16": dict(d=512, ell=64, m=16, rows_per_site=256),
}


def _p5_rows(w, rounds, seed):
    from synth import basis, low_rank_noisy
    d, m, b = w["d"], w["m"], w["rows_per_site"]
    V = basis(d, 50, seed=seed)
    sig = 10.0 * 0.85 ** np.arange(50)
    sig5 = 5.0 * 0.85 ** np.arange(5)
    out = []
    ch = 4096 if m <= 16 else max(1, rounds * b)   # many sites: draw only the rows used
    for j in range(m):
        shared = low_rank_noisy(rounds * b, d, 50, sig, noise=0.01, seed=seed, stream=2 * j + 1, V=V, chunk=ch)
        own = low_rank_noisy(rounds * b, d, 5, sig5, noise=0.0, seed=seed, stream=2 * j + 2,
                             V=basis(d, 5, seed=seed, stream=j + 1), chunk=ch)
        out.append((shared + own).astype(np.float32))
    return out


def serve_arm(args) -> None:
    """The serving runtime on the C4 session mix: sessions admitted by their
    footprint, requests (host rows, pinned) submitted by a host loop and run
    with continuous batching; every phase is timed from its first submission
    to its last completion."""
    import time

    import torch

    import paper_2601_02019_gb300 as p
    from synth import low_rank_noisy, serving_mix, spectrum
    w = EXTRA[args.workload]
    S, R, dmax, P = w["sessions"], w["requests"], w["dmax"], w["pool_rows"]
    torch.cuda.set_device(0)
    mix = serving_mix(S, R, seed=0)
    # one pinned pool of rows in d = 8192 (rank 20, sigma_i = 10 * 0.9^i);
    # a request of session s with b rows reads b consecutive rows' first d_s
    # columns (row stride 8192)
    pool = torch.from_numpy(low_rank_noisy(P, dmax, 20, spectrum("geometric", 20), seed=0)).pin_memory()
    g = np.random.default_rng(1)
    offs = g.integers(0, P - mix["rows"] + 1)
    phases = 1 + len(w["loads"])
    planned = np.zeros(S)
    np.add.at(planned, mix["session"], mix["rows"])
    sv = p.Server()
    t0 = time.perf_counter()
    sid, refused = {}, 0
    for s in range(S):
        try:
            sid[s] = sv.open(int(mix["d"][s]), int(mix["ell"][s]), stream_id=s, prec=PRECISIONS[args.prec],
                             mass_ratio=max(1.0, 10.0 * (phases * planned[s] + args.warmup * 64)))
        except p.AeroSketchError as e:
            if "AS_EBUSY" not in str(e):
                raise
            refused += 1
    open_s = time.perf_counter() - t0
    reqs = [(int(mix["session"][k]), int(mix["rows"][k]), int(offs[k])) for k in range(R)]
    reqs = [r for r in reqs if r[0] in sid]

    def view(s, b, off):
        return pool[off:off + b, : int(mix["d"][s])]

    for k in range(args.warmup):                                   # warm-up requests
        s, b, off = reqs[k % len(reqs)]
        sv.submit(sid[s], view(s, min(b, 64), off))
    sv.drain()

    def phase(lam):
        sv.reset_stats()
        if lam is None:
            for s, b, off in reqs:
                sv.submit(sid[s], view(s, b, off))
        else:
            arr = np.cumsum(np.random.default_rng(2).exponential(1.0 / lam, len(reqs)))
            t_start = time.perf_counter()
            for (s, b, off), a in zip(reqs, arr):
                dt = t_start + a - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                sv.submit(sid[s], view(s, b, off))
        sv.drain()
        st = sv.stats()
        return {"rows_per_s": st["rows_done"] / st["span_s"], "requests_per_s": st["requests_done"] / st["span_s"],
                "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"], "span_s": st["span_s"],
                "failed": st["requests_failed"]}

    with ClockSampler(0) as clk:
        sat = phase(None)
        sweep = []
        for f in w["loads"]:
            lam = f * sat["requests_per_s"]
            r = phase(lam)
            r["offered_requests_per_s"] = lam
            r["load"] = f
            sweep.append(r)
    fp = sv.stats()["footprint_bytes"]
    sv.close()
    print(json.dumps({
        "metric": "rows/s of the serving loop at saturation (host-fed requests)", "value": sat["rows_per_s"],
        "unit": "rows/s", "n_gpus": 1, "steps": phases, "warmup": args.warmup,
        "ms_per_step": 1e3 * sat["span_s"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32 products", "bf16": "bf16 tensor products (f32 acc)",
                  "bf16x3": "2-level split-bf16 tensor products (f32 acc)",
                  "bf16x6": "3-level split-bf16 tensor products (f32 acc)"}[args.prec]
                 + "; f64 orthonormalisation and Rayleigh-Ritz; df64 (~48-bit) eigensolver", "data": "synthetic",
        "config": {"workload": args.workload, "precision": args.prec, "sessions": S, "admitted": len(sid),
                   "refused": refused,
                   "requests_per_phase": len(reqs), "rows_per_phase": int(sum(b for _, b, _ in reqs)),
                   "footprint_GB": fp / 1e9, "open_s": open_s, "workers": 16,
                   "l2": "per-session state re-read from HBM; rows copied from pinned host memory per request"},
        "saturation": sat, "load_sweep": sweep, "clocks": clk.summary(),
    }))


def group_arm(args) -> None:
    """sketch_update_grouped over 16 sketches (each on its own worker thread,
    their batched iterations grouped by the launch combiner) and, on fresh sketches, the same rows through sketch_update_many
    (each sketch progressing independently on a worker thread).
    Both calls return after their work is done, so each step is timed on the
    host clock with the device synchronised on both sides."""
    import torch

    import paper_2601_02019_gb300 as p
    w = EXTRA[args.workload]
    K, W = args.steps, args.warmup
    torch.cuda.set_device(0)
    rows = [torch.from_numpy(x).cuda() for x in _p5_rows(w, W + K, seed=0)]
    b, m, d, ell = w["rows_per_site"], w["m"], w["d"], w["ell"]

    def make():
        return [p.Sketch(d, ell, stream_id=j, stream=torch.cuda.Stream()) for j in range(m)]

    def grouped(sks, k):
        p.update_grouped(sks, [x[k * b:(k + 1) * b] for x in rows])

    def threaded(sks, k):
        p.update_many(sks, [x[k * b:(k + 1) * b] for x in rows])

    out = {}
    with ClockSampler(0) as clk:
        for name, fn in (("grouped", grouped), ("independent", threaded)):
            sks = make()
            for k in range(W):
                fn(sks, k)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for k in range(W, W + K):
                fn(sks, k)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            out[name] = {"rows_per_s": K * b * m / dt, "ms_per_step": 1e3 * dt / K,
                         "grouped_batches": int(sum(x.stats()["grouped_batches"] for x in sks))}
    print(json.dumps({
        "metric": "rows/s of sketch_update_grouped (16 sketches, grouped launches)",
        "value": out["grouped"]["rows_per_s"],
        "unit": "rows/s", "n_gpus": 1, "steps": K, "warmup": W, "ms_per_step": out["grouped"]["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 products; f64 orthonormalisation and Rayleigh-Ritz; df64 (~48-bit) eigensolver",
        "data": "synthetic",
        "config": {"workload": args.workload, "d": d, "ell": ell, "sketches": m, "rows_per_sketch_per_step": b,
                   "timing": "host clock around synchronous calls, device synchronised on both sides",
                   "l2": "per-sketch state far below L2; rows resident in HBM"},
        "modes": out, "clocks": clk.summary(),
    }))


def extra_arm(args) -> None:
    import torch

    import paper_2601_02019_gb300 as p
    from synth import low_rank_noisy, spectrum
    w = EXTRA[args.workload]
    K, W = args.steps, args.warmup
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    if args.workload.startswith("p5"):
        rows = _p5_rows(w, W + K, seed=0)
        b, m = w["rows_per_site"], w["m"]
        g = p.P5(w["d"], w["ell"], m, stream=stream, prec=PRECISIONS[args.prec])
        step_rows = b * m

        def step(k):
            g.round([x[k * b:(k + 1) * b] for x in rows])
        cfg = {"workload": args.workload, "d": w["d"], "ell": w["ell"], "sites": m, "rows_per_site_per_round": b,
               "l2": "per-site state far below L2; inputs staged from host each round"}
    else:
        d, ell, N, B = w["d"], w["ell"], w["N"], w["rows_per_step"]
        drift = w.get("drift")
        if drift:
            # rows [s0, s0 + N) fill the window before the warm-up steps; the timed
            # steps start at the rotation (row `drift`)
            from synth import drifting_rows
            s0 = drift - N - W * B
            pre = N
            A = drifting_rows(pre + (W + K) * B, d, 20, spectrum("geometric", 20), period=drift, seed=0, start=s0)
        else:
            pre = 0
            A = low_rank_noisy((W + K) * B, d, 20, spectrum("geometric", 20), seed=0)
        A *= 1.0 / np.sqrt(np.min(np.sum(A.astype(np.float64) ** 2, axis=1)))   # ||a||^2 >= 1 (the model)
        A = A.astype(np.float32)
        R = 2.0 ** np.ceil(np.log2(np.max(np.sum(A.astype(np.float64) ** 2, axis=1))))
        A_dev = torch.from_numpy(A).cuda()
        g = p.SlidingWindow(d, ell, N, R, stream=stream, prec=PRECISIONS[args.prec])
        step_rows = B
        for t0 in range(0, pre, B):
            g.update(A_dev[t0:min(pre, t0 + B)])

        def step(k):
            g.update(A_dev[pre + k * B:pre + (k + 1) * B])
        cfg = {"workload": args.workload, "d": d, "ell": ell, "window": N, "rows_per_step": B, "R": R,
               "levels": g.stats()["levels"], "l2": "rows resident in HBM; per-level state re-read each step"}
        if drift:
            cfg.update({"drift_every_rows": drift, "stream_rows": f"{s0}..{s0 + pre + (W + K) * B - 1}",
                        "timed_rows": f"{drift}..{drift + K * B - 1} (the first {K * B} rows after the rotation)"})
    for k in range(W):
        step(k)
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(W, W + K):
            step(k)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    value = K * step_rows / (ms / 1e3)
    print(json.dumps({
        "metric": "rows/s of the " + ("P5 round (all sites)" if args.workload.startswith("p5")
                                      else "sliding-window update"),
        "value": value, "unit": "rows/s", "n_gpus": 1, "steps": K, "warmup": W, "ms_per_step": ms / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.prec],
        "data": "synthetic", "config": dict(cfg, precision=args.prec), "clocks": clk.summary(),
    }))


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tight_d4096_l1024", choices=sorted(WORKLOADS) + sorted(EXTRA))
    ap.add_argument("--rows-per-step", type=int, default=1024)
    ap.add_argument("--cpu-rows", type=int, default=48)
    ap.add_argument("--cpu-rows-1core", type=int, default=8,
                    help="rows of the CPU-baseline sample also timed with BLAS on one thread (0: skip)")
    ap.add_argument("--ref-rows", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-err", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--prec", default="bf16x6", choices=sorted(PRECISIONS))
    ap.add_argument("--forms", default="fp32,bf16,bf16x3,bf16x6",
                    help="precision forms measured side by side (comma-separated)")
    args = ap.parse_args()
    if args.workload in EXTRA:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle arm is timed on the headline workload"}))
        elif args.workload.startswith("serve"):
            serve_arm(args)
        elif args.workload.startswith("group"):
            group_arm(args)
        else:
            extra_arm(args)
    elif args.impl == "reference":
        reference_arm(args)
    else:
        our_arm(args)


if __name__ == "__main__":
    main()
