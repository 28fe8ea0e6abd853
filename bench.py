#!/usr/bin/env python
"""Walker-slices/s of the ph-FT-AFQMC slice path on one GB300.

Workload: UEG N=66 (33 up, 33 down), M=257 plane waves, r_s=1, Theta=0.0625,
dtau=0.025 (n=348 slices), 1024 walkers, fields x ~ N(0,1) from a seeded
Philox stream (synthetic).  One *step* is one stabilisation block: s=5 slices
of the whole slice path for every walker (force bias, HS fields, B applied
to the chain, one QRCP, G(tau) and ln det per slice, phaseless weights).  The
timed region also contains one evaluation of the estimators (E, N), i.e.
more estimator work than the path needs (one per 348 slices).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
    python bench.py --impl reference ...   (the CPU oracle on the host cores)

Multi-GPU (torchrun): independent replicas with different seeds, no
collective on the data path; value = walker-slices of all ranks / max time.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synthetic_inputs import WORKLOADS, gaussian_fields  # noqa: E402

METRIC = "walker-slices/sec at M=257 (mixed vs FP64, same GB300) at ≤1e-5 Ha/e error"
WORKLOAD = "ueg_n66_m257"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 FMA pipe: 152 SMs x 2 FP64 FMA/clk/SM x 2 flop x 2.07 GHz (nominal
# 1.25 TFLOP/s for this part); a register-loop FMA probe measured 1.20.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--walkers", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-sample", nargs=2, type=int, default=None, metavar=("WALKERS", "SLICES"),
                    help=argparse.SUPPRESS)
    return ap.parse_args()


# ---------------------------------------------------------------- oracle timing
def oracle_sample(walkers, slices):
    """Time the CPU oracle on `walkers` walkers x `slices` slices of the
    workload (run in a child process with the BLAS thread count set)."""
    from oracle import afqmc
    from oracle.ueg import UEG
    c = WORKLOADS[WORKLOAD]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    f = gaussian_fields(c["seed"], slices, walkers, s.N_alpha)
    t0 = time.perf_counter()
    afqmc.run(s, f, afqmc.Options(), n_slices=slices, want_estimator=False)
    dt = time.perf_counter() - t0
    print(json.dumps({"seconds": dt, "walker_slices": walkers * slices}))


def run_oracle_child(walkers, slices, threads):
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    env["CUDA_VISIBLE_DEVICES"] = ""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", str(walkers), str(slices)],
                       capture_output=True, text=True, env=env, cwd=ROOT, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline(walkers=6, slices=5):
    cores = os.cpu_count() or 1
    res = run_oracle_child(walkers, slices, cores)
    return {"value": res["walker_slices"] / res["seconds"], "unit": "walker-slices/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{walkers} walkers x {slices} slices (one stabilisation block) of {WORKLOAD}, "
                      f"{res['seconds']:.1f} s, NumPy/SciPy BLAS threads = {cores}"}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- roofline
def kernel_flops(kind, M, W, p, precision):
    """Algorithmic real flops of ONE launch of a kernel class (complex MAC = 8)."""
    if kind == "chain":          # one Horner step: V (M x M) times Z (M x M), per walker
        return 8.0 * M ** 3 * W
    if kind == "green":          # LU (8/3 M^3) + two triangular solves with M right-hand sides (8 M^3)
        return (8.0 / 3.0 + 8.0) * M ** 3 * W
    if kind == "qrcp":           # Householder QR (16/3) + forming Q (16/3) + T^-1 update (4)
        return (16.0 / 3.0 + 16.0 / 3.0 + 4.0) * M ** 3 * W
    return None


def roofline(prof, M, W, p, precision):
    dom = max((k for k in prof if prof[k]["n_timed"] > 0), key=lambda k: prof[k]["ms"])
    d = prof[dom]
    avg_s = d["ms"] / d["n_timed"] / 1e3
    fl = kernel_flops(dom, M, W, p, precision)
    if fl is None:
        return {"kernel": dom, "bound": "hbm", "achieved": None, "peak": None, "unit": "GB/s", "frac": None,
                "traffic": None}
    ach = fl / avg_s / 1e12
    return {"kernel": dom, "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
            "peak_source": "FP64 FMA pipe derived from unit counts and clock (152 SMs x 2 DFMA/clk x 2.07 GHz)",
            "avg_launch_ms": avg_s * 1e3, "share_of_step": d["ms"] / sum(v["ms"] for v in prof.values())}


# ---------------------------------------------------------------- ours
def run_ours(args, rank, world, local_rank):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2012_12228_gb300 as ftq

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    c = dict(WORKLOADS[WORKLOAD])
    W = args.walkers or c["walkers"]
    stab = 5
    p_order = 6
    prec = ftq.FTQ_FP64 if args.precision == "fp64" else ftq.FTQ_MIXED
    stream = torch.cuda.current_stream(dev)
    prop = ftq.Propagator(c["N"], c["M"], c["rs"], c["theta"], c["dtau"], walkers=W, stabilise_every=stab,
                          exp_order=p_order, precision=prec, stream=stream)
    M, na, n = prop.M, prop.n_alpha, prop.n_slices
    steps_total = args.warmup + args.steps
    if steps_total * stab > n:
        raise SystemExit(f"warmup + steps must cover at most {n // stab} blocks of {stab} slices")
    seed = c["seed"] + 1000 * rank
    host = gaussian_fields(seed, steps_total * stab, W, na).reshape(steps_total, stab, W, na)
    fields = torch.from_numpy(host).to(dev)
    pinned = torch.from_numpy(host).pin_memory()
    staging = torch.empty((stab, W, na), dtype=torch.float64, device=dev)
    wbuf = torch.empty((W, 8), dtype=torch.float64, device=dev)
    wpin = torch.empty((W, 8), dtype=torch.float64).pin_memory()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(x):
        if world > 1:
            import torch.distributed as dist
            t = torch.tensor([x], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            return float(t.item())
        return x

    # ---- device-resident inputs (value)
    for s in range(args.warmup):
        prop.propagate(fields[s])
    torch.cuda.synchronize(dev)
    barrier()
    launches0 = prop.launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for s in range(args.warmup, steps_total):
            prop.propagate(fields[s])
        est = prop.estimators(per_walker=False)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    barrier()
    launches = prop.launches() - launches0
    t_ms = max_over_ranks(e0.elapsed_time(e1))
    ws_per_step = W * stab
    value = world * ws_per_step * args.steps / (t_ms / 1e3)

    # ---- end to end through the public API with host buffers
    prop.reset()
    for s in range(args.warmup):
        staging.copy_(pinned[s], non_blocking=True)
        prop.propagate(staging)
    torch.cuda.synchronize(dev)
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for s in range(args.warmup, steps_total):
        staging.copy_(pinned[s], non_blocking=True)
        prop.propagate(staging)
        prop.lib.ftq_weights(prop.h, __import__("ctypes").c_void_p(wbuf.data_ptr()))
        wpin.copy_(wbuf, non_blocking=True)
    est2 = prop.estimators(per_walker=False)
    f1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    te_ms = max_over_ranks(f0.elapsed_time(f1))
    e2e_value = world * ws_per_step * args.steps / (te_ms / 1e3)

    # ---- per-kernel launch durations (CUDA events on the launching stream)
    prop.reset()
    prop.propagate(fields[0])
    before = prop.profile_read()
    prop.profile(True)
    prop.propagate(fields[1])
    prop.estimators(per_walker=False)
    after = prop.profile_read()
    prop.profile(False)
    prof = {k: {"ms": after[k][0], "n_timed": after[k][1] - before[k][1]} for k in after}
    rl = roofline(prof, M, W, p_order, args.precision)
    status = prop.status()
    dtau = prop.query_f64("DTAU")
    prop.close()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "walker-slices/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128" if args.precision == "fp64" else "c64(3xtf32)+c128",
        "data": "synthetic: seeded N(0,1) Philox fields; UEG tables from (N, M, r_s, Theta, dtau)",
        "config": {"workload": WORKLOAD, "N": c["N"], "M": M, "rs": c["rs"], "theta": c["theta"],
                   "dtau": dtau, "n_slices": n, "walkers": W,
                   "slices_per_step": stab, "exp_order": p_order, "precision": args.precision,
                   "step": "one stabilisation block (5 slices) for all walkers; one estimator call per timed run",
                   "l2": "inputs larger than L2: walker state %.1f GB per rank" % (W * 7 * M * M * 16 / 1e9),
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": rl,
        "e2e": {"value": e2e_value, "unit": "walker-slices/s",
                "h2d_bytes_per_step": int(stab * W * na * 8), "d2h_bytes_per_step": int(W * 8 * 8),
                "note": "fields copied from pinned host memory and per-walker weights read back every step"},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "kernel_ms_per_step": {k: v["ms"] for k, v in prof.items() if v["ms"] > 0},
        "estimate": {"E_per_electron": (est["E"].real / c["N"]), "N": est["N"].real, "alive": est["n_alive"]},
        "device_status": status,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    walkers, slices = 1, 5
    times = []
    for s in range(args.warmup + args.steps):
        r = run_oracle_child(walkers, slices, cores)
        if s >= args.warmup:
            times.append(r["seconds"])
    tot = sum(times)
    value = walkers * slices * args.steps / tot
    c = WORKLOADS[WORKLOAD]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "walker-slices/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": {"workload": WORKLOAD, "N": c["N"], "M": c["M"], "rs": c["rs"],
                                            "theta": c["theta"], "dtau": c["dtau"], "walkers_sampled": walkers,
                                            "slices_per_step": slices},
            "cpu_baseline": {"value": value, "unit": "walker-slices/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step: {walkers} walker x {slices} slices of {WORKLOAD} "
                                       "through the CPU oracle (NumPy/SciPy, complex128)"},
            "e2e": {"value": value, "unit": "walker-slices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.oracle_sample:
        oracle_sample(*args.oracle_sample)
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" and torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local_rank)
        dist.init_process_group(backend=backend)
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
