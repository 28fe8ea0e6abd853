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
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synthetic_inputs import RAGGED, WORKLOADS, gaussian_fields  # noqa: E402

METRIC = "walker-slices/sec at M=257 (mixed vs FP64, same GB300) at ≤1e-5 Ha/e error"
WORKLOAD = "ueg_n66_m257"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Pipe peaks from the SM count (device properties), the maximum SM clock
# (MEASURED_PEAKS.json, driver-written) and the per-SM issue rates of this
# part: 2 FP64 FMA and 128 FP32 FMA per clock per SM, 2 flop per FMA
# (nominal FP64 1.25 TFLOP/s).  Set by set_device_peaks() once the device is
# known; the defaults below are the same formula for 152 SMs at 2.07 GHz.
SMS, SM_GHZ = 152, 2.07
FP64_PEAK_TFLOPS = SMS * 2 * 2 * SM_GHZ * 1e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--fp64-steps", type=int, default=2, help="timed steps of the complex128 comparison")
    ap.add_argument("--no-compare", action="store_true", help="skip the complex128 comparison run")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the mixed-vs-FP64 energy check")
    ap.add_argument("--no-ragged", action="store_true", help="skip the ragged-batch measurement")
    ap.add_argument("--no-configs", action="store_true", help="skip the M=57 and M=123 whole-path lines")
    ap.add_argument("--walkers", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--lowrank", action="store_true",
                    help="add the low-rank truncation measurement (complex128, N=14, M=515, r_s=0.5, Theta=0.125)")
    ap.add_argument("--lowrank-walkers", type=int, default=152)
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
    """The oracle on a bounded sample of the workload, with all host cores
    and, beside it, with one BLAS thread (one walker)."""
    cores = os.cpu_count() or 1
    res = run_oracle_child(walkers, slices, cores)
    one = run_oracle_child(1, slices, 1)
    return {"value": res["walker_slices"] / res["seconds"], "unit": "walker-slices/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{walkers} walkers x {slices} slices (one stabilisation block) of {WORKLOAD}, "
                      f"{res['seconds']:.1f} s, NumPy/SciPy BLAS threads = {cores}",
            "one_core": {"value": one["walker_slices"] / one["seconds"], "cores": 1,
                         "sample": f"1 walker x {slices} slices, {one['seconds']:.1f} s, BLAS threads = 1"}}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"ftq_clocks_{os.getpid()}.csv")

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
PEAKS = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
FP32_PEAK_TFLOPS = SMS * 128 * 2 * SM_GHZ * 1e9 / 1e12


def set_device_peaks(torch, dev):
    """SM count from the device properties and the maximum SM clock from
    MEASURED_PEAKS.json (else 2.07 GHz); recomputes the pipe peaks."""
    global SMS, SM_GHZ, FP64_PEAK_TFLOPS, FP32_PEAK_TFLOPS
    SMS = torch.cuda.get_device_properties(dev).multi_processor_count
    SM_GHZ = PEAKS.get("sm_max_mhz", 2070.0) / 1e3
    FP64_PEAK_TFLOPS = SMS * 2 * 2 * SM_GHZ * 1e9 / 1e12
    FP32_PEAK_TFLOPS = SMS * 128 * 2 * SM_GHZ * 1e9 / 1e12

# DRAM bytes (read + write) per walker and launch from one ncu capture of the
# kernel as it stands (files under profiles/); the launches process walkers
# independently with working sets far above L2, so traffic scales with the
# walker count.  An entry is removed when its kernel changes.
TRAFFIC_PER_WALKER = {     # (bytes per walker, summary file, walkers in the capture)
    ("mixed", "green"): ((15.221e9 + 4.772e9) / 608, "profiles/green32b_ueg_n66_m257_w608.md", 608),
    ("mixed", "chain"): ((0.43736e9 + 0.22356e9) / 256, "profiles/chain_tc_ueg_n66_m257_w256.md", 256),
    ("fp64", "chain"): (0.3867e9 / 128, "profiles/chain_fp64_ueg_n66_m257_w128.md", 128),
}


def kernel_model(kind, M, W, precision, green_tc=False):
    """(algorithmic flops of ONE launch, bound, peak TFLOP/s, peak source).

    Real flops; a complex multiply-add counts 8.  The tensor-core chain runs
    the complex product as three tf32 products (3xTF32), so its tensor work is
    3 x 8 M^3 per walker and its peak is the tf32 dense rate: the measured
    bf16 GEMM rate times the nominal tf32/bf16 ratio 1.1/2.25."""
    fp64 = ("alu", FP64_PEAK_TFLOPS, f"FP64 FMA pipe: {SMS} SMs (device properties) x 2 DFMA/clk x 2 x "
                                      f"{SM_GHZ:.2f} GHz (max SM clock)")
    fp32 = ("alu", FP32_PEAK_TFLOPS, f"FP32 FMA pipe: {SMS} SMs (device properties) x 128 FMA/clk x 2 x "
                                      f"{SM_GHZ:.2f} GHz (max SM clock)")
    bf16 = PEAKS.get("bf16_tflops", 1900.0)
    tf32 = ("tensor", bf16 * 1.1 / 2.25,
            f"tf32 dense = measured bf16 {bf16:.1f} TFLOP/s x 1.1/2.25 (MEASURED_PEAKS.json)"
            if "bf16_tflops" in PEAKS else "tf32 dense = fallback bf16 1900 TFLOP/s x 1.1/2.25")
    if kind == "chain":          # one Horner step: V (M x M) times Z (M x M), per walker
        if precision == "mixed":
            return (3 * 8.0 * M ** 3 * W,) + tf32
        return (8.0 * M ** 3 * W,) + (fp64 if precision == "fp64" else fp32)
    if kind == "green":
        if green_tc:             # Gauss-Jordan on [Mt^T | B^T]: 1.5 M^3 complex MACs, as 3xTF32 MMAs
            return (3 * 12.0 * M ** 3 * W,) + tf32
        # LU (8/3 M^3) + two triangular solves with M right-hand sides (8 M^3)
        return ((8.0 / 3.0 + 8.0) * M ** 3 * W,) + (fp64 if precision == "fp64" else fp32)
    if kind == "qrcp":
        if precision == "fp64":  # Householder QR (16/3) + forming Q (16/3) + T^-1 update (4)
            return ((16.0 / 3.0 + 16.0 / 3.0 + 4.0) * M ** 3 * W,) + fp64
        return ((16.0 / 3.0) * M ** 3 * W,) + fp32          # FP32 Householder of Y Pi (Q: bridge class)
    if kind == "tinv":           # T^-1 <- T^-1 Pi U^-1: a triangular solve with M right-hand sides
        return (4.0 * M ** 3 * W,) + fp64
    return None


def roofline(prof, M, W, precision, green_tc=False):
    timed = {k: v for k, v in prof.items() if v["n_timed"] > 0}
    dom = max(timed, key=lambda k: timed[k]["ms"])
    d = prof[dom]
    avg_s = d["ms"] / d["n_timed"] / 1e3
    share = d["ms"] / sum(v["ms"] for v in timed.values())
    model = kernel_model(dom, M, W, precision, green_tc)
    if model is None:
        return {"kernel": dom, "bound": "hbm", "achieved": None, "peak": None, "unit": "GB/s", "frac": None,
                "traffic": None, "avg_launch_ms": avg_s * 1e3, "share_of_step": share}
    fl, bound, peak, src = model
    ach = fl / avg_s / 1e12
    tr = None if (dom == "green" and green_tc) else TRAFFIC_PER_WALKER.get((precision, dom))
    out = {"kernel": dom, "bound": bound, "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
           "traffic": None if tr is None else tr[0] * W, "peak_source": src, "avg_launch_ms": avg_s * 1e3,
           "share_of_step": share}
    if tr is not None:
        out["traffic_source"] = (f"dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture at {tr[2]} "
                                 f"walkers ({tr[1]}), scaled to {W} walkers")
    return out


# ---------------------------------------------------------------- ours
def measure_path(ftq, torch, dev, precision, W, steps, warmup, world, rank, barrier, max_over_ranks,
                 with_e2e=True, with_clocks=None):
    c = dict(WORKLOADS[WORKLOAD])
    stab, p_order = 5, 6
    stream = torch.cuda.current_stream(dev)
    prec = ftq.FTQ_FP64 if precision == "fp64" else ftq.FTQ_MIXED
    prop = ftq.Propagator(c["N"], c["M"], c["rs"], c["theta"], c["dtau"], walkers=W, stabilise_every=stab,
                          exp_order=p_order, precision=prec, stream=stream)
    M, na, n = prop.M, prop.n_alpha, prop.n_slices
    tuned = prop.autotune() if precision == "mixed" else None
    total = warmup + steps
    if total * stab > n:
        raise SystemExit(f"warmup + steps must cover at most {n // stab} blocks of {stab} slices")
    seed = c["seed"] + 1000 * rank
    host = gaussian_fields(seed, total * stab, W, na).reshape(total, stab, W, na)
    fields = torch.from_numpy(host).to(dev)
    out = {"M": M, "n_slices": n, "dtau": prop.query_f64("DTAU"), "walkers": W, "stab": stab, "p": p_order,
           "autotune": None if tuned is None else {"column_tiles": tuned[0], "ms_per_horner_step": tuned[1],
                                                   "qr_panel": prop.query("QR_PANEL"),
                                                   "green_kernel": {1: "tensor-core Gauss-Jordan",
                                                                    2: "CUDA-core blocked LU"}.get(
                                                       prop.query("GREEN_KERNEL"), "none")}}

    for s in range(warmup):
        prop.propagate(fields[s])
    torch.cuda.synchronize(dev)
    barrier()
    launches0 = prop.launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(dev.index) if with_clocks else None
    if clk:
        clk.__enter__()
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for s in range(warmup, total):
        prop.propagate(fields[s])
    est = prop.estimators(per_walker=False)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if clk:
        clk.__exit__()
        out["clocks"] = clk.summary()
    barrier()
    out["gpu_launches"] = prop.launches() - launches0
    t_ms = max_over_ranks(e0.elapsed_time(e1))
    out["ms_per_step"] = t_ms / steps
    out["value"] = world * W * stab * steps / (t_ms / 1e3)
    if world > 1:                   # weighted estimate over the walkers of every replica
        from paper_2012_12228_gb300 import replicas
        est = replicas.combine_estimates(est, device=dev)
    out["estimate"] = {"E_per_electron": est["E"].real / c["N"], "N": est["N"].real, "alive": est["n_alive"]}

    if with_e2e:
        pinned = torch.from_numpy(host).pin_memory()
        staging = torch.empty((stab, W, na), dtype=torch.float64, device=dev)
        wbuf = torch.empty((W, 8), dtype=torch.float64, device=dev)
        wpin = torch.empty((W, 8), dtype=torch.float64).pin_memory()
        prop.reset()
        for s in range(warmup):
            staging.copy_(pinned[s], non_blocking=True)
            prop.propagate(staging)
        torch.cuda.synchronize(dev)
        barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for s in range(warmup, total):
            staging.copy_(pinned[s], non_blocking=True)
            prop.propagate(staging)
            prop.lib.ftq_weights(prop.h, ctypes.c_void_p(wbuf.data_ptr()))
            wpin.copy_(wbuf, non_blocking=True)
        prop.estimators(per_walker=False)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        te_ms = max_over_ranks(f0.elapsed_time(f1))
        out["e2e"] = {"value": world * W * stab * steps / (te_ms / 1e3), "unit": "walker-slices/s",
                      "h2d_bytes_per_step": int(stab * W * na * 8), "d2h_bytes_per_step": int(W * 8 * 8),
                      "note": "fields copied from pinned host memory and per-walker weights read back every "
                              "step, one estimator read-back per timed run"}

    # per-kernel launch durations: CUDA events on the launching stream, one block
    prop.reset()
    prop.propagate(fields[0])
    before = prop.profile_read()
    prop.profile(True)
    prop.propagate(fields[1])
    prop.estimators(per_walker=False)
    after = prop.profile_read()
    prop.profile(False)
    prof = {k: {"ms": after[k][0], "n_timed": after[k][1] - before[k][1]} for k in after}
    out["kernel_ms_per_step"] = {k: v["ms"] for k, v in prof.items() if v["ms"] > 0}
    out["roofline"] = roofline(prof, M, W, precision, green_tc=prop.query("GREEN_KERNEL") == 1)
    out["device_status"] = prop.status()
    out["slice_average"] = measure_tracking(torch, prop, stream, fields)
    out["population_control"] = measure_comb(torch, prop, stream, precision, fields)
    prop.close()
    return out


def measure_tracking(torch, prop, stream, fields):
    """Cost of the time-slice estimates (Results, the slice-averaged
    estimator): one block of 5 slices with the estimators evaluated and
    recorded after every slice, against the same block without; and one
    estimator evaluation at tau_k alone (CUDA events on the launching
    stream)."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {}
    for every in (0, 1):
        prop.reset()
        prop.propagate(fields[0])
        prop.track_estimates(every)
        torch.cuda.synchronize()
        e0.record(stream)
        prop.propagate(fields[1])
        e1.record(stream)
        torch.cuda.synchronize()
        res[every] = e0.elapsed_time(e1)
    prop.track_estimates(0)
    before = prop.profile_read()
    prop.profile(True)
    prop.estimators(per_walker=False)
    after = prop.profile_read()
    prop.profile(False)
    est_ms = after["estimators"][0] - 0.0
    prop.reset()
    return {"ms_per_block_plain": res[0], "ms_per_block_tracked": res[1],
            "overhead_ms_per_slice": (res[1] - res[0]) / 5.0,
            "estimator_ms_per_call_c128": est_ms,
            "note": "5-slice block with the estimators of every slice recorded vs without; "
                    "estimator call on the complex128 G at tau_k"}


def measure_comb(torch, prop, stream, precision, fields):
    """Comb population control of all walkers (after the measured blocks; one
    untimed block of 5 slices before each comb so that the weights differ):
    ms per comb and the achieved copy bandwidth (each copied walker's state
    is read once and written once)."""
    M, W = prop.M, prop.W
    Kp, LD = (M + 15) // 16 * 16, (M + 7) // 8 * 8
    walker_bytes = (16 * M * M + 16 * M * M + 16 * M + 8 * 16 +
                    (16 * M * M if precision == "fp64" else 8 * LD * 2 * Kp + 8 * M * M))
    draws = [0.37, 0.71]
    ms, moved = 0.0, 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ident = torch.arange(W, device="cuda", dtype=torch.int32)
    for i, x in enumerate(draws):
        prop.propagate(fields[2 + i])
        torch.cuda.synchronize()
        e0.record(stream)
        par = prop.population_control(x)
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        moved += int((par != ident).sum().item())
    ms /= len(draws)
    gbs = 2.0 * walker_bytes * moved / len(draws) / (ms / 1e3) / 1e9
    return {"ms_per_comb": ms, "walkers_copied_per_comb": moved / len(draws), "bytes_per_walker": walker_bytes,
            "copy_GBps": gbs, "hbm_frac": gbs / PEAKS.get("hbm_gbs", 6800.0),
            "note": "comb of all walkers after the measured blocks (not part of the timed step); "
                    "hbm_frac of the measured copy bandwidth"}


def measure_ragged(ftq, torch, dev, steps=4, warmup=3):
    """Walker-slices/s of the ragged batch (four systems of M = 57, 123, 171,
    257, 256 walkers each, one persistent tensor-core launch per Horner step,
    CUDA-graph-captured blocks of 5 slices, autotuned column tiles)."""
    b = ftq.Batch(RAGGED)
    tuned = b.autotune()
    stab = 5
    fl = []
    for sd, m in zip(RAGGED, b.members):
        fl.append(torch.from_numpy(gaussian_fields(sd["seed"], (warmup + steps) * stab, sd["walkers"],
                                                   m.n_alpha)).to(dev))
    for s in range(warmup):
        b.propagate([f[s * stab:(s + 1) * stab].contiguous() for f in fl])
    torch.cuda.synchronize(dev)
    l0 = b.launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(dev)
    e0.record(stream)
    for s in range(warmup, warmup + steps):
        b.propagate([f[s * stab:(s + 1) * stab].contiguous() for f in fl])
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    ws = sum(sd["walkers"] for sd in RAGGED) * stab * steps
    res = {"value": ws / (ms / 1e3), "unit": "walker-slices/s", "ms_per_step": ms / steps, "steps": steps,
           "warmup": warmup, "gpu_launches": b.launches() - l0, "graph": "one CUDA graph launch per step",
           "systems": [dict(N=sd["N"], M=sd["M"], rs=sd["rs"], theta=sd["theta"], dtau=sd["dtau"],
                            walkers=sd["walkers"], column_tiles=t[0]) for sd, t in zip(RAGGED, tuned)]}
    # per-kernel times of one block (event timing turns the graph off for this block)
    ctxs = [b] + b.members
    for c in ctxs:
        c.profile(True)
    res["roofline"] = ragged_roofline(b, fl, stab, ctxs)
    for c in ctxs:
        c.profile(False)
    b.close()
    res["sequential"] = measure_ragged_sequential(ftq, torch, dev, steps, warmup)
    res["batch_over_sequential"] = res["value"] / res["sequential"]["value"]
    return res


def ragged_roofline(b, fl, stab, ctxs):
    """Dominant kernel class of one batched block of 5 slices (the members
    are reset and run their first block again) with its algorithmic flops
    summed over the systems."""
    for m in b.members:
        m.reset()
    b.propagate([f[0:stab].contiguous() for f in fl])
    prof = [c.profile_read() for c in ctxs]
    kinds = {}
    for p in prof:
        for k, (ms, _) in p.items():
            kinds[k] = kinds.get(k, 0.0) + ms
    dom = max(kinds, key=lambda k: kinds[k])
    flops = 0.0
    model = None
    for sd, m in zip(RAGGED, b.members):
        per_block = {"chain": 6 * stab, "green": stab, "qrcp": 1, "tinv": 1}.get(dom, 0)
        mm = kernel_model(dom, m.M, m.W, "mixed")
        if mm is None or per_block == 0:
            model = None
            break
        model = mm
        flops += mm[0] * per_block
    out = {"kernel": dom, "ms_per_block_by_kernel": kinds}
    if model is not None:
        ach = flops / (kinds[dom] / 1e3) / 1e12
        out.update({"bound": model[1], "achieved": ach, "peak": model[2], "unit": "TFLOP/s",
                    "frac": ach / model[2], "peak_source": model[3]})
    return out


def measure_ragged_sequential(ftq, torch, dev, steps, warmup):
    """The same four systems run one after another as separate contexts
    (mixed precision, autotuned column tiles, same fields and block count):
    the sum of their times is what the batch replaces."""
    stab = 5
    total_ms = 0.0
    ws = 0
    stream = torch.cuda.current_stream(dev)
    for sd in RAGGED:
        p = ftq.Propagator(sd["N"], sd["M"], sd["rs"], sd["theta"], sd["dtau"], walkers=sd["walkers"],
                           precision=ftq.FTQ_MIXED, stream=stream)
        p.autotune()
        f = torch.from_numpy(gaussian_fields(sd["seed"], (warmup + steps) * stab, sd["walkers"],
                                             p.n_alpha)).to(dev)
        for s_ in range(warmup):
            p.propagate(f[s_ * stab:(s_ + 1) * stab].contiguous())
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for s_ in range(warmup, warmup + steps):
            p.propagate(f[s_ * stab:(s_ + 1) * stab].contiguous())
        e1.record(stream)
        torch.cuda.synchronize(dev)
        total_ms += e0.elapsed_time(e1)
        ws += sd["walkers"] * stab * steps
        p.close()
    return {"value": ws / (total_ms / 1e3), "unit": "walker-slices/s", "ms_per_step": total_ms / steps,
            "note": "the four systems as four contexts, one after another, same steps"}


LOWRANK = dict(N=14, M=515, rs=0.5, theta=0.125, dtau=0.05, seed=1240)


def measure_lowrank(ftq, torch, dev, W, thr=1e-6):
    """Whole-path complex128 throughput with and without low-rank truncation
    (threshold 1e-6) on a system with M >> N-bar at low temperature (N = 14,
    M = 515, r_s = 0.5, Theta = 0.125, dtau = 0.05: 22 slices), the same
    fields for both, plus the kept ranks along the path: m_R of the right
    block after every stabilisation (ftq_ranks) and m_L of the trial block."""
    c = LOWRANK
    stream = torch.cuda.current_stream(dev)
    res = {}
    for t, prec, name in ((0.0, ftq.FTQ_FP64, "full_rank"), (thr, ftq.FTQ_FP64, "low_rank"),
                          (0.0, ftq.FTQ_MIXED, "mixed_full_rank"), (thr, ftq.FTQ_MIXED, "mixed_low_rank")):
        p = ftq.Propagator(c["N"], c["M"], c["rs"], c["theta"], c["dtau"], walkers=W, stabilise_every=5,
                           exp_order=6, precision=prec, stream=stream, low_rank=t)
        n, na = p.n_slices, p.n_alpha
        f = torch.from_numpy(gaussian_fields(c["seed"], n, W, na)).to(dev)
        p.propagate(f[:1].contiguous())          # warm-up (first launches, shared-memory attributes)
        p.reset()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        p.propagate(f)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        est = p.estimators(per_walker=True)
        pw = est["per_walker"].cpu().numpy()
        alive = pw[:, 2] > 0.5
        out = {"value": W * n / (ms / 1e3), "unit": "walker-slices/s", "ms_path": ms,
               "E_per_electron": float(np.mean(pw[alive, 3]) / c["N"]), "N": float(np.mean(pw[alive, 5])),
               "alive": int(alive.sum()), "status": p.status()}
        if t > 0 and prec == ftq.FTQ_FP64:
            trace = []
            p.reset()
            for k0 in range(0, n, 5):
                p.propagate(f[k0:min(k0 + 5, n)].contiguous())
                trace.append(int(np.max(p.ranks())))
            L, mu_t, dt = p.query_f64("L"), p.query_f64("MU_T"), p.query_f64("DTAU")
            eps = 0.5 * (2 * np.pi / L) ** 2 * np.sum(np.array(p.basis(), dtype=np.float64) ** 2, axis=1)
            m_left = [int(np.sum(np.exp(-(n - k) * dt * (eps - mu_t)) >= t)) for k in range(5, n + 1, 5)]
            out.update({"threshold": t, "m_R_max_after_each_stabilisation": trace,
                        "m_L_at_each_stabilisation": m_left})
        res[name] = out
        p.close()
    res["compression"] = [compression_trace(ftq, torch, dev, stream, t_, thr)
                          for t_ in (0.125, 0.5)]
    res["compression_m1189"] = [compression_trace(ftq, torch, dev, stream, t_, thr, W=8, M=1189)
                                for t_ in (0.125, 0.5)]
    res.update({"workload": "ueg_n14_m515 (r_s=0.5, Theta=0.125, dtau=0.05)", "M": c["M"], "walkers": W,
                "n_slices": n, "precision": "c128 and mixed (tensor-core chain on the kept columns)",
                "speedup": res["low_rank"]["value"] / res["full_rank"]["value"],
                "mixed_speedup": res["mixed_low_rank"]["value"] / res["mixed_full_rank"]["value"],
                "mixed_low_rank_over_fp64_low_rank": res["mixed_low_rank"]["value"] / res["low_rank"]["value"],
                "mixed_low_rank_E_per_electron_abs_diff": abs(res["mixed_low_rank"]["E_per_electron"]
                                                              - res["low_rank"]["E_per_electron"]),
                "E_per_electron_abs_diff": abs(res["low_rank"]["E_per_electron"] - res["full_rank"]["E_per_electron"]),
                "N_abs_diff": abs(res["low_rank"]["N"] - res["full_rank"]["N"])})
    return res


def compression_trace(ftq, torch, dev, stream, theta, thr, W=16, dtau=0.01, M=None):
    """Ranks along the path of N = 14, M = 515 (or the given M), r_s = 0.5 at
    temperature Theta (dtau = 0.01): m_R (largest over the walkers) after
    every stabilisation, m_L of the trial block and m_T = min(m_R, m_L) at
    the same slices, and the compression 1 - m/M of each (the quantities of
    the paper's low-rank compression figure, whose basis is M = 1189)."""
    c = dict(LOWRANK)
    if M is not None:
        c["M"] = M
    p = ftq.Propagator(c["N"], c["M"], c["rs"], theta, dtau, walkers=W, stabilise_every=5, exp_order=6,
                       precision=ftq.FTQ_FP64, stream=stream, low_rank=thr)
    n, na, M = p.n_slices, p.n_alpha, p.M
    f = torch.from_numpy(gaussian_fields(c["seed"] + 1, n, W, na)).to(dev)
    L, mu_t, dt = p.query_f64("L"), p.query_f64("MU_T"), p.query_f64("DTAU")
    eps = 0.5 * (2 * np.pi / L) ** 2 * np.sum(np.array(p.basis(), dtype=np.float64) ** 2, axis=1)
    rows = []
    for k0 in range(0, n - n % 5, 5):
        p.propagate(f[k0:k0 + 5].contiguous())
        k = k0 + 5
        m_r = int(np.max(p.ranks()))
        m_l = int(np.sum(np.exp(-(n - k) * dt * (eps - mu_t)) >= thr))
        rows.append({"tau": k * dt, "m_R": m_r, "m_L": m_l, "m_T": min(m_r, m_l)})
    status = p.status()
    p.close()
    return {"M": M, "theta": theta, "dtau": dt, "n_slices": n, "walkers": W, "status": status, "trace": rows,
            "mean_compression_T": float(np.mean([1.0 - r["m_T"] / M for r in rows]))}


def measure_config(ftq, torch, dev, wl, precision, with_mu=False):
    """Walker-slices/s of the whole path (all n slices, the estimators at
    tau = beta) of a smaller workload at its own walker count; with_mu adds
    the chemical-potential derivative (forward accumulation along the path,
    evaluated by ftq_mu_grad at tau = beta) and its cost."""
    c = dict(WORKLOADS[wl])
    W = c["walkers"]
    stream = torch.cuda.current_stream(dev)
    prec = ftq.FTQ_FP64 if precision == "fp64" else ftq.FTQ_MIXED
    p = ftq.Propagator(c["N"], c["M"], c["rs"], c["theta"], c["dtau"], walkers=W, precision=prec, stream=stream)
    if precision == "mixed":
        p.autotune()
    n = p.n_slices
    f = torch.from_numpy(gaussian_fields(c["seed"], n, W, p.n_alpha)).to(dev)
    p.propagate(f[:5].contiguous())            # warm-up
    p.reset()
    torch.cuda.synchronize(dev)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    l0 = p.launches()
    e0.record(stream)
    p.propagate(f)
    est = p.estimators(per_walker=False)
    e1.record(stream)
    out = {"workload": wl, "precision": precision, "N": c["N"], "M": p.M, "walkers": W, "n_slices": n}
    if with_mu:
        g = p.mu_grad(per_walker=False)
        e2.record(stream)
        torch.cuda.synchronize(dev)
        out["mu_derivative"] = {"dN_dmu": g["dN"], "dE_dmu": g["dE"], "ms_mu_grad_call": e1.elapsed_time(e2),
                                "note": "tangents accumulated in the Green epilogues of every slice; "
                                        "ftq_mu_grad evaluates them at tau = beta"}
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    out.update({"value": W * n / (ms / 1e3), "unit": "walker-slices/s", "ms_path": ms,
                "gpu_launches": int(p.launches() - l0), "E_per_electron": est["E"].real / c["N"],
                "N": est["N"].real, "alive": est["n_alive"], "status": p.status()})
    p.close()
    return out


def accuracy_vs_fp64(ftq, torch, dev, W=32):
    """E/N at tau = beta of the mixed and the complex128 path on identical
    fields (whole path, W walkers)."""
    c = dict(WORKLOADS[WORKLOAD])
    stream = torch.cuda.current_stream(dev)
    res = {}
    n = 0
    for name, prec in (("fp64", ftq.FTQ_FP64), ("mixed", ftq.FTQ_MIXED)):
        prop = ftq.Propagator(c["N"], c["M"], c["rs"], c["theta"], c["dtau"], walkers=W, stabilise_every=5,
                              exp_order=6, precision=prec, stream=stream)
        n = prop.n_slices
        f = torch.from_numpy(gaussian_fields(c["seed"] + 777, n, W, prop.n_alpha)).to(dev)
        t0 = time.perf_counter()
        prop.propagate(f)
        est = prop.estimators(per_walker=True)
        pw = est["per_walker"].cpu().numpy()
        res[name] = {"E_per_electron": est["E"].real / c["N"], "N": est["N"].real, "alive": est["n_alive"],
                     "seconds": time.perf_counter() - t0, "alive_mask": (pw[:, 2] > 0.5).tolist(),
                     "status": prop.status()}
        prop.close()
    d = abs(res["mixed"]["E_per_electron"] - res["fp64"]["E_per_electron"])
    return {"E_per_electron_abs_diff": d, "bound": 1e-5, "within_bound": d <= 1e-5,
            "E_per_electron_fp64": res["fp64"]["E_per_electron"], "E_per_electron_mixed": res["mixed"]["E_per_electron"],
            "N_fp64": res["fp64"]["N"], "N_mixed": res["mixed"]["N"],
            "same_killed_walkers": res["fp64"]["alive_mask"] == res["mixed"]["alive_mask"],
            "walkers": W, "slices": n, "fields": "seeded N(0,1), identical for both paths"}


def run_ours(args, rank, world, local_rank):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2012_12228_gb300 as ftq

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    set_device_peaks(torch, dev)
    c = dict(WORKLOADS[WORKLOAD])
    W = args.walkers or c["walkers"]

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    from paper_2012_12228_gb300 import replicas

    def max_over_ranks(x):
        return replicas.max_over_ranks(x, device=dev) if world > 1 else x

    head = measure_path(ftq, torch, dev, args.precision, W, args.steps, args.warmup, world, rank, barrier,
                        max_over_ranks, with_e2e=True, with_clocks=True)
    comparison = None
    if args.precision == "mixed" and not args.no_compare:
        comparison = measure_path(ftq, torch, dev, "fp64", W, args.fp64_steps, args.warmup, world, rank, barrier,
                                  max_over_ranks, with_e2e=False, with_clocks=False)
    acc = None
    if args.precision == "mixed" and not args.no_accuracy and rank == 0:
        acc = accuracy_vs_fp64(ftq, torch, dev)
    lowrank = measure_lowrank(ftq, torch, dev, args.lowrank_walkers) if args.lowrank and rank == 0 else None
    ragged = None
    if args.precision == "mixed" and not args.no_ragged and rank == 0:
        ragged = measure_ragged(ftq, torch, dev)
    others = None
    if args.precision == "mixed" and not args.no_configs and rank == 0:
        others = {"ueg_n2_m7": measure_config(ftq, torch, dev, "ueg_n2_m7", "fp64"),
                  "ueg_n14_m57": {p_: measure_config(ftq, torch, dev, "ueg_n14_m57", p_) for p_ in ("mixed", "fp64")},
                  "ueg_n14_m123": measure_config(ftq, torch, dev, "ueg_n14_m123", "fp64", with_mu=True)}
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": head["value"], "unit": "walker-slices/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c128" if args.precision == "fp64" else "c64(tf32 hi+lo)+c128",
        "data": "synthetic: seeded N(0,1) Philox fields; UEG tables from (N, M, r_s, Theta, dtau)",
        "config": {"workload": WORKLOAD, "N": c["N"], "M": head["M"], "rs": c["rs"], "theta": c["theta"],
                   "dtau": head["dtau"], "n_slices": head["n_slices"], "walkers": W,
                   "slices_per_step": head["stab"], "exp_order": head["p"], "precision": args.precision,
                   "step": "one stabilisation block (5 slices) for all walkers; one estimator call per timed run "
                           "(the path evaluates the estimators once, at tau = beta, every 348 slices)",
                   "l2": "inputs larger than L2: walker state > 7 GB per rank",
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": head["roofline"],
        "e2e": head["e2e"],
        "gpu_launches": int(head["gpu_launches"]),
        "clocks": head.get("clocks"),
        "kernel_ms_per_step": head["kernel_ms_per_step"],
        "estimate": head["estimate"],
        "device_status": head["device_status"],
        "population_control": head["population_control"],
        "slice_average": head["slice_average"],
    }
    if comparison:
        line["fp64_path"] = {"value": comparison["value"], "ms_per_step": comparison["ms_per_step"],
                             "steps": args.fp64_steps, "warmup": args.warmup,
                             "speedup_mixed_over_fp64": head["value"] / comparison["value"],
                             "roofline": comparison["roofline"],
                             "kernel_ms_per_step": comparison["kernel_ms_per_step"]}
    if acc:
        line["error_vs_fp64"] = acc
    if ragged:
        line["ragged_batch"] = ragged
    if others:
        line["other_configs"] = others
    if lowrank:
        line["low_rank"] = lowrank
    if head.get("autotune"):
        line["config"]["autotune"] = head["autotune"]
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
