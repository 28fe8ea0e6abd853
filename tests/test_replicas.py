"""Replicas on two CPU processes (gloo, world size 2): the combined weighted
estimate equals the estimate over the union of both ranks' walkers, a rank
with no alive walker contributes nothing, and the timing reduction takes the
maximum.  The per-rank sums are formed the way the library's walker
reduction forms them (weights exp(ln|w| - s) e^{i arg w} of the alive
walkers, s the rank's largest ln|w|)."""
import math
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def local_sums(lw, ph, alive, E, N):
    if not alive.any():
        return dict(sum_w=0j, sum_wE=0j, sum_wN=0j, log_scale=0.0, n_alive=0)
    s = np.max(lw[alive])
    w = np.where(alive, np.exp(lw - s) * np.exp(1j * ph), 0.0)
    return dict(sum_w=complex(w.sum()), sum_wE=complex((w * E).sum()), sum_wN=complex((w * N).sum()),
                log_scale=float(s), n_alive=int(alive.sum()))


def walkers(seed, W, dead=0.2, none_alive=False):
    rng = np.random.default_rng(seed)
    lw = rng.normal(0.0, 30.0, W) + 100.0 * seed          # very different scales on the two ranks
    ph = rng.uniform(-0.3, 0.3, W)
    alive = rng.random(W) > dead
    if none_alive:
        alive[:] = False
    E = rng.normal(1.0, 0.5, W) + 1j * rng.normal(0.0, 0.01, W)
    N = rng.normal(14.0, 1.0, W) + 1j * rng.normal(0.0, 0.01, W)
    return lw, ph, alive, E, N


def _worker(rank, world, port, case, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    from paper_2012_12228_gb300 import replicas
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        data = walkers(rank + 1, 40 + 9 * rank, none_alive=(case == "empty" and rank == 1))
        comb = replicas.combine_estimates(local_sums(*data))
        t = replicas.max_over_ranks(1.5 + rank)
        out.put((rank, comb, t))
    finally:
        dist.destroy_process_group()


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("case", ["both", "empty"])
def test_two_rank_combination_equals_union(case):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, case, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    parts = [walkers(r + 1, 40 + 9 * r, none_alive=(case == "empty" and r == 1)) for r in range(2)]
    union = [np.concatenate([p[i] for p in parts]) for i in range(5)]
    ref = local_sums(*union)
    E_ref, N_ref = ref["sum_wE"] / ref["sum_w"], ref["sum_wN"] / ref["sum_w"]
    for rank, comb, t in res:
        assert t == 2.5
        assert comb["n_alive"] == ref["n_alive"]
        assert comb["log_scale"] == ref["log_scale"]
        assert abs(comb["sum_w"] - ref["sum_w"]) < 1e-12 * abs(ref["sum_w"])
        assert abs(comb["E"] - E_ref) < 1e-12 * abs(E_ref)
        assert abs(comb["N"] - N_ref) < 1e-12 * abs(N_ref)


def test_reference_arm_under_torchrun_prints_one_line():
    """bench.py --impl reference under torchrun with two CPU ranks: rank 0
    alone times the oracle sample and prints the JSON line; rank 1 exits 0."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, cwd=root, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
    for key in ("metric", "unit", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling", "vs_baseline",
                "dtype", "data", "config"):
        assert key in d, key
    assert d["higher_is_better"] is True and d["config"]["workload"] == "ueg_n66_m257"
    assert d["e2e"]["value"] == d["value"] and d["cpu_baseline"]["value"] == d["value"]
