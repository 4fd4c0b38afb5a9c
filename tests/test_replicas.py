"""The multi-GPU form's host logic (replicas, max-over-ranks timing, whole-job throughput, rank-0
output) with world_size 2 on CPU over gloo.  The data path has no collective: each rank denoises
its own stream; these tests exercise what the ranks share."""
import os
import socket
import subprocess
import sys
import time

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist                      # noqa: E402
import torch.multiprocessing as mp                    # noqa: E402

from paper_2312_06827_gb300 import replicas, scene    # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _ranks(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # the slower rank sets the job's time
        dist.barrier()
        t0 = time.perf_counter()
        time.sleep(0.05 + 0.25 * rank)
        local = time.perf_counter() - t0
        t_max = replicas.max_over_ranks(dist, local)
        rate = replicas.whole_job_rate(world, 1000.0, 4, t_max)
        # every rank's replica is its own stream: a scene of the same kind and size, own layout and noise
        sc = scene.SceneConfig(32, 24, seed=0, stream=replicas.replica_stream(rank))
        fr = scene.render_frame(sc, 0, want=("noisy", "gbuf_nz"))
        checksum = torch.tensor([float(fr["noisy"].sum()), float(fr["gbuf_nz"].sum())], dtype=torch.float64)
        gathered = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(gathered, checksum)
        out.put((rank, local, t_max, rate, [g.tolist() for g in gathered]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_run_distinct_streams():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_ranks, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, l0, m0, v0, g0), (r1, l1, m1, v1, g1) = res
    assert m0 == m1 == pytest.approx(max(l0, l1)) and l1 > l0 + 0.2
    assert v0 == v1 == pytest.approx(2 * 1000.0 * 4 / m0)
    assert g0 == g1
    (noisy0, g_0), (noisy1, g_1) = g0
    assert noisy0 != noisy1 and g_0 != g_1           # independent streams


def test_single_process_helpers():
    assert replicas.max_over_ranks(None, 1.5) == 1.5
    assert replicas.whole_job_rate(1, 10.0, 3, 2.0) == 15.0
    with pytest.raises(ValueError):
        replicas.whole_job_rate(2, 1.0, 1, 0.0)
    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK") if k in os.environ}
    try:
        assert replicas.rank_info() == (1, 0, 0)
    finally:
        os.environ.update(env)


def test_reference_arm_prints_on_rank_zero_only():
    """Under the launcher, a rank other than 0 of the reference arm exits 0 without output."""
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
