"""bench.py host logic without a GPU: the multi-rank timing reduction on two
gloo ranks, and the reference arm's JSON line (the FP64 oracle on the small
workload) with the silence of non-zero ranks."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 * (rank + 1), world, torch.device("cpu"))
    value, ms_tot = bench.aggregate([ms], [7 * world])
    out.put((rank, ms, value, ms_tot))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    """Every rank gets the slowest rank's time; the whole-job value counts all
    ranks' vectors over that time."""
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value, ms_tot in res:
        assert ms == 20.0 and ms_tot == 20.0
        assert value == pytest.approx(14 / 0.020)


def _bench(args, env_extra=None):
    env = dict(os.environ, **(env_extra or {}))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True, text=True,
                          env=env, cwd=ROOT, timeout=600)


def test_reference_arm_json_line():
    r = _bench(["--impl", "reference", "--workload", "fio_n4096_r12", "--steps", "2", "--warmup", "3"])
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["unit"] == "vectors/s" and d["steps"] == 2 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_reference_arm_other_ranks_exit_silently():
    r = _bench(["--impl", "reference", "--workload", "fio_n4096_r12", "--steps", "2", "--warmup", "3"],
               {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_warmup_below_three_is_rejected():
    r = _bench(["--impl", "reference", "--workload", "fio_n4096_r12", "--steps", "1", "--warmup", "2"])
    assert r.returncode != 0


def test_tensor_core_traffic_model_follows_the_tile_width():
    """The bytes the benchmark charges a tensor-core apply: 8 two-level passes
    at N = 2^20, L = 16, leaf 16, r = 16 read 16384 dense 64 x 64 complex
    blocks each (32 KB, once per RHS tile), the caller's vectors in and out,
    and 7 intermediates of R = 2^20 positions written and read, W RHS wide."""
    sys.path.insert(0, ROOT)
    import bench

    class F:
        L, n0, r, h, m, N = 16, 16, 16, 8, 256, 1 << 20

    R = (1 << F.L) * F.r
    blocks = 8 * 16384 * 32768
    for nrhs, W in ((128, 128), (32, 32), (20, 32), (64, 64)):
        assert bench.tc_tile_width(nrhs) == W
        assert bench.tc_traffic_bytes(F, nrhs) == blocks + 8 * nrhs * 2 * F.N + 8 * W * 2 * R * 7
    assert abs(bench.tc_traffic_bytes(F, 128) / 1e9 - 21.47) < 0.01
    # several tiles: evened out, whole warps
    assert [bench.tc_tile_width(n) for n in (1, 33, 100, 129, 200, 257)] == [32, 64, 128, 96, 128, 96]
    assert bench.tc_traffic_bytes(F, 256) == 2 * blocks + 8 * 256 * 2 * F.N + 8 * 256 * 2 * R * 7
