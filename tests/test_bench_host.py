"""Host logic of bench.py: sample sharding and the max-over-ranks reduction."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def test_first_sample_partition_is_disjoint():
    seen = set()
    for step in range(5):
        for rank in range(4):
            f = bench.first_sample(step, rank, 4, 64)
            block = set(range(f, f + 64))
            assert not (block & seen)
            seen |= block
    assert seen == set(range(5 * 4 * 64))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_env()
    bench.barrier(w)
    m = bench.reduce_max(10.0 * (r + 1), w)
    q.put((r, m, bench.first_sample(3, r, w, 64)))
    dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [m for _, m, _ in res] == [20.0, 20.0]
    assert [f for _, _, f in res] == [3 * 2 * 64, (3 * 2 + 1) * 64]


@pytest.mark.parametrize("n", [4, 8, 16])
def test_bench_dct_leg_matches_oracle(n):
    """The bench's torch.fft DCT comparison leg equals the oracle's scipy DCT solve (CPU tensors)."""
    import torch
    from oracle import mixed
    xi = np.random.default_rng(n).standard_normal((3, n ** 3))
    got = bench.dct_field(torch.tensor(xi), n, 1.0 / n, 20.0, 1.3).numpy()
    ref = mixed.solve_dct(n, 20.0, 1.3, xi)
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
    x = torch.tensor(xi[0].reshape(n, n, n))
    for d in range(3):
        assert torch.allclose(bench.idct_ortho(bench.dct_ortho(x, d), d), x, atol=1e-13)


def test_reference_arm_reports_the_time_it_spent(capsys):
    """The reference arm times whole oracle samples of the headline workload; its ms_per_step must be
    wall time it actually spent (steps x ms_per_step fits in the call's own duration)."""
    import json
    import time
    args = type("A", (), {"steps": 2, "warmup": 1, "gpus": 1})()
    t0 = time.perf_counter()
    bench.run_reference(args)
    wall = time.perf_counter() - t0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "samples/s"
    assert line["steps"] * line["ms_per_step"] / 1000.0 <= wall
    assert abs(line["value"] - 1000.0 / line["ms_per_step"]) <= 1e-9 * line["value"]
    assert line["cpu_baseline"]["value"] == line["value"] and line["cpu_baseline"]["kind"] == "oracle"
    assert line["config"]["grid_n"] == 128 and line["config"]["batch"] == 64
