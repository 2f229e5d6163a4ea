"""Host-side checks: the seeded input generator, the benchmark's reference arm
contract, and the replica aggregation over two gloo ranks."""
import json
import os
import subprocess
import sys

import pytest
import torch

from synth import inputs as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_splitmix64_matches_scalar_definition():
    idx = torch.arange(0, 64, dtype=torch.int64)
    got = S.splitmix64(12345, idx)
    for i in range(64):
        want = S.splitmix64_scalar(12345, i)
        assert (int(got[i]) & (2 ** 64 - 1)) == want


def test_uniform_ranges_and_determinism():
    a = S.uniform_pm1(7, 0, 10000)
    b = S.uniform_pm1(7, 0, 10000)
    assert torch.equal(a, b)
    assert float(a.min()) >= -1.0 and float(a.max()) < 1.0
    assert abs(float(a.mean())) < 0.05
    c = S.complex_wide_range(3, (1000,))
    mags = torch.log2(c.abs())
    assert float(mags.min()) >= -30.0 - 1e-9 and float(mags.max()) <= 30.0 + 1e-9
    assert S.complex_uniform(1, (4, 5)).dtype == torch.complex128
    # streams are independent: the imaginary part is not the real part
    z = S.complex_uniform(1, (100,))
    assert not torch.equal(z.real, z.imag)


def test_uneven_batch_recipe():
    dims = S.UNEVEN_BATCH
    assert len(dims) == 40
    assert sum(d[0] * d[1] * d[2] for d in dims) == 180355072


def test_reference_arm_json_contract():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--size", "64"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["unit"] == "ms" and line["higher_is_better"] is False
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["value"] > 0


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    v = bench.max_over_ranks(dist, 10.0 + 5.0 * rank)
    q.put((rank, v))
    dist.destroy_process_group()


def test_replicas_take_max_over_two_gloo_ranks():
    import multiprocessing as mp
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = dict(q.get(timeout=10) for _ in range(2))
    assert res == {0: 15.0, 1: 15.0}
