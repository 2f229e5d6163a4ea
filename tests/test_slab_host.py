"""Slab decomposition of one grid over two ranks (gloo on CPU): the geometry
and the all-to-all exchange of paper_2606_23698_gb300.slab, with the local
axis passes done by numpy's FFT in the library's rotated layouts, reproduce
numpy's 3-D FFT.  The GPU version of the same path (the library's kernels for
the passes) is checked bit for bit in tests/test_gpu_slab.py."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from synth import inputs as S


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _pass(x, dir):
    """One axis pass in the library's layout: transform the contiguous last
    axis and rotate it to the front, [A1][A2][n] -> [n][A1][A2]."""
    f = np.fft.fft(x, axis=-1) if dir < 0 else np.fft.ifft(x, axis=-1) * x.shape[-1]
    return np.ascontiguousarray(np.moveaxis(f, -1, 0))


def _worker(rank, world, port, shape, dir, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2606_23698_gb300.slab import exchange, slab_geometry
        n0, n1, n2 = shape
        g = slab_geometry(n0, n1, n2, world)
        x = S.complex_uniform(41, shape).numpy()
        slab = x[rank * g["n0_local"]:(rank + 1) * g["n0_local"]]
        a = _pass(_pass(slab, dir), dir)                      # [n1][n2][n0/R]
        assert a.shape == (n1, n2, g["n0_local"])
        recv = exchange(torch.from_numpy(a).reshape(world, g["lines_local"], g["n0_local"]), world, "host")
        b = recv.numpy().transpose(1, 0, 2).reshape(g["lines_local"], n0)   # transpose_blocks
        y = _pass(b, dir)                                      # [n0][T/R]
        parts = [torch.empty_like(torch.from_numpy(y)) for _ in range(world)]
        dist.all_gather(parts, torch.from_numpy(y))
        if rank == 0:
            full = np.concatenate([p.numpy() for p in parts], axis=1).reshape(n0, n1, n2)
            want = np.fft.fftn(x) if dir < 0 else np.fft.ifftn(x) * x.size
            q.put(float(np.max(np.abs(full - want)) / np.max(np.abs(want))))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("shape,dir", [((8, 6, 10), -1), ((12, 4, 7), +1), ((2, 3, 8), -1)])
def test_slab_exchange_reproduces_fftn(shape, dir):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    mp.start_processes(_worker, args=(2, _free_port(), shape, dir, q), nprocs=2, start_method="spawn")
    assert q.get(timeout=60) < 1e-13


def test_slab_geometry_rejects_indivisible():
    from paper_2606_23698_gb300.slab import slab_geometry
    assert slab_geometry(8, 6, 10, 2) == {"n0_local": 4, "lines": 60, "lines_local": 30}
    with pytest.raises(ValueError):
        slab_geometry(9, 6, 10, 2)
    with pytest.raises(ValueError):
        slab_geometry(8, 3, 5, 2)
