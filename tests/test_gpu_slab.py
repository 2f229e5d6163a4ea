"""Slab decomposition on the GPU: two processes share this box's one GPU,
each transforms its slab with the library's kernels (obfft_exec_axes), the
exchange is staged through host memory over gloo, and the gathered result is
bit-identical to the single-GPU transform of the whole grid.  The two ranks'
kernels never wait on each other (the exchange is a host-side collective).
Also: the partial-pass and block-transpose entry points on their own."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from synth import inputs as S
from tests.helpers import bits_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2606_23698_gb300 import build as B
    B.build()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, shape, mode, dir, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        from paper_2606_23698_gb300 import SlabPlan
        n0 = shape[0]
        x = S.complex_uniform(51, shape).to("cuda")
        sp = SlabPlan(*shape, world=world, rank=rank, mode=mode, how="host")
        y = sp.exec(x[rank * sp.n0l:(rank + 1) * sp.n0l].contiguous(), dir=dir)
        torch.cuda.synchronize()
        parts = [torch.empty_like(y.cpu()) for _ in range(world)]
        dist.all_gather(parts, y.cpu())
        sp.close()
        if rank == 0:
            full = torch.cat(parts, dim=1).reshape(shape).numpy()
            q.put(full)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("mode,shape,dir", [("fp8", (32, 24, 16), -1), ("fp16", (16, 32, 20), +1),
                                            ("int8", (8, 16, 12), -1), ("fp64", (32, 24, 16), -1)])
def test_two_rank_slab_bit_identical_to_single_gpu(mode, shape, dir):
    from paper_2606_23698_gb300 import Plan
    x = S.complex_uniform(51, shape).to("cuda")
    want = Plan(*shape, mode=mode).exec(x, dir=dir).cpu().numpy()
    torch.cuda.synchronize()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    mp.start_processes(_worker, args=(2, _free_port(), shape, mode, dir, q), nprocs=2, start_method="spawn")
    got = q.get(timeout=300)
    assert bits_equal(got, want), mode


def test_exec_axes_composes_to_exec():
    from paper_2606_23698_gb300 import Plan, _lib
    shape = (12, 20, 16)
    x = S.complex_gaussian(52, shape).to("cuda")
    pl = Plan(*shape, mode="fp8")
    want = pl.exec(x).cpu().numpy()
    s = torch.cuda.current_stream().cuda_stream
    a = torch.empty_like(x)
    b = torch.empty_like(x)
    _lib.obfft_exec_axes(pl.handle, 2, 1, x.data_ptr(), a.data_ptr(), -1, s)
    _lib.obfft_exec_axes(pl.handle, 0, 0, a.data_ptr(), b.data_ptr(), -1, s)
    torch.cuda.synchronize()
    assert bits_equal(b.cpu().numpy(), want)
    with pytest.raises(Exception):
        _lib.obfft_exec_axes(pl.handle, 1, 2, x.data_ptr(), a.data_ptr(), -1, s)
    pl.close()


def test_transpose_blocks():
    from paper_2606_23698_gb300 import _lib
    nb, rows, cols = 3, 5, 7
    src = torch.arange(nb * rows * cols, dtype=torch.float64, device="cuda").to(torch.complex128)
    src = src.reshape(nb, rows, cols)
    dst = torch.empty((rows, nb * cols), dtype=torch.complex128, device="cuda")
    _lib.obfft_transpose_blocks(src.data_ptr(), dst.data_ptr(), nb, rows, cols * 16,
                                torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    want = src.cpu().numpy().transpose(1, 0, 2).reshape(rows, nb * cols)
    assert np.array_equal(dst.cpu().numpy(), want)
    with pytest.raises(Exception):
        _lib.obfft_transpose_blocks(src.data_ptr(), src.data_ptr() + 16, nb, rows, cols * 16, 0)
