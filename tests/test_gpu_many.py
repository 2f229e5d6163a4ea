"""A10: several grids of uneven sizes in one plan, executed as one captured
CUDA graph; results bit-identical to single-grid plans and to the oracle, the
graph replayed on later calls, and the split autotuner's choice honoured."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from synth import inputs as S
from tests.helpers import bits_equal, mismatch_report, oracle_full

pytestmark = pytest.mark.gpu

DIMS = [(16, 16, 16), (8, 12, 24), (16, 16, 16), (32, 8, 16), (4, 4, 96)]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2606_23698_gb300 import build as B
    B.build()


@pytest.mark.parametrize("mode", ["fp8", "int8", "fp64", "fp16"])
def test_many_matches_single_plans_and_replays(mode, monkeypatch):
    # untuned: the single-grid plans use the default splits too
    monkeypatch.setenv("OBFFT_AUTOTUNE", "0")
    from paper_2606_23698_gb300 import Plan, PlanMany
    xs = [S.complex_gaussian(S.SEED_UNEVEN + i, d).to("cuda") for i, d in enumerate(DIMS)]
    pm = PlanMany(DIMS, mode=mode)
    outs = [torch.empty_like(x) for x in xs]
    for rep in range(3):  # first call captures, later calls replay the graph
        pm.exec(xs, outs, dir=-1)
        torch.cuda.synchronize()
        for d, x, o in zip(DIMS, xs, outs):
            ref = Plan(*d, batch=1, mode=mode).exec(x, dir=-1)
            torch.cuda.synchronize()
            assert bits_equal(o.cpu().numpy(), ref.cpu().numpy()), (mode, d, rep)
    # new pointers: recapture
    outs2 = [torch.empty_like(x) for x in xs]
    pm.exec(xs, outs2, dir=+1)
    torch.cuda.synchronize()
    if mode != "fp64":
        for i, d in enumerate(DIMS[:3]):
            sp = tuple(pm_split(pm, i, a) for a in range(3))
            want = oracle_full(xs[i].cpu().numpy(), sp, +1)
            got = outs2[i].cpu().numpy()
            assert bits_equal(got, want), mismatch_report(got, want)


def pm_split(pm, grid, axis):
    from paper_2606_23698_gb300 import _lib
    return _lib.obfft_plan_get_splits(pm.handle, grid, axis)


def test_autotuned_splits_stay_exact():
    code = r'''
import sys, numpy as np, torch
sys.path.insert(0, %r)
from paper_2606_23698_gb300 import Plan
from synth import inputs as S
from tests.helpers import oracle_full, bits_equal
shape = (8, 96, 48)
x = S.complex_uniform(7, shape).numpy()
pl = Plan(*shape, mode="fp8")
sp = tuple(pl.splits(a) for a in range(3))
y = pl.exec(torch.from_numpy(x).cuda()).cpu().numpy()
assert bits_equal(y, oracle_full(x, sp, -1)), sp
print("splits", sp)
''' % os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, OBFFT_AUTOTUNE="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "splits" in r.stdout


def test_many_single_grid_and_all_identical_grids(monkeypatch):
    """Edge cases of the grouping: a plan of one grid, a plan whose grids all
    share one shape (one batched group), and exec_many on a one-grid plan made
    by obfft_plan_create."""
    monkeypatch.setenv("OBFFT_AUTOTUNE", "0")  # compared with untuned single-grid plans
    from paper_2606_23698_gb300 import Plan, PlanMany, _lib
    d = (8, 12, 16)
    for dims in ([d], [d, d, d]):
        xs = [S.complex_gaussian(40 + i, d).to("cuda") for i in range(len(dims))]
        outs = PlanMany(dims, mode="fp8").exec(xs, dir=-1)
        torch.cuda.synchronize()
        for x, o in zip(xs, outs):
            ref = Plan(*d, mode="fp8").exec(x, dir=-1)
            torch.cuda.synchronize()
            assert bits_equal(o.cpu().numpy(), ref.cpu().numpy()), dims
    pl = Plan(*d, mode="fp8")
    x = S.complex_gaussian(50, d).to("cuda")
    y = torch.empty_like(x)
    _lib.obfft_exec_many(pl.handle, [x.data_ptr()], [y.data_ptr()], -1, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert bits_equal(y.cpu().numpy(), pl.exec(x, dir=-1).cpu().numpy())


@pytest.mark.parametrize("mode", ["fp8", "fp16", "int8"])
def test_many_random_grids_match_oracle(mode):
    """Twelve seeded random grids (repeated shapes form batched groups, the
    rest run alone; the groups are parallel branches of one graph): every
    output bit-exact against the oracle with the plan's splits."""
    from paper_2606_23698_gb300 import PlanMany
    rng = np.random.default_rng(20261205)
    lengths = [2, 5, 8, 12, 16, 24, 32, 48, 64]
    shapes = []
    while len(shapes) < 8:
        d = tuple(int(rng.choice(lengths)) for _ in range(3))
        if d[0] * d[1] * d[2] <= 60000:
            shapes.append(d)
    dims = shapes + [shapes[0], shapes[3], shapes[3], shapes[5]]  # repeats: batched groups
    xs = [S.complex_gaussian(S.SEED_UNEVEN + 100 + i, d).to("cuda") for i, d in enumerate(dims)]
    outs = [torch.empty_like(x) for x in xs]
    pm = PlanMany(dims, mode=mode)
    pm.exec(xs, outs, dir=-1)
    torch.cuda.synchronize()
    for i, d in enumerate(dims):
        sp = tuple(pm_split(pm, i, a) for a in range(3))
        want = oracle_full(xs[i].cpu().numpy(), sp, -1)
        got = outs[i].cpu().numpy()
        assert bits_equal(got, want), (i, d) + (mismatch_report(got, want),)
    pm.close()


def test_many_rejects_overlapping_ranges():
    """The groups run as concurrent graph branches, so an output that overlaps
    another grid's input or output is refused with OBFFT_ERR_ARG (inputs may
    share memory)."""
    from paper_2606_23698_gb300 import ObfftError, _lib
    dims = [(8, 8, 8), (4, 4, 16)]
    pm = _lib.obfft_plan_create_many(dims, _lib.OBFFT_MODE_FP64_NATIVE)
    try:
        buf = torch.zeros(4096, dtype=torch.complex128, device="cuda")
        base = buf.data_ptr()
        s = torch.cuda.current_stream().cuda_stream
        e = 16  # bytes per complex128
        ok = ([base, base + 1024 * e], [base + 2048 * e, base + 2560 * e])
        _lib.obfft_exec_many(pm, ok[0], ok[1], -1, s)
        torch.cuda.synchronize()
        shared_in = ([base, base], [base + 2048 * e, base + 2560 * e])  # one input read by both
        _lib.obfft_exec_many(pm, shared_in[0], shared_in[1], -1, s)
        torch.cuda.synchronize()
        bad = [([base, base + 1024 * e], [base + 2048 * e, base + 100 * e]),    # out 1 inside in 0
               ([base, base + 1024 * e], [base + 2048 * e, base + 2300 * e]),   # out 1 overlaps out 0
               ([base, base + 1024 * e], [base + 1200 * e, base + 3000 * e])]   # out 0 overlaps in 1
        for ins, outs in bad:
            with pytest.raises(ObfftError) as ei:
                _lib.obfft_exec_many(pm, ins, outs, -1, s)
            assert "overlap" in str(ei.value)
    finally:
        _lib.obfft_destroy(pm)


@pytest.mark.parametrize("mode", ["fp8", "fp16"])
def test_default_tuning_reported_and_exact(mode):
    """Multi-grid plans are tuned by default (splits and lines per TMEM lane);
    obfft_plan_get_tuning reports valid choices and the outputs stay
    bit-exact against the oracle with the reported splits."""
    from paper_2606_23698_gb300 import PlanMany, _lib
    dims = [(64, 64, 64), (16, 32, 96), (64, 64, 64), (8, 8, 8)]
    xs = [S.complex_uniform(S.SEED_UNEVEN + 300 + i, d).to("cuda") for i, d in enumerate(dims)]
    pm = PlanMany(dims, mode=mode)
    outs = pm.exec(xs, dir=-1)
    torch.cuda.synchronize()
    for i, d in enumerate(dims):
        sp = []
        for a in range(3):
            p, q, l1, l2 = _lib.obfft_plan_get_tuning(pm.handle, i, a)
            assert p * q == d[a] and max(p, q) <= 32
            for K, lpv in ((q, l1), (p, l2)):
                if d[a] > 1:
                    top = 4 if K <= 8 else (2 if K <= 16 else 1)
                    assert lpv == top or (top == 4 and lpv == 2), (d, a, K, lpv)
            sp.append((p, q))
        want = oracle_full(xs[i].cpu().numpy(), tuple(sp), -1)
        assert bits_equal(outs[i].cpu().numpy(), want), d
    pm.close()


def test_uneven_batch_40_grids_dd_spot_outputs():
    """The 40-grid uneven batch as bench.py times it (16 x 64^3, 12 x
    96x128x128, 8 x 192^3, 4 x 256x256x384, N(0,1) inputs, default tuning),
    FP8 mode, against the oracle's double-double 3-D DFT at eight sampled
    outputs of the first grid of every size: the normwise error over each
    size's samples is below 1e-14 and at most twice the native FP64 kernel's
    on the same grid."""
    from oracle import ref
    from paper_2606_23698_gb300 import Plan, PlanMany
    dims = S.UNEVEN_BATCH
    xs = [S.complex_gaussian(S.SEED_UNEVEN + i, d, device="cuda") for i, d in enumerate(dims)]
    pm = PlanMany(dims, mode="fp8")
    outs = pm.exec(xs, dir=-1)
    torch.cuda.synchronize()
    rng = np.random.default_rng(40)
    firsts = {}
    for i, d in enumerate(dims):
        firsts.setdefault(d, i)
    for d, i in firsts.items():
        spots = [(0, 0, 0)] + [tuple(int(rng.integers(0, n)) for n in d) for _ in range(7)]
        nat = Plan(*d, mode="fp64")
        yn = nat.exec(xs[i], dir=-1)
        torch.cuda.synchronize()
        y8 = outs[i].reshape(d)
        yn = yn.reshape(d)
        got = {"fp8": np.array([complex(y8[k].item()) for k in spots]),
               "fp64": np.array([complex(yn[k].item()) for k in spots])}
        nat.close()
        xh = xs[i].cpu().numpy().reshape(d)
        dd = np.array([ref.dft3d_dd_point(xh, k) for k in spots])
        errs = {}
        for mode, y in got.items():
            dr = (y.real - dd[:, 0]) - dd[:, 1]
            di = (y.imag - dd[:, 2]) - dd[:, 3]
            errs[mode] = float(np.sqrt(np.sum(dr * dr + di * di) / np.sum(dd[:, 0] ** 2 + dd[:, 2] ** 2)))
        print(d, "sampled normwise error vs double-double:", errs)
        assert errs["fp8"] < 1e-14 and errs["fp64"] < 1e-14, (d, errs)
        assert errs["fp8"] <= 2 * errs["fp64"], (d, errs)
    pm.close()
