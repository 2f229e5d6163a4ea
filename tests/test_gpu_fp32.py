"""GPU parity of the FP32-precision variant (Sec. "Ozaki-II for FP32") and its
native FP32 comparator, through the C ABI.

The Ozaki FP32 mode reaches the exact integer sum_j F~ x~ of every stage
(24-bit significands, six moduli) and rounds once to binary32, so every output
float must equal the oracle's bit for bit."""
import numpy as np
import pytest
import torch

from oracle import constants as C
from oracle import ref
from synth import inputs as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2606_23698_gb300 import build as B
    B.build()
    assert torch.cuda.is_available()


def plan(shape, mode="fp32", batch=1):
    from paper_2606_23698_gb300 import Plan
    return Plan(*shape, batch=batch, mode=mode)


def splits_of(pl):
    return tuple(pl.splits(a) for a in range(3))


def c64(x):
    return np.ascontiguousarray(np.asarray(x), dtype=np.complex64)


def run(pl, x_host, dir=-1):
    x = torch.from_numpy(c64(x_host)).cuda()
    y = pl.exec(x, dir=dir)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def oracle32(x, splits, sign):
    y, _ = ref.obfft3d(c64(x), splits, sign, use_crt=False, prec="fp32")
    return y


def same_bits(a, b):
    return np.array_equal(c64(a).view(np.uint32), c64(b).view(np.uint32))


def report(a, b, limit=5):
    av, bv = c64(a).view(np.uint32).ravel(), c64(b).view(np.uint32).ravel()
    af, bf = c64(a).view(np.float32).ravel(), c64(b).view(np.float32).ravel()
    idx = np.nonzero(av != bv)[0]
    return f"{idx.size} of {av.size} floats differ; first: " + ", ".join(
        f"[{i}] {af[i]!r} vs {bf[i]!r}" for i in idx[:limit])


@pytest.mark.parametrize("shape", [(8, 8, 8), (4, 12, 16), (2, 32, 5), (16, 16, 16), (1, 1, 64),
                                   (3, 27, 10), (6, 40, 48), (5, 7, 33)])
def test_fp32_small_grids_bit_exact(shape):
    """Includes odd line lengths and odd stage-2 factors, where the kernel loads
    its input tile with plain loads instead of TMA bulk copies."""
    x = S.complex_uniform(S.SEED_64, shape).numpy()
    pl = plan(shape)
    y = run(pl, x)
    assert y.dtype == np.complex64
    r = oracle32(x, splits_of(pl), -1)
    assert same_bits(y, r), report(y, r)


def test_fp32_64cube_bit_exact_and_accurate():
    shape = (64, 64, 64)
    x = c64(S.complex_uniform(S.SEED_64, shape).numpy())
    pl = plan(shape)
    assert splits_of(pl) == ((8, 8), (8, 8), (8, 8))
    y = run(pl, x)
    r = oracle32(x, splits_of(pl), -1)
    assert same_bits(y, r), report(y, r)
    err = ref.normwise_error(y.astype(np.complex128), ref.dft3d_dd(x.astype(np.complex128)))
    assert err < 12 * 2.0 ** -24


def test_fp32_inverse_and_batch():
    shape = (8, 16, 24)
    x = S.complex_gaussian(7, (3,) + shape).numpy()
    pl = plan(shape, batch=3)
    y = run(pl, x, dir=+1)
    r = oracle32(x, splits_of(pl), +1)
    assert same_bits(y, r), report(y, r)


def test_fp32_edge_inputs():
    shape = (8, 8, 16)
    pl = plan(shape)
    sp = splits_of(pl)
    u = lambda seed: S.complex_uniform(seed, shape).numpy()
    cases = {
        "zeros": np.zeros(shape, np.complex64),
        "impulse": np.zeros(shape, np.complex64),
        "wide": S.complex_wide_range(S.SEED_256_WIDE, shape).numpy(),
        "subnormal": u(3) * 2.0 ** -140,
        "mixed_subnormal": u(6) * np.where(np.arange(16) % 2 == 0, 2.0 ** -130, 2.0 ** -100),
        "huge": u(4) * 2.0 ** 100,
        "sparse_cols": u(5) * (np.arange(16) % 3 == 0),
    }
    cases["impulse"][0, 0, 0] = 1.0
    for name, x in cases.items():
        y = run(pl, x)
        r = oracle32(x, sp, -1)
        assert same_bits(y, r), name + ": " + report(y, r)
    assert np.all(run(pl, cases["impulse"]) == 1.0)


def test_fp32_wide_range_256_stage_sampled():
    shape = (256, 256, 256)
    pl = plan(shape)
    x = S.complex_wide_range(S.SEED_256_WIDE, shape, device="cuda").to(torch.complex64)
    _check_pass_sampled(pl, x, shape, dir=-1, nsample=48)


def test_fp32_four_lines_per_lane_sampled():
    """256 x 256 x 64: the axis-2 stages (K = 8) run four lines per TMEM
    lane, the others (K = 16) two; sampled lines of every stage match the
    oracle bit for bit."""
    shape = (256, 256, 64)
    pl = plan(shape)
    assert pl.splits(2) == (8, 8)
    x = S.complex_uniform(S.SEED_64 + 5, shape, device="cuda").to(torch.complex64)
    _check_pass_sampled(pl, x, shape, dir=-1, nsample=64)


@pytest.mark.parametrize("shape,batch", [((5, 60, 24), 1), ((3, 20, 48), 3), ((1, 240, 12), 1)])
def test_fp32_lines_per_lane_ragged_tiles(shape, batch):
    """Line counts that leave the last tile of a launch or of a twiddle group
    partly empty, with two lines per lane, stay bit-exact."""
    x = S.complex_uniform(S.SEED_64 + 11, (batch,) + shape if batch > 1 else shape).numpy()
    pl = plan(shape, batch=batch)
    y = run(pl, x)
    ref_ = oracle32(c64(x), splits_of(pl), -1)
    assert same_bits(y, ref_), report(y, ref_)


def test_fp32_full_size_1024cube_sampled_and_parseval():
    """1024^3 complex64 (8 GiB), splits 32 x 32: every stage of every axis pass
    matches the oracle on sampled lines; the transform satisfies Parseval."""
    shape = (1024, 1024, 1024)
    if torch.cuda.get_device_properties(0).total_memory < 80 * 2 ** 30:
        pytest.skip("needs ~40 GiB of device memory")
    pl = plan(shape)
    assert splits_of(pl) == ((32, 32), (32, 32), (32, 32))
    x = S.complex_uniform(S.SEED_1024, shape, device="cuda").to(torch.complex64)
    _check_pass_sampled(pl, x, shape, dir=-1, nsample=24)
    y = pl.exec(x, dir=-1)
    torch.cuda.synchronize()
    ex = float(torch.sum(torch.abs(x.to(torch.complex128)) ** 2))
    ey = float(torch.sum(torch.abs(y.to(torch.complex128)) ** 2))
    N = 1024 ** 3
    assert abs(ey - N * ex) / (N * ex) < 1e-5
    del x, y
    torch.cuda.empty_cache()


def _check_pass_sampled(pl, x, shape, dir, nsample):
    rng = np.random.default_rng(1)
    cur = x.clone()
    scratch = torch.empty_like(cur)
    out = torch.empty_like(cur)
    n = list(shape)
    sexp = C.SIGMA_F_EXP_FP32
    for axis in (2, 1, 0):
        p, q = pl.splits(axis)
        N = n[axis]
        L = cur.numel() // N
        pl.exec_stage(axis, 1, cur, scratch, dir)
        pl.exec_stage(axis, 2, scratch, out, dir)
        torch.cuda.synchronize()
        lines = torch.from_numpy(rng.choice(L, size=min(nsample, L), replace=False)).cuda()
        xin = cur.reshape(L, N)[lines].cpu().numpy()
        y1 = scratch.reshape(L, N)[lines].cpu().numpy()
        c1 = xin.reshape(-1, q, p).transpose(0, 2, 1).reshape(-1, q)
        r1, _, _ = ref.stage32(c1, ref.table_q(q, dir, sexp), None, use_crt=False)
        r1 = r1.reshape(-1, p, q).transpose(0, 2, 1).reshape(-1, N)
        assert same_bits(y1, r1), f"axis {axis} stage 1: " + report(y1, r1)
        c2 = y1.reshape(-1, q, p).reshape(-1, p)
        grp = np.tile(np.arange(q, dtype=np.int32), lines.numel())
        r2, _, _ = ref.stage32(c2, ref.table_p(p, q, dir, sexp), grp, use_crt=False)
        z = r2.reshape(-1, q, p).transpose(0, 2, 1).reshape(-1, N)
        got = out.reshape(N, L)[:, lines].T.cpu().numpy()
        assert same_bits(got, z), f"axis {axis} stage 2: " + report(got, z)
        cur, out = out, cur


def test_fp32_native_comparator_and_ozaki_accuracy():
    """The native FP32 six-step comparator and the Ozaki FP32 variant against
    double-double: both at binary32 accuracy; the Ozaki result within 2x of
    the native one's error (or better)."""
    shape = (32, 32, 32)
    x = c64(S.complex_uniform(S.SEED_64, shape).numpy())
    yd = ref.dft3d_dd(x.astype(np.complex128))
    e_nat = ref.normwise_error(run(plan(shape, "fp32native"), x).astype(np.complex128), yd)
    e_oz = ref.normwise_error(run(plan(shape, "fp32"), x).astype(np.complex128), yd)
    assert e_nat < 1e-6 and e_oz < 12 * 2.0 ** -24
    assert e_oz <= 2 * e_nat
    # mixed radix (3 and 5) in the native comparator
    shape2 = (12, 20, 45)
    x2 = c64(S.complex_uniform(9, shape2).numpy())
    e2 = ref.normwise_error(run(plan(shape2, "fp32native"), x2).astype(np.complex128),
                            ref.dft3d_dd(x2.astype(np.complex128)))
    assert e2 < 1e-6


def test_fp32_roundtrip():
    shape = (16, 32, 24)
    x = c64(S.complex_gaussian(11, shape).numpy())
    pl = plan(shape)
    y = run(pl, x, -1)
    z = run(pl, y, +1) / np.float32(np.prod(shape))
    assert np.linalg.norm(z - x) / np.linalg.norm(x) < 16 * 2.0 ** -24


@pytest.mark.parametrize("mode", ["fp32", "fp32native"])
def test_fp32_exec_host_matches_device_exec(mode):
    shape, batch = (64, 96, 128), 2
    pl = plan(shape, mode, batch=batch)
    x = S.complex_gaussian(12, (batch,) + shape).to(torch.complex64)
    yd = pl.exec(x.cuda(), dir=-1).cpu()
    torch.cuda.synchronize()
    yh = pl.exec_host(x.pin_memory(), dir=-1)
    torch.cuda.synchronize()
    assert torch.equal(yh.view(torch.float32), yd.view(torch.float32))


def test_fp32_many_matches_single_plans(monkeypatch):
    monkeypatch.setenv("OBFFT_AUTOTUNE", "0")  # compared with untuned single-grid plans
    from paper_2606_23698_gb300 import PlanMany
    dims = [(16, 16, 16), (8, 24, 12), (32, 32, 32), (4, 4, 64)]
    xs = [S.complex_gaussian(20 + i, d, device="cuda").to(torch.complex64) for i, d in enumerate(dims)]
    pm = PlanMany(dims, mode="fp32")
    ys = pm.exec(xs, dir=-1)
    torch.cuda.synchronize()
    for d, x, y in zip(dims, xs, ys):
        ref_y = plan(d).exec(x, dir=-1)
        torch.cuda.synchronize()
        assert torch.equal(y.view(torch.float32), ref_y.view(torch.float32))


def test_fp32_autograd_adjoint():
    """Backward of the complex64 transform is the conjugate-direction transform:
    the gradient of sum |F(x) w|^2 matches the FP64 mode's to binary32 accuracy."""
    from paper_2606_23698_gb300 import fft3_autograd
    shape = (2, 16, 16, 16)
    x = S.complex_uniform(S.SEED_GRAD, shape, device="cuda")
    w = S.spectral_mask(S.SEED_GRAD, shape, device="cuda")
    grads = {}
    for mode, dt in (("fp32", torch.complex64), ("fp64", torch.complex128)):
        xr = x.to(dt).clone().requires_grad_(True)
        loss = (torch.abs(fft3_autograd(xr, mode) * w.to(dt)) ** 2).sum()
        loss.backward()
        grads[mode] = xr.grad.to(torch.complex128)
    rel = torch.linalg.vector_norm(grads["fp32"] - grads["fp64"]) / torch.linalg.vector_norm(grads["fp64"])
    assert float(rel) < 1e-6


def test_fp32_argument_errors_and_dtype_checks():
    """complex64 plans reject complex128 tensors and the usual bad pointers;
    FP32-precision plans refuse factors above 32."""
    from paper_2606_23698_gb300 import ObfftError, _lib
    pl = plan((8, 8, 8))
    x64 = torch.zeros(512, dtype=torch.complex64, device="cuda")
    x128 = torch.zeros(512, dtype=torch.complex128, device="cuda")
    with pytest.raises(TypeError):
        pl.exec(x128)
    with pytest.raises(ObfftError):
        _lib.obfft_exec(pl.handle, x64.data_ptr(), x64.data_ptr(), -1, 0)      # in == out
    with pytest.raises(ObfftError):
        _lib.obfft_exec(pl.handle, x64.data_ptr() + 8, x64.data_ptr() + 4096, -1, 0)  # misaligned
    with pytest.raises(ObfftError):
        plan((8, 8, 2048))                       # 2048 = 32 x 64: a factor above 32
    y = plan((8, 8, 4096), "fp32native")         # 64 x 64: the native comparator allows it
    y.close()


def test_fp32_stage_entry_matches_oracle_stage():
    """obfft_exec_stage in the FP32 mode: one stage-1 launch against the
    oracle's FP32 stage on every column."""
    shape = (4, 8, 96)
    pl = plan(shape)
    p, q = pl.splits(2)
    x = torch.from_numpy(c64(S.complex_uniform(3, shape).numpy())).cuda()
    out = torch.empty_like(x)
    pl.exec_stage(2, 1, x, out, -1)
    torch.cuda.synchronize()
    L, N = x.numel() // 96, 96
    xin = x.reshape(L, N).cpu().numpy()
    c1 = xin.reshape(-1, q, p).transpose(0, 2, 1).reshape(-1, q)
    r1, mism, _ = ref.stage32(c1, ref.table_q(q, -1, C.SIGMA_F_EXP_FP32), None, use_crt=True)
    assert mism == 0
    r1 = r1.reshape(-1, p, q).transpose(0, 2, 1).reshape(-1, N)
    got = out.reshape(L, N).cpu().numpy()
    assert same_bits(got, r1), report(got, r1)


def _random_cases(n_cases=48, seed=20261204):
    lengths = [1, 2, 3, 5, 7, 8, 11, 12, 16, 17, 20, 24, 27, 31, 32, 36, 40, 48, 60, 64, 96, 100, 128, 256]
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n_cases:
        shape = tuple(int(rng.choice(lengths)) for _ in range(3))
        elems = shape[0] * shape[1] * shape[2]
        if elems > 80000 or elems < 8:
            continue
        batch = int(rng.integers(1, 4)) if elems < 15000 else 1
        out.append((shape, batch, -1 if rng.random() < 0.7 else +1))
    return out


@pytest.mark.parametrize("shape,batch,dirn", _random_cases())
def test_fp32_random_shape_bit_exact(shape, batch, dirn):
    """Seeded random shapes, batches and directions (one, two and four lines
    per TMEM lane, prime lengths): bit-exact against the oracle."""
    full = (batch,) + shape if batch > 1 else shape
    x = S.complex_gaussian(S.SEED_64 + sum(shape) + batch, full).numpy()
    pl = plan(shape, batch=batch)
    y = run(pl, x, dir=dirn)
    ref_ = oracle32(c64(x), splits_of(pl), dirn)
    assert same_bits(y, ref_), report(y, ref_)
