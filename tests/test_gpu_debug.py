"""Integer-stage parity: every integer the kernels compute, against the oracle.

obfft_exec_debug runs one Bailey stage and dumps, per DFT column and output,
the kernel's column exponent e, the deconstructed x~, its CRT operands, its
Phase-A accumulators, its lift quotient and the centred CRT value R
(Algorithm 1 one half, Algorithm 2).  The oracle's stage (oracle/ozaki_ref.c,
`ref.stage(dump=True)`) is fed the same stage input (the GPU's own pass
inputs, as the transform runs them) and its integers are compared:

* e and x~ bit-exact;
* INT8 mode: D, E, F mod m_k and the canonical combine v_k bit-exact;
* tensor-core modes: the kernel feeds the CRT offset residues r + 1024 with
  r = v_k (mod m_k) and |r| <= m_k/2 + 1 (any representative of the residue
  class gives the same CRT value; the offset is removed with the Kulisch
  bias).  Reading used here: the residue is checked modulo m_k against the
  oracle's canonical v_k, the range is checked, and the Phase-A words are
  checked exactly against sum_k (r_k + 1024) u_k^(s) and sum_k (r_k + 1024)
  w_k^(t) recomputed from the dumped operands with the oracle's constants;
* the lift: zhat equals the rounding of the dumped lift partials, and
  E - zhat M - 1024 equals R up to the two-sided correction (0 or +-M);
* R bit-exact (128 bits) against the oracle's R, for every output.

In full at 64^3 (every mode, both stages of every axis pass); on sampled
columns at 1024^3.
"""
import numpy as np
import pytest
import torch

from oracle import constants as C
from oracle import ref
from synth import inputs as S

pytestmark = pytest.mark.gpu

MODES = ["fp8", "fp16", "int8", "fp32"]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2606_23698_gb300 import build as B
    B.build()


def _sections(buf, off, ncols, K, nm, na):
    b = buf
    return dict(
        e=b[off[0]:off[0] + ncols * 4].view(np.int32),
        xt=b[off[1]:off[1] + ncols * K * 16].view(np.int64).reshape(ncols, K, 2),
        def_=b[off[2]:off[2] + ncols * K * nm * 6].view(np.uint16).reshape(ncols, K, nm, 3),
        res=b[off[3]:off[3] + ncols * K * 2 * nm * 2].view(np.uint16).reshape(ncols, K, 2, nm),
        acc=b[off[4]:off[4] + ncols * K * 2 * na * 4].view(np.uint32).reshape(ncols, K, 2, na),
        zhat=b[off[5]:off[5] + ncols * K * 16].view(np.int64).reshape(ncols, K, 2),
        R=b[off[6]:off[6] + ncols * K * 32].view(np.uint32).reshape(ncols, K, 2, 4))


def _run_debug(pl, axis, stage, x, col0, ncols):
    from paper_2606_23698_gb300 import _lib
    p, q = pl.splits(axis)
    K = q if stage == 1 else p
    off = _lib.obfft_debug_layout(pl.mode, K, K, ncols)
    dump = torch.empty(off[7], dtype=torch.uint8, device="cuda")
    out = torch.empty_like(x)
    _lib.obfft_exec_debug(pl.handle, axis, stage, x.data_ptr(), out.data_ptr(), -1, col0, ncols, dump.data_ptr(),
                          torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    fp32 = pl.mode == 4
    nm, na = (6, 11) if fp32 else (12, 21)
    return out, _sections(dump.cpu().numpy(), off, ncols, K, nm, na)


def _stage_columns(a, L, p, q, stage):
    """Columns of one stage in the debug (logical) order: stage 1 c = l p + j1,
    elements j2; stage 2 c = k2 L + l, elements j1 (a = the stage input as [L][n])."""
    if stage == 1:
        return a.reshape(L, q, p).transpose(0, 2, 1).reshape(L * p, q), None
    cols = a.reshape(L, q, p).transpose(1, 0, 2).reshape(q * L, p)
    return cols, np.repeat(np.arange(q, dtype=np.int32), L)


def _R128(words):
    w = words.astype(object)
    v = w[..., 0] + (w[..., 1] << 32) + (w[..., 2] << 64) + (w[..., 3] << 96)
    return v


def _check_stage(mode, dump, want, sel):
    """Compare the kernel's dump with the oracle's (both for the columns `sel`)."""
    fp32 = mode == "fp32"
    moduli = np.array(C.MODULI_FP32 if fp32 else C.MODULI, np.int64)
    us = np.array(C.U_SLICES_FP32 if fp32 else C.U_SLICES, np.int64)      # [k][s]
    ws = np.array(C.W_SLICES_FP32 if fp32 else C.W_SLICES, np.int64)      # [k][t]
    M = C.M_FP32 if fp32 else C.M
    ns, nt = us.shape[1], ws.shape[1]
    assert np.array_equal(dump["e"], want["col_exp"][sel]), "column exponents"
    assert np.array_equal(dump["xt"], want["xt"][sel]), "deconstructed integers"
    v = want["v"][sel].astype(np.int64)                                      # [c][k][2][nm]
    res = dump["res"].astype(np.int64)
    if mode == "int8":
        assert np.array_equal(dump["def_"], want["def"][sel]), "D, E, F mod m_k"
        assert np.array_equal(res, v), "canonical combine v_k"
    else:
        r = res - 1024
        assert np.all(np.abs(r) <= moduli // 2 + 1), "offset residue range"
        assert np.array_equal(np.mod(r, moduli), v), "offset residues = v_k (mod m_k)"
        acc = dump["acc"].astype(np.int64) - 0x4B000000
        P, Q = acc[..., :ns], acc[..., ns:ns + nt]
        assert np.array_equal(P, res @ us), "Phase-A slice sums"
        assert np.array_equal(Q, res @ ws), "Phase-A lift partials"
        fb = 24 if fp32 else 48
        z = (Q << (8 * np.arange(nt))).sum(-1)
        assert np.array_equal(dump["zhat"], (z + (1 << (fb - 1))) >> fb), "lift quotient"
    # the exact centred CRT value of every output
    if fp32:
        R = dump["R"][..., 0].astype(np.uint64) | (dump["R"][..., 1].astype(np.uint64) << np.uint64(32))
        assert np.array_equal(R.view(np.int64), want["R"][sel]), "R"
    else:
        lo = want["Rlimbs"][sel][..., 0].astype(np.uint64)
        hi = want["Rlimbs"][sel][..., 1].astype(np.uint64)
        w = np.stack([lo & 0xFFFFFFFF, lo >> np.uint64(32), hi & 0xFFFFFFFF, hi >> np.uint64(32)], -1)
        assert np.array_equal(dump["R"].astype(np.uint64), w), "R (128 bits)"
    # lift identity on a sample of outputs: E - zhat M - offset = R (+- M)
    rng = np.random.default_rng(7)
    flat = dump["res"].reshape(-1, dump["res"].shape[-1])
    idx = rng.choice(flat.shape[0], size=min(400, flat.shape[0]), replace=False)
    zh = dump["zhat"].reshape(-1)[idx]
    Rv = _R128(dump["R"].reshape(-1, 4)[idx])
    u = C.U_FP32 if fp32 else C.U
    for i, j in enumerate(idx):
        E = sum(int(flat[j, k]) * u[k] for k in range(len(u)))
        Rj = int(Rv[i])
        Rj = Rj - (1 << 128) if Rj >= (1 << 127) else Rj
        off = 0 if mode == "int8" else 1024
        d = E - int(zh[i]) * M - off - Rj
        assert d in (0, M, -M), (j, d)


@pytest.mark.parametrize("mode", MODES)
def test_integer_stages_64cube_in_full(mode):
    from paper_2606_23698_gb300 import Plan
    shape = (64, 64, 64)
    pl = Plan(*shape, mode=mode)
    prec = "fp32" if mode == "fp32" else "fp64"
    ctype, sexp = ref.PRECISIONS[prec]
    st = ref.stage if prec == "fp64" else ref.stage32
    x = S.complex_uniform(S.SEED_64, shape).numpy().astype(ctype)
    a = torch.from_numpy(x).to("cuda")
    for axis in (2, 1, 0):
        p, q = pl.splits(axis)
        n = shape[axis]
        L = x.size // n
        for stage in (1, 2):
            K = q if stage == 1 else p
            ncols = L * (p if stage == 1 else q)
            out, dump = _run_debug(pl, axis, stage, a, 0, ncols)
            ah = a.cpu().numpy().reshape(L, n)
            cols, grp = _stage_columns(ah, L, p, q, stage)
            tab = ref.table_q(q, -1, sexp) if stage == 1 else ref.table_p(p, q, -1, sexp)
            y, mism, want = st(cols, tab, grp, True, dump=True)
            assert mism == 0
            _check_stage(mode, dump, want, slice(None))
            # the stage output itself, bit for bit
            oh = out.cpu().numpy()
            if stage == 1:
                wy = y.reshape(L, p, q).transpose(0, 2, 1).reshape(-1)
            else:
                wz = y.reshape(q, L, p).transpose(1, 0, 2)           # [l][k2][k1]
                Y = wz.transpose(0, 2, 1).reshape(L, n)              # pass output, line order
                # rotated layout [n][A1][A2]: element (l, k) at k * L + l
                wy = np.ascontiguousarray(Y.T).reshape(-1)
            word = np.uint32 if prec == "fp32" else np.uint64
            assert np.array_equal(oh.reshape(-1).view(word), wy.view(word)), (mode, axis, stage)
            a = out
    pl.close()


@pytest.mark.parametrize("mode", ["fp8", "fp16", "int8"])
def test_integer_stages_1024cube_sampled(mode):
    """1024^3: one axis pass (axis 2), both stages, on sampled column ranges of
    the full-size launch (the dumped columns run inside the same launch as
    all the others)."""
    from paper_2606_23698_gb300 import Plan
    shape = (1024, 1024, 1024)
    pl = Plan(*shape, mode=mode)
    x = S.complex_uniform(S.SEED_1024, shape, device="cuda")
    p, q = pl.splits(2)
    n, L = 1024, 1024 * 1024
    out1 = torch.empty_like(x)
    rng = np.random.default_rng(1024)
    for stage in (1, 2):
        src = x if stage == 1 else out1
        ncols_all = L * (p if stage == 1 else q)
        for col0 in sorted(rng.integers(0, ncols_all - 256, size=3)):
            col0 = int(col0) // 32 * 32
            out, dump = _run_debug(pl, 2, stage, src, col0, 256)
            # the 256 columns' elements from the stage input
            if stage == 1:
                lines = np.arange(col0 // p, (col0 + 255) // p + 1)
                sub = src.reshape(L, n)[torch.from_numpy(lines).cuda()].cpu().numpy()
                cols, _ = _stage_columns(sub, len(lines), p, q, 1)
                cols = cols[col0 - lines[0] * p: col0 - lines[0] * p + 256]
                grp, tab = None, ref.table_q(q, -1)
            else:
                k2 = np.arange(col0, col0 + 256) // L
                l = np.arange(col0, col0 + 256) % L
                a2 = src.reshape(L, q, p)
                cols = a2[torch.from_numpy(l).cuda(), torch.from_numpy(k2).cuda()].cpu().numpy()
                grp, tab = k2.astype(np.int32), ref.table_p(p, q, -1)
            y, mism, want = ref.stage(np.ascontiguousarray(cols), tab, grp, True, dump=True)
            assert mism == 0
            _check_stage(mode, dump, want, slice(None))
            if stage == 1:
                out1 = out
    pl.close()


def test_debug_argument_errors():
    from paper_2606_23698_gb300 import ObfftError, Plan, _lib
    pl = Plan(8, 8, 8, mode="fp64")
    x = torch.zeros(512, dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(ObfftError):  # native modes have no integer stages
        _lib.obfft_exec_debug(pl.handle, 2, 1, x.data_ptr(), y.data_ptr(), -1, 0, 8, y.data_ptr(), 0)
    pl.close()
    pl = Plan(8, 8, 8, mode="fp8")
    p, q = pl.splits(2)  # stage 1 of the axis-2 pass has 64 lines x p columns
    with pytest.raises(ObfftError):  # columns beyond the stage
        _lib.obfft_exec_debug(pl.handle, 2, 1, x.data_ptr(), y.data_ptr(), -1, 64 * p - 4, 8, y.data_ptr(), 0)
    pl.close()
    with pytest.raises(ObfftError):
        _lib.obfft_debug_layout(2, 8, 8, 4)
