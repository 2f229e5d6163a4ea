"""A11: the adjoint.  loss = sum |F(x) * w|^2 through the autograd Function;
its gradient must equal the closed form 2 F^H(|w|^2 * F x) computed by the CPU
oracle, and central finite differences (step 1e-6) on sampled coordinates."""
import numpy as np
import pytest
import torch

from oracle import ref
from synth import inputs as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2606_23698_gb300 import build as B
    B.build()


@pytest.mark.parametrize("mode", ["fp8", "int8", "fp64", "fp16"])
def test_gradient_matches_oracle_and_finite_differences(mode):
    from paper_2606_23698_gb300 import fft3_autograd, Plan
    batch, shape = 2, (16, 32, 16)
    x0 = S.complex_uniform(S.SEED_GRAD, (batch,) + shape)
    w = S.spectral_mask(S.SEED_GRAD, (batch,) + shape)
    x = x0.to("cuda").requires_grad_(True)
    wd = w.to("cuda")
    y = fft3_autograd(x, mode)
    loss = (torch.abs(y * wd) ** 2).sum()
    loss.backward()
    g = x.grad.cpu().numpy()
    # oracle gradient: 2 F^H (|w|^2 F x), with the plan's splits
    pl = Plan(*shape, batch=batch, mode=mode)
    splits = tuple(pl.splits(a) for a in range(3))
    xn, wn = x0.numpy(), w.numpy()
    Fx, _ = ref.obfft3d(xn, splits, -1, use_crt=False)
    gref, _ = ref.obfft3d((np.abs(wn) ** 2) * Fx, splits, +1, use_crt=False)
    gref = 2 * gref
    assert np.linalg.norm(g - gref) / np.linalg.norm(gref) < 1e-13
    # central finite differences on sampled real/imaginary coordinates
    rng = np.random.default_rng(0)
    flat = x0.reshape(-1)
    h = 1e-6

    def L(v):
        yy = fft3_autograd(v.reshape(x0.shape).to("cuda"), mode)
        return float((torch.abs(yy * wd) ** 2).sum())

    for idx in rng.choice(flat.numel(), size=16, replace=False):  # 32 real coordinates
        for part in (1.0, 1j):
            xp = flat.clone()
            xm = flat.clone()
            xp[idx] += h * part
            xm[idx] -= h * part
            fd = (L(xp) - L(xm)) / (2 * h)
            # PyTorch's complex gradient is dL/dRe + i dL/dIm
            an = g.reshape(-1)[idx].real if part == 1.0 else g.reshape(-1)[idx].imag
            assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (idx, part, fd, an)
