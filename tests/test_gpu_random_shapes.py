"""GPU parity on seeded random shapes: axis lengths with every split class of
the stage kernels (one, two or four lines per TMEM lane; INT8 with one or two
limb blocks; prime lengths with a trivial factor), random batch sizes and
both directions, every Ozaki mode bit-exact against the oracle."""
import numpy as np
import pytest
import torch

from synth import inputs as S
from tests.helpers import bits_equal, mismatch_report, oracle_full

pytestmark = pytest.mark.gpu

# lengths n = p q with p, q <= 32 (all tcgen05 and INT8 paths), including
# primes (p = 1), squares, and factors on both sides of 8 and 16
LENGTHS = [1, 2, 3, 5, 7, 8, 11, 12, 16, 17, 20, 24, 27, 31, 32, 36, 40, 48, 60, 64, 72, 96, 100, 128, 160, 256]
MODES = ["fp8", "fp16", "int8"]


def _cases(n_cases=96, seed=20261203):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n_cases:
        shape = tuple(int(rng.choice(LENGTHS)) for _ in range(3))
        elems = shape[0] * shape[1] * shape[2]
        if elems > 80000 or elems < 8:
            continue
        batch = int(rng.integers(1, 4)) if elems < 15000 else 1
        out.append((shape, batch, MODES[len(out) % 3], -1 if rng.random() < 0.7 else +1))
    return out


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2606_23698_gb300 import build as B
    B.build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("shape,batch,mode,dirn", _cases())
def test_random_shape_bit_exact(shape, batch, mode, dirn):
    from paper_2606_23698_gb300 import Plan
    pl = Plan(*shape, batch=batch, mode=mode)
    full = (batch,) + shape if batch > 1 else shape
    x = S.complex_gaussian(S.SEED_64 + sum(shape) + batch, full).numpy()
    y = pl.exec(torch.from_numpy(x).cuda(), dir=dirn)
    torch.cuda.synchronize()
    y = y.cpu().numpy()
    splits = tuple(pl.splits(a) for a in range(3))
    ref_ = oracle_full(x, splits, dirn)
    assert bits_equal(y, ref_), mismatch_report(y, ref_)
