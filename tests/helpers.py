"""Shared test helpers: oracle comparisons for GPU outputs."""
import numpy as np

from oracle import ref


def oracle_full(x, splits, sign):
    """Oracle transform of x [..., n0, n1, n2] (direct exact products: bit-identical
    to the CRT pipeline, which the oracle tests pin separately)."""
    y, _ = ref.obfft3d(x, splits, sign, use_crt=False)
    return y


def bits_equal(a: np.ndarray, b: np.ndarray) -> bool:
    return np.array_equal(np.ascontiguousarray(a).view(np.uint64), np.ascontiguousarray(b).view(np.uint64))


def mismatch_report(a, b, limit=5):
    av = np.ascontiguousarray(a).view(np.uint64).ravel()
    bv = np.ascontiguousarray(b).view(np.uint64).ravel()
    idx = np.nonzero(av != bv)[0]
    af = np.ascontiguousarray(a).view(np.float64).ravel()
    bf = np.ascontiguousarray(b).view(np.float64).ravel()
    return f"{idx.size} of {av.size} doubles differ; first: " + ", ".join(
        f"[{i}] {af[i]!r} vs {bf[i]!r}" for i in idx[:limit])
