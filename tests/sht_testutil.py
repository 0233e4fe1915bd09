"""Shared helpers for the GPU tests (no transform arithmetic here)."""
import numpy as np

# FP64 path tolerance: relative L2 of the whole output and max abs error
# relative to the largest reference magnitude (the FP64 recurrence, FFT and
# contractions each contribute O(1e-15 sqrt(K)) rounding; 1e-12 leaves two
# orders of margin at T639).
FP64_REL_L2 = 1e-12
FP64_REL_MAX = 1e-12


def built_lib():
    from paper_1711_11296_gb300 import build
    return build.build()


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def assert_fp64_close(got, ref, rel_l2_tol=FP64_REL_L2, rel_max_tol=FP64_REL_MAX):
    got = np.asarray(got)
    ref = np.asarray(ref)
    assert got.shape == ref.shape
    r = rel_l2(got, ref)
    scale = np.abs(ref).max() if ref.size else 1.0
    mx = np.abs(got - ref).max() / (scale if scale > 0 else 1.0) if ref.size else 0.0
    assert r <= rel_l2_tol and mx <= rel_max_tol, (r, mx)
    return r, mx


def to_cuda(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda").to(dtype)
