"""Helpers for the GPU parity tests (imported only by tests marked gpu)."""
import numpy as np


def dev():
    import torch
    return torch.device("cuda:0")


def to_dev(a: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def c64_to_dev(z: np.ndarray):
    return to_dev(np.ascontiguousarray(z, dtype=np.complex64).view(np.float32))


def c64_from_dev(t) -> np.ndarray:
    return t.cpu().numpy().view(np.complex64)


def sample_rows(batch: int, k: int = 48, seed: int = 7) -> np.ndarray:
    """First, last and k pseudo-random rows of a batch (sorted, unique)."""
    rng = np.random.default_rng(seed)
    rows = set([0, batch - 1])
    rows.update(rng.integers(0, batch, size=min(k, batch)).tolist())
    return np.array(sorted(rows), dtype=np.int64)


def fft_rel_err(X: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """Per-signal relative L2 error ||X - ref|| / ||ref||."""
    return np.linalg.norm(X.astype(np.complex128) - ref, axis=-1) / np.linalg.norm(ref, axis=-1)


def tri_rel_err(x: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """Per-system relative infinity-norm error."""
    return np.max(np.abs(x.astype(np.float64) - ref), axis=-1) / np.max(np.abs(ref), axis=-1)
