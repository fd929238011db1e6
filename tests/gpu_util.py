"""Helpers for the GPU tests: device buffers through torch, relative errors."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def to_dev(x: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex64)).cuda()


def to_host(t) -> np.ndarray:
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


def relerr(a, b) -> float:
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rng_fields(P, N, seed, scale=1.0):
    r = np.random.default_rng(seed)
    return (r.standard_normal((P, N)) + 1j * r.standard_normal((P, N))) * scale


def stream_ptr() -> int:
    return torch.cuda.current_stream().cuda_stream
