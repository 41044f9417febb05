"""Helpers for the GPU tests: build/load the library, move arrays with torch."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def lib_context(model, q_list, max_rhs=2, **kw):
    from paper_1512_06126_gb300 import build, ie
    build.build()
    return ie.Context(model.grid, model.layers, model.sigma_a, model.freqs[:len(q_list)], q_list, max_rhs=max_rhs, **kw)


def to_dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def to_host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
