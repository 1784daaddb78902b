"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_21794_gb300 import build
    build.build()
    return torch


def periodic_diff(a, b, L):
    d = np.asarray(a) - np.asarray(b)
    return np.mod(d + L / 2, L) - L / 2


def rel_max(a, b):
    """max |a - b| / max |b| (norm-wise relative error)."""
    a = np.asarray(a, dtype=np.float64); b = np.asarray(b, dtype=np.float64)
    s = np.abs(b).max() if b.size else 1.0
    return float(np.abs(a - b).max() / s) if a.size else 0.0


def cast_state(st, precision):
    """Round a host FP64 state to the storage precision and back (exactly
    what the device arrays hold after init_particles)."""
    dt = np.float32 if precision == 32 else np.float64
    return {k: (None if v is None else v.astype(dt).astype(np.float64)) for k, v in st.items()}
