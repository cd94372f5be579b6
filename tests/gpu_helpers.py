"""Helpers shared by the -m gpu tests: move seeded numpy inputs to the GPU
and compare states with the oracle."""
import numpy as np

KEYS = ("x", "px", "y", "py", "sigma", "psigma")


def to_gpu(state):
    import torch
    return {k: torch.from_numpy(np.ascontiguousarray(state[k])).cuda() for k in KEYS}


def to_host(state):
    return {k: state[k].cpu().numpy() for k in KEYS}


def rel_state_err(a, b):
    """max over coordinates of max|a-b| / rms(b) (each coordinate's own scale)."""
    out = {}
    for k in KEYS:
        scale = np.sqrt(np.mean(b[k] ** 2)) or 1.0
        out[k] = float(np.max(np.abs(a[k] - b[k])) / scale)
    return out


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
