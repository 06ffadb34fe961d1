"""Shared helpers for the test-suite: build oracle and CUDA lattices from the
same seeded workload object."""
import numpy as np

from oracle import oracle as orc


def as_oracle(p, delta=None):
    return orc.Lattice(p.Lx, p.Ly, p.periodic_x, p.periodic_y, p.eps, p.mu, p.hop, p.pairing,
                       p.coupling, p.delta0 if delta is None else delta)


def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def max_abs(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)))) if np.size(a) else 0.0
