"""Shared helpers of the GPU parity tests: move seeded inputs to the device, make handles."""
import numpy as np
import torch

from paper_2301_12836_gb300 import lsm


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda().contiguous()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def handle(medium, omega, precision=lsm.LSM_FP64, green=lsm.LSM_GREEN_EXACT, **kw):
    o = lsm.lsm_default_opts(precision=precision, green=green, **kw)
    dC = dev(medium.dC.astype(np.float64))
    drho = dev(medium.drho.astype(np.float64))
    return lsm.lsm_create(medium.n, medium.h, medium.lam0, medium.mu0, medium.rho0, dC, drho, omega, o)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def field(shape, seed, dtype=np.complex128):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((3,) + shape) + 1j * rng.standard_normal((3,) + shape)).astype(dtype)
