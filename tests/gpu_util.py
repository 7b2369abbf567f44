"""Helpers shared by the GPU tests (test-side only)."""
import numpy as np
import torch

import bse_inputs as bi


def dev():
    return torch.device("cuda:0")


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev())


def problem_on_device(P):
    return to_dev(P.A), to_dev(P.B)


def rel_fro(X, Y):
    return float(np.linalg.norm(X - Y) / np.linalg.norm(Y))


def starts(n, nevex, seed, nvec=4):
    return bi.start_block(n, nevex, seed), bi.lanczos_starts(n, nvec, seed)
