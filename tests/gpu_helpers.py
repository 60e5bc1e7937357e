"""Shared helpers for the GPU parity tests: move canonical oracle arrays into
the library's device layout and back."""
import numpy as np
import torch

from paper_2103_05034_gb300 import layout

DEV = "cuda"


def half_dev(psi, L, parity, prec):
    return torch.from_numpy(layout.complex_to_real(layout.to_half(psi, L, parity), prec)).to(DEV)


def full_dev(psi, L, prec):
    return torch.from_numpy(layout.complex_to_real(layout.to_full(psi, L), prec)).to(DEV)


def dev_to_half(t, Ls):
    return layout.real_to_complex(t.double().cpu().numpy()).reshape(-1, 4, 3, Ls)


def dev_to_full_canon(t, L, Ls):
    return layout.from_full(layout.real_to_complex(t.double().cpu().numpy()).reshape(2, -1, 4, 3, Ls), L)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
