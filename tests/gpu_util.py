"""Helpers for the GPU tests: marshalling between numpy AoS and CUDA SoA."""
import numpy as np
import torch


def soa(pos):
    return torch.tensor(np.ascontiguousarray(np.asarray(pos, np.float64).T), dtype=torch.float64, device="cuda")


def aos(t):
    return t.detach().cpu().numpy().T.copy()


def virial_aos(t):
    return t.detach().cpu().numpy().T.reshape(-1, 3, 3)


def f32_exact(z):
    """The parameter vector both sides use: FP32 values, exact in FP64."""
    return np.asarray(z, np.float32).astype(np.float64)
