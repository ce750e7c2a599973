"""Small geometry helpers for tests (no method arithmetic)."""
import numpy as np


def rotation(axis, angle):
    axis = np.asarray(axis, float)
    axis = axis / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * K @ K


def cluster(n=10, seed=0, box_len=40.0, spread=2.2, min_dist=1.8):
    """A compact non-periodic cluster centred in a box much larger than
    2 x cutoff, so periodic images never interact."""
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < n:
        p = rng.normal(0, spread, 3)
        if all(np.linalg.norm(p - q) > min_dist for q in pts):
            pts.append(p)
    pos = np.array(pts) + box_len / 2
    return pos, np.eye(3) * box_len


def cheb_g(r, rc, n, T=None):
    """g_n(r) from scipy's Chebyshev T_n and the cosine cutoff (independent of the oracle)."""
    from scipy.special import eval_chebyt
    x = 2 * (r / rc - 1) ** 2 - 1
    fc = 0.5 * (1 + np.cos(np.pi * r / rc)) if r <= rc else 0.0
    return 0.5 * (eval_chebyt(n, x) + 1) * fc
