"""Small helpers shared by the tests (no method arithmetic)."""
import numpy as np


def rel_inf(a, b):
    """max |a - b| / max |b| (relative to the reference b)."""
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def rotation(seed, angle=None):
    g = np.random.Generator(np.random.PCG64(seed))
    axis = g.normal(size=3)
    axis /= np.linalg.norm(axis)
    th = g.uniform(0.2, 1.2) if angle is None else angle
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K
