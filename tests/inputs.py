"""Seeded synthetic inputs shared by the oracle tests and the CUDA parity tests.

This module holds none of the method's arithmetic: it only makes bead
conformations (straight rods with Gaussian jitter, in scaled units) and
chain descriptors from a numpy PCG64 stream.  Random numbers that the method
itself draws (thermal noise, equilibrium starts) come from Philox inside the
oracle and inside the CUDA library, never from here.
"""
import numpy as np


def jittered_rods(C: int, M: int, spacing: float = 3.3, jitter: float = 0.3,
                  seed: int = 0) -> np.ndarray:
    """C straight rods of M beads, random orientations, iid Gaussian jitter.

    Returns float64 positions ``[C][3][M]`` with each centroid at the origin.
    """
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(C, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    s = (np.arange(M) - 0.5 * (M - 1)) * spacing
    r = d[:, :, None] * s[None, None, :] + jitter * rng.normal(size=(C, 3, M))
    r -= r.mean(axis=2, keepdims=True)
    return r


def job_ids(C: int, base: int = 0) -> np.ndarray:
    return (base + np.arange(C)).astype(np.uint32)
