"""Hand-built scenes for the oracle pins (no method arithmetic beyond the input recipe)."""
import math

import numpy as np

from paper_2509_13536_gb300 import scenegen as sg

Y00 = 1.0 / (2.0 * math.sqrt(math.pi))  # degree-0 real spherical harmonic


def logit(o):
    return math.log(o) - math.log1p(-o)


def make_scene(means, scales, quats, opacities, colours, sh_degree=0, sh=None, birth=None):
    n = len(means)
    k = (sh_degree + 1) ** 2
    if sh is None:
        sh = np.zeros((n, k, 3))
        sh[:, 0, :] = (np.asarray(colours, np.float64).reshape(n, 3) - 0.5) / Y00
    f = np.float32
    return sg.Scene(np.asarray(means, f).reshape(n, 3), np.log(np.asarray(scales, np.float64)).astype(f).reshape(n, 3),
                    np.asarray(quats, f).reshape(n, 4),
                    np.array([logit(o) for o in opacities], f), np.asarray(sh, f).reshape(n, k, 3),
                    np.arange(n, dtype=np.uint64) if birth is None else np.asarray(birth, np.uint64),
                    sh_degree)


def camera(width, height, fx, fy, cx, cy, R=None, t=None):
    return sg.Camera(np.eye(3, dtype=np.float32) if R is None else np.asarray(R, np.float32),
                     np.zeros(3, np.float32) if t is None else np.asarray(t, np.float32),
                     fx, fy, cx, cy, width, height)


def random_scene(rng, n, sh_degree=0, spread=1.0, depth=3.0):
    means = rng.uniform(-spread, spread, size=(n, 3)) + np.array([0, 0, depth])
    scales = np.exp(rng.uniform(math.log(0.02), math.log(0.2), size=(n, 3)))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    q *= rng.uniform(0.5, 2.0, size=(n, 1))  # un-normalised on purpose
    op = rng.uniform(0.1, 0.9, size=n)
    k = (sh_degree + 1) ** 2
    sh = rng.normal(0, 0.3, size=(n, k, 3))
    sh[:, 0, :] = (rng.random((n, 3)) - 0.5) / Y00
    return make_scene(means, scales, q, op, None, sh_degree, sh)
