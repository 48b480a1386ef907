"""Observation operator (FP64).

Sec. 6, Eq. (obj)/(dis_obj): the data are the state seen by sensors. Here a
sensor is a point x_s in (0,1)^d and observes the bilinear (2D) / trilinear
(3D) interpolant of the grid values; boundary nodes carry the Dirichlet
value 0 and so drop out. A sensor exactly on a node observes that node
alone. Observed steps are obs_every, 2*obs_every, ..., nt (t=0 is never
observed).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp


def observation_matrix(n: int, dim: int, points: np.ndarray) -> sp.csr_matrix:
    """B with B[s, p] = interpolation weight of node p for sensor s.

    Plain loops: for each sensor, each of the 2^d cell corners.
    """
    h = 1.0 / (n + 1)
    rows, cols, vals = [], [], []
    for s, x in enumerate(np.asarray(points, dtype=np.float64)):
        base = []
        frac = []
        for a in range(dim):
            t = x[a] / h                  # position in units of h; node i at t = i+1
            c = math.floor(t)
            base.append(c - 1)            # node index of the lower corner
            frac.append(t - c)
        for corner in range(1 << dim):
            w = 1.0
            idx = []
            for a in range(dim):
                up = (corner >> a) & 1
                w *= frac[a] if up else (1.0 - frac[a])
                idx.append(base[a] + up)
            if w == 0.0:
                continue
            if any(i < 0 or i > n - 1 for i in idx):
                continue                  # boundary node: value 0
            p = 0
            stride = 1
            for a in range(dim):
                p += idx[a] * stride
                stride *= n
            rows.append(s)
            cols.append(p)
            vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(len(points), n ** dim))


def observed_steps(nt: int, every: int):
    return list(range(every, nt + 1, every))
