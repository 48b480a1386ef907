"""Spatial operators (FP64, SciPy sparse).

Grid: n interior nodes per axis, h = 1/(n+1); node (i0, i1, ...) sits at
((i0+1)h, (i1+1)h, ...) and has flat index p = i0 + n*i1 + n^2*i2 (first
coordinate fastest). Zero Dirichlet data on the whole boundary.

L = -div(kappa grad) (Sec. 6, Eq. (pde): the heat equation uses L=-Laplace;
the 3D workload adds a spatially varying diffusivity) discretised in flux
form: every face f between nodes p and q contributes kappa_f/h^2 to L[p,p]
and L[q,q] and -kappa_f/h^2 to L[p,q] and L[q,p]; a face between node p and
the boundary contributes kappa_f/h^2 to L[p,p] only. With kappa = 1 this is
the 5-point (2D) / 7-point (3D) Laplacian.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _node_index(idx, n):
    """Flat index of node coordinates idx[0] (fastest), idx[1], ..."""
    p = np.zeros_like(idx[0])
    stride = 1
    for a in range(len(idx)):
        p = p + idx[a] * stride
        stride *= n
    return p


def laplacian(n: int, dim: int, kappa=None) -> sp.csr_matrix:
    """L = -div(kappa grad_h) with zero Dirichlet data, as a CSR matrix.

    kappa: None (kappa = 1) or a list of dim face arrays in the layout of
    ``synth.kappa_faces`` (C order, axis 0 = last coordinate; faces normal to
    axis d have n+1 entries along d, face i_d lying between node i_d-1 and
    node i_d).
    """
    nx = n ** dim
    h2inv = float(n + 1) ** 2
    rows, cols, vals = [], [], []
    diag = np.zeros(nx)
    for d in range(dim):
        shape = [n] * dim
        shape[d] = n + 1
        # face coordinates, first coordinate first
        grids = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
        if kappa is None:
            kf = np.ones(shape)
        else:
            # stored with the last coordinate as axis 0 -> reverse the axes
            kf = np.asarray(kappa[d], dtype=np.float64).transpose(tuple(range(dim))[::-1])
            assert list(kf.shape) == shape, (kf.shape, shape)
        g = [x.ravel() for x in grids]
        kf = kf.ravel() * h2inv
        lo = [x.copy() for x in g]
        lo[d] = g[d] - 1          # node on the low side of the face
        hi = g                    # node on the high side of the face
        lo_in = lo[d] >= 0
        hi_in = hi[d] <= n - 1
        p_lo = _node_index(lo, n)
        p_hi = _node_index(hi, n)
        np.add.at(diag, p_lo[lo_in], kf[lo_in])
        np.add.at(diag, p_hi[hi_in], kf[hi_in])
        both = lo_in & hi_in
        rows += [p_lo[both], p_hi[both]]
        cols += [p_hi[both], p_lo[both]]
        vals += [-kf[both], -kf[both]]
    rows.append(np.arange(nx))
    cols.append(np.arange(nx))
    vals.append(diag)
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nx, nx))
    return A.tocsr()


def upwind_convection(n: int, dim: int, wind) -> sp.csr_matrix:
    """W = w . grad_h by first-order upwind differences with zero Dirichlet
    data: for w_a > 0, (W y)_p += w_a (y_p - y_{p - e_a}) / h (the upstream
    neighbour is the one on the low side); for w_a < 0, w_a (y_{p + e_a} -
    y_p) / h. Upwinding replaces the paper's SUPG stabilisation of the
    convection-diffusion experiment (Sec. 6.2); W is not symmetric."""
    nx = n ** dim
    hinv = float(n + 1)
    rows, cols, vals = [], [], []
    idx = np.arange(nx)
    coords = []
    rem = idx.copy()
    for a in range(dim):
        coords.append(rem % n)
        rem = rem // n
    for a in range(dim):
        wa = float(wind[a])
        if wa == 0.0:
            continue
        stride = n ** a
        c = abs(wa) * hinv
        rows.append(idx)
        cols.append(idx)
        vals.append(np.full(nx, c))
        if wa > 0:
            has = coords[a] > 0          # upstream neighbour p - e_a inside the grid
            rows.append(idx[has])
            cols.append(idx[has] - stride)
        else:
            has = coords[a] < n - 1      # upstream neighbour p + e_a inside the grid
            rows.append(idx[has])
            cols.append(idx[has] + stride)
        vals.append(np.full(int(has.sum()), -c))
    if not rows:
        return sp.csr_matrix((nx, nx))
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(nx, nx)).tocsr()


def convection_diffusion(n: int, dim: int, nu: float, wind) -> sp.csr_matrix:
    """L = -nu Laplace_h + w . grad_h (Sec. 6.2's operator, upwind convection)."""
    return (nu * laplacian(n, dim, None) + upwind_convection(n, dim, wind)).tocsr()


def shifted(L: sp.spmatrix, c: float) -> sp.csc_matrix:
    """I + c*L: the implicit-Euler step matrix (c = tau, Sec. 6.1, block row
    of Eq. (st_pde) with M = I) or the prior root R (c = alpha)."""
    return (sp.identity(L.shape[0], format="csr") + c * L).tocsc()


def sine_mode(n: int, dim: int, modes) -> np.ndarray:
    """Discrete Dirichlet sine mode prod_a sin(m_a pi x_a) sampled at nodes
    (Sec. 5: the eigenfunctions sin(m pi x1) sin(n pi x2) of the Laplacian)."""
    x = (np.arange(n) + 1.0) / (n + 1)
    v = np.ones(1)
    for a in range(dim):
        s = np.sin(modes[a] * np.pi * x)
        v = np.kron(s, v)  # first coordinate fastest
    return v


def sine_eigenvalue(n: int, modes) -> float:
    """Eigenvalue of the discrete -Laplace_h for a sine mode:
    sum_a (4/h^2) sin^2(m_a pi h / 2) (the discrete analogue of the
    pi^2 (m^2 + n^2) of Sec. 5)."""
    h = 1.0 / (n + 1)
    return float(sum(4.0 / h ** 2 * np.sin(m * np.pi * h / 2.0) ** 2 for m in modes))
