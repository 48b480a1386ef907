"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds *no* arithmetic of the method (no operators, no solves, no
observation weights): only the random or fixed raw inputs that both sides take
as given — sensor coordinates, the diffusivity field sampled at face midpoints,
Gaussian blocks — and the workload parameter sets.

Workloads (synthetic stand-ins; the paper publishes no dataset):

* ``tiny``  — 2D heat equation, 31x31 interior (nx=961), nt=100, T=1, prior
  alpha=0.1, 7x7 sensor lattice at (i/8, j/8) observed every 10th step,
  sigma=1e-2, rank k=30.
* ``heat2d_127`` — 2D, 127x127 interior (nx=16129), nt=500, 400 uniform
  sensors observed at every step, sigma=1e-3, alpha=0.05, time truncation
  1e-8 with time rank <= 40, k=100.
* ``heat3d_63`` — 3D, 63^3 interior (250047), kappa=exp(g) with g a smooth
  Gaussian random field (std 0.5, correlation length 0.2), nt=1000, 400
  uniform sensors every 10th step, sigma=1e-3, alpha=0.05, k=200, block 16.
* ``batched`` — 64 independent 2D instances with per-instance grid, nt,
  sensor count and sigma.
* ``serving`` — a Poisson stream of posterior queries.

Seeds: 1000 + workload index, plus the instance or request index.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict
from typing import List, Optional

import numpy as np

WORKLOAD_INDEX = {"tiny": 0, "heat2d_127": 1, "heat3d_63": 2, "batched": 3, "serving": 4}


def rng(seed: int) -> np.random.Generator:
    """The one generator family used for every synthetic input."""
    return np.random.Generator(np.random.PCG64(seed))


def lattice_sensors(per_side: int, dim: int) -> np.ndarray:
    """Sensor points on the regular lattice i/(per_side+1), i=1..per_side.

    Returned as an (per_side**dim, dim) array ordered with the first
    coordinate fastest.
    """
    g = np.arange(1, per_side + 1, dtype=np.float64) / (per_side + 1)
    mesh = np.meshgrid(*([g] * dim), indexing="ij")
    # first coordinate fastest: reverse the axes before flattening
    pts = np.stack([m.transpose(tuple(range(dim))[::-1]).ravel() for m in mesh], axis=1)
    return np.ascontiguousarray(pts)


def uniform_sensors(n_obs: int, dim: int, seed: int) -> np.ndarray:
    """n_obs points uniform in the open unit square/cube."""
    return rng(seed).uniform(0.0, 1.0, size=(n_obs, dim))


def kappa_faces(n: int, dim: int, seed: int, ell: float = 0.2, std: float = 0.5,
                n_features: int = 512) -> List[np.ndarray]:
    """Diffusivity kappa = exp(g) sampled at the face midpoints of the grid.

    g is a random-Fourier-feature draw of a zero-mean Gaussian field with the
    squared-exponential covariance std^2 exp(-|x-x'|^2 / (2 ell^2)):
    g(x) = std * sqrt(2/J) * sum_j cos(w_j . x + phi_j), w_j ~ N(0, ell^-2 I),
    phi_j ~ U[0, 2 pi).

    Grid: interior node i (0-based) along each axis sits at (i+1)h, h=1/(n+1).
    Faces normal to axis d are indexed by i_d = 0..n along that axis (face i_d
    lies between node i_d-1 and node i_d; i_d=0 and i_d=n touch the boundary)
    and 0..n-1 along the other axes. The returned arrays use C order with
    axis 0 = the last coordinate, so the first coordinate is fastest:
    2D: kx.shape=(n, n+1), ky.shape=(n+1, n);
    3D: kx.shape=(n, n, n+1), ky.shape=(n, n+1, n), kz.shape=(n+1, n, n).
    """
    r = rng(seed)
    w = r.normal(0.0, 1.0 / ell, size=(n_features, dim))
    phi = r.uniform(0.0, 2.0 * math.pi, size=n_features)
    h = 1.0 / (n + 1)
    amp = std * math.sqrt(2.0 / n_features)
    out = []
    for d in range(dim):
        # coordinates along each axis (first coordinate = axis index 0)
        axes = []
        for a in range(dim):
            if a == d:
                axes.append((np.arange(n + 1) + 0.5) * h)
            else:
                axes.append((np.arange(n) + 1.0) * h)
        # shape in C order: (coord[dim-1], ..., coord[0])
        grids = np.meshgrid(*axes[::-1], indexing="ij")
        coords = np.stack(grids[::-1], axis=-1)  # [..., dim] with coord 0 first
        shape = coords.shape[:-1]
        xy = coords.reshape(-1, dim)
        g = np.zeros(xy.shape[0])
        # chunk to bound memory
        for s in range(0, n_features, 64):
            arg = xy @ w[s:s + 64].T + phi[s:s + 64]
            g += np.cos(arg).sum(axis=1)
        out.append(np.exp(amp * g).reshape(shape))
    return out


def flatten_kappa(faces: Optional[List[np.ndarray]]) -> Optional[np.ndarray]:
    """Concatenate the face arrays (x faces, then y, then z) in memory order."""
    if faces is None:
        return None
    return np.ascontiguousarray(np.concatenate([f.ravel() for f in faces]))


def normal_block(nx: int, b: int, seed: int) -> np.ndarray:
    """Standard normal (nx, b) block, column j = vector j."""
    return rng(seed).standard_normal(size=(nx, b))


@dataclass
class ProblemSpec:
    """Raw parameters of one inverse problem (no derived operators)."""
    name: str
    dim: int
    n: int
    nt: int
    T: float
    prior_alpha: float
    sigma: float
    obs_every: int
    sensors: np.ndarray = field(repr=False)
    kappa: Optional[List[np.ndarray]] = field(default=None, repr=False)
    k: int = 30
    block: int = 1
    time_trunc_tol: float = 1e-8
    time_rank_max: int = 40
    seed: int = 0
    prior_kind: int = 0       # 0: (I + alpha L0)^-2; 1: gamma I
    prior_gamma: float = 0.0
    pde: str = "heat"         # "heat" or "convdiff" (-nu Laplace + wind . grad)
    conv_nu: float = 0.0
    wind: tuple = (0.0, 0.0, 0.0)

    @property
    def nx(self) -> int:
        return self.n ** self.dim

    @property
    def n_obs(self) -> int:
        return int(self.sensors.shape[0])

    @property
    def obs_steps(self) -> List[int]:
        return list(range(self.obs_every, self.nt + 1, self.obs_every))


def workload(name: str, **overrides) -> ProblemSpec:
    """The parameter set of a named workload (see module docstring)."""
    seed = 1000 + WORKLOAD_INDEX.get(name, 0)
    if name == "tiny":
        spec = ProblemSpec(name=name, dim=2, n=31, nt=100, T=1.0, prior_alpha=0.1,
                           sigma=1e-2, obs_every=10, sensors=lattice_sensors(7, 2),
                           k=30, block=1, seed=seed)
    elif name == "heat2d_127":
        spec = ProblemSpec(name=name, dim=2, n=127, nt=500, T=1.0, prior_alpha=0.05,
                           sigma=1e-3, obs_every=1, sensors=uniform_sensors(400, 2, seed),
                           k=100, block=16, time_trunc_tol=1e-8, time_rank_max=40,
                           seed=seed)
    elif name == "heat3d_63":
        spec = ProblemSpec(name=name, dim=3, n=63, nt=1000, T=1.0, prior_alpha=0.05,
                           sigma=1e-3, obs_every=10, sensors=uniform_sensors(400, 3, seed),
                           kappa=kappa_faces(63, 3, seed + 7), k=200, block=16, seed=seed)
    else:
        raise KeyError(name)
    for k, v in overrides.items():
        setattr(spec, k, v)
    return spec


def _patch_sensors(n: int):
    """Point sensors on every node of the 9 square patches of side 1/16
    (1/256 of the domain) centred at (i/4, j/4), i, j = 1..3: the nodes whose
    coordinates lie in the half-open square [c - 1/32, c + 1/32)^2."""
    h = 1.0 / (n + 1)
    half = (n + 1) // 32  # nodes on each side of a centre (n + 1 a multiple of 32)
    pts = []
    for cj in (1, 2, 3):
        for ci in (1, 2, 3):
            bi, bj = ci * (n + 1) // 4 - half, cj * (n + 1) // 4 - half
            for dj in range(2 * half):
                for di in range(2 * half):
                    pts.append(((bi + di) * h, (bj + dj) * h))
    return np.asarray(pts)


def paper_heat_spec(ratio: float, nt: int = 30) -> ProblemSpec:
    """The 2D heat experiment of the paper's numerical section on finite
    differences: 64 x 64 cells (63^2 interior nodes), nt = 30, T = 1; 9
    square sensor patches of side 1/16 (1/256 of the domain) centred at
    (i/4, j/4), i, j = 1..3, every node of a patch (4 x 4 nodes: the half-open
    square [c - 1/32, c + 1/32)^2) a point sensor, observed at every step;
    Gamma_prior = 10 I; noise level for beta_noise = ratio * beta_prior:
    sigma^2 = 10 / (ratio * tau) (the misfit integral weighs each node and
    step by tau h^2 and the prior term each node by h^2, so Gamma_prior =
    10 I fixes beta_prior h^2 = 0.1 and Gamma_noise^-1 = 0.1 ratio tau)."""
    n = 63
    tau = 1.0 / nt
    sigma = math.sqrt(10.0 / (ratio * tau))
    return ProblemSpec(name=f"paper_heat_r{ratio:g}", dim=2, n=n, nt=nt, T=1.0, prior_alpha=0.0, sigma=sigma,
                       obs_every=1, sensors=_patch_sensors(n), k=50, block=1, seed=1000 + 5,
                       prior_kind=1, prior_gamma=10.0)


def paper_convdiff_spec(nu: float, ratio: float = 1e4, nt: int = 90) -> ProblemSpec:
    """The convection-diffusion experiment of the paper's numerical section on
    finite differences: 32 x 32 cells (31^2 interior nodes), L = -nu Laplace
    + w . grad with w = (0, 1) (upwind differences in place of SUPG), zero
    Dirichlet data (the perturbation problem: the inflow data of the paper's
    example only shift the state and leave the Hessian unchanged), nt = 90,
    T = 1, the 9 sensor patches of the heat experiment (2 x 2 nodes each on
    this grid), Gamma_prior = 10 I and beta_noise = ratio * beta_prior
    (sigma^2 = 10 / (ratio * tau), as for the heat experiment)."""
    n = 31
    tau = 1.0 / nt
    sigma = math.sqrt(10.0 / (ratio * tau))
    return ProblemSpec(name=f"paper_convdiff_nu{nu:g}", dim=2, n=n, nt=nt, T=1.0, prior_alpha=0.0, sigma=sigma,
                       obs_every=1, sensors=_patch_sensors(n), k=50, block=1, seed=1000 + 6,
                       prior_kind=1, prior_gamma=10.0, pde="convdiff", conv_nu=nu, wind=(0.0, 1.0, 0.0))


def small_spec(dim: int = 2, n: int = 7, nt: int = 12, obs_every: int = 3,
               n_obs: int = 5, sigma: float = 0.05, alpha: float = 0.1,
               with_kappa: bool = False, seed: int = 7, lattice: bool = False) -> ProblemSpec:
    """A small problem for oracle pins and parity tests."""
    sensors = lattice_sensors(n_obs, dim) if lattice else uniform_sensors(n_obs, dim, seed)
    kap = kappa_faces(n, dim, seed + 1) if with_kappa else None
    return ProblemSpec(name=f"small{dim}d_n{n}", dim=dim, n=n, nt=nt, T=1.0,
                       prior_alpha=alpha, sigma=sigma, obs_every=obs_every,
                       sensors=sensors, kappa=kap, k=min(8, n ** dim), seed=seed)


def batched_instances(count: int = 64, seed: int = 1000 + WORKLOAD_INDEX["batched"]):
    """Per-instance parameters of the batched workload: grid n in {63,127,255},
    nt uniform in [200, 2000], sensor count uniform in [50, 1000], sigma
    log-uniform in [1e-4, 1e-2]; all steps observed, alpha=0.05, k=50."""
    r = rng(seed)
    out = []
    for i in range(count):
        n = int(r.choice([63, 127, 255]))
        nt = int(r.integers(200, 2001))
        n_obs = int(r.integers(50, 1001))
        sigma = float(10.0 ** r.uniform(-4, -2))
        out.append(ProblemSpec(name=f"inst{i}", dim=2, n=n, nt=nt, T=1.0, prior_alpha=0.05,
                               sigma=sigma, obs_every=1,
                               sensors=uniform_sensors(n_obs, 2, seed * 7919 + i),
                               k=50, block=1, seed=seed + i))
    return out


def serving_requests(count: int = 1000, rate_hz: float = 200.0,
                     seed: int = 1000 + WORKLOAD_INDEX["serving"]):
    """Poisson arrivals (exponential gaps with mean 1/rate) over mixed sizes:
    half 2D 127^2 (nt=500), half 3D with n in {31, 63} (nt=100). Each request
    has sigma log-uniform in [1e-4, 1e-2], a seed for its data and noise,
    1024 query nodes and 8 samples."""
    r = rng(seed)
    t = 0.0
    reqs = []
    for i in range(count):
        t += float(r.exponential(1.0 / rate_hz))
        if r.uniform() < 0.5:
            size = ("2d", 127)
        else:
            size = ("3d", int(r.choice([31, 63])))
        reqs.append(dict(index=i, arrival_s=t, size=size,
                         sigma=float(10.0 ** r.uniform(-4, -2)),
                         seed=seed * 104729 + i, n_query=1024, n_samples=8))
    return reqs


def serving_model_spec(size) -> ProblemSpec:
    """The fixed problem behind each request size of the serving workload:
    ("2d", 127) is the 127^2 workload (nt=500, 400 uniform sensors observed
    at every step); ("3d", n) is the 3D workload's setting on an n^3 grid
    (kappa field, 400 uniform sensors every 10th step) with nt=100. The
    factors are computed at sigma0 = 1e-3 and rescaled per request."""
    dim, n = size
    if dim == "2d":
        return workload("heat2d_127")
    seed = 1000 + WORKLOAD_INDEX["serving"] + n
    return ProblemSpec(name=f"serve3d_n{n}", dim=3, n=n, nt=100, T=1.0, prior_alpha=0.05, sigma=1e-3,
                       obs_every=10, sensors=uniform_sensors(400, 3, seed), kappa=kappa_faces(n, 3, seed + 7),
                       k=50, block=16, seed=seed)


def query_nodes(nx: int, count: int, seed: int) -> np.ndarray:
    """count distinct grid-node indices drawn uniformly (sorted, int32)."""
    count = min(count, nx)
    return np.sort(rng(seed).choice(nx, size=count, replace=False)).astype(np.int32)


def spec_dict(spec: ProblemSpec) -> dict:
    d = asdict(spec)
    d.pop("sensors")
    d.pop("kappa")
    d["n_obs"] = spec.n_obs
    return d
