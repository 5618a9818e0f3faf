"""Seeded synthetic functional data for multi-dimensional FPCA.

This module draws inputs only. It holds none of the estimator's arithmetic
(no binning, no smoothing, no solve, no eigendecomposition): both the FP64
oracle and the CUDA path take their inputs from here, so the two sides see
the same numbers and share nothing else.

Data follow the observation model of Section 2.1, Eq. (2.1)-(2.2):
    Y_ij = mu(t_ij) + sum_l A_il phi_l(t_ij) + eps_ij,
with A_il ~ N(0, lambda_l) uncorrelated and eps_ij ~ N(0, sigma^2).

The workload shapes follow the paper's simulation designs (Section 4:
Simulation I is a 1-D design with Fourier-type eigenfunctions, Simulation II
a 3-D grid with sine-product eigenfunctions and mean exp{(t-.5)'(t-.5)}):

  * ``dense_2d_full``   n=50 surfaces on a full 16x16 grid, four eigenfunctions
  * ``dense_2d_disk``   n=1000 surfaces on a 64x64 grid, disk domain, 10% dropout
  * ``sparse_2d``       n=20000 subjects with 5..20 uniform points each
  * ``dense_3d``        n=2000 volumes on a 32^3 grid, ten eigenfunctions

Eigenfunctions are tensor products of the 1-D functions sqrt(2) sin(2 pi m x)
and sqrt(2) cos(2 pi m x), ordered by the total frequency sum(m), then by the
frequency tuple lexicographically, then sine before cosine per coordinate.
Grid nodes sit at bin centres (k + 1/2)/M, where these products are exactly
orthonormal under the Riemann sum with cell volume prod(1/M_k) whenever every
frequency is below M/2.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1510044390


# ----------------------------------------------------------------------------
# basis functions (the true model; used to synthesise data and to score
# recovered eigenfunctions, never by the estimator itself)
# ----------------------------------------------------------------------------

def fourier_basis_specs(d: int, count: int):
    """Return ``count`` (freqs, types) tuples for d-dim tensor Fourier products.

    ``types[k]`` is 's' or 'c' for sqrt(2) sin / sqrt(2) cos along axis k.
    """
    specs = []
    total = d
    while len(specs) < count:
        freqs_at_total = sorted(
            f for f in itertools.product(range(1, total + 1), repeat=d) if sum(f) == total
        )
        for freqs in freqs_at_total:
            for types in itertools.product("sc", repeat=d):
                specs.append((tuple(freqs), tuple(types)))
                if len(specs) == count:
                    return specs
        total += 1
    return specs


def eval_fourier(spec, pts: np.ndarray) -> np.ndarray:
    """Evaluate one tensor-product basis function at points ``pts`` (N x d)."""
    freqs, types = spec
    out = np.ones(pts.shape[0])
    for k, (m, ty) in enumerate(zip(freqs, types)):
        arg = 2.0 * math.pi * m * pts[:, k]
        out = out * (math.sqrt(2.0) * (np.sin(arg) if ty == "s" else np.cos(arg)))
    return out


def mean_sincos(pts: np.ndarray) -> np.ndarray:
    """mu(t) = sin(2 pi t1) cos(2 pi t2) (2-D designs)."""
    return np.sin(2 * math.pi * pts[:, 0]) * np.cos(2 * math.pi * pts[:, 1])


def mean_exp(pts: np.ndarray) -> np.ndarray:
    """mu(t) = exp{(t - .5)'(t - .5)}, the 3-D mean of Simulation II."""
    c = pts - 0.5
    return np.exp(np.sum(c * c, axis=1))


def mean_1d(pts: np.ndarray) -> np.ndarray:
    """A smooth 1-D mean on [0,1] (Simulation I's t + sin t mapped to [0,1])."""
    t = 10.0 * pts[:, 0]
    return (t + np.sin(t)) / 10.0


def grid_centres(m) -> np.ndarray:
    """Bin centres (k + 1/2)/M of a regular grid, flattened in C order (P x d)."""
    axes = [(np.arange(mk) + 0.5) / mk for mk in m]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([a.ravel() for a in mesh], axis=1)


# ----------------------------------------------------------------------------
# datasets
# ----------------------------------------------------------------------------

@dataclass
class DenseData:
    """Functional data observed at the nodes of a regular grid.

    y    : (n, P) float64, value at node p (undefined where mask is 0)
    mask : (n, P) uint8, 1 where subject i is observed at node p
    """
    d: int
    m: tuple
    y: np.ndarray
    mask: np.ndarray
    lam: np.ndarray
    specs: list
    mean_fn: object
    sigma: float
    seed: int
    name: str = ""

    @property
    def n(self):
        return self.y.shape[0]

    @property
    def P(self):
        return int(np.prod(self.m))

    def true_mean(self):
        return self.mean_fn(grid_centres(self.m))

    def true_phi(self):
        """(P, L) true eigenfunctions at the grid nodes."""
        c = grid_centres(self.m)
        return np.stack([eval_fourier(s, c) for s in self.specs], axis=1)

    def true_gamma(self):
        ph = self.true_phi()
        return (ph * self.lam) @ ph.T


@dataclass
class SparseData:
    """Longitudinal data: subject i owns observations offs[i]:offs[i+1].

    t : (N, d) float64 locations in [0,1]^d;  y : (N,) float64 values.
    """
    d: int
    m: tuple
    offs: np.ndarray
    t: np.ndarray
    y: np.ndarray
    lam: np.ndarray
    specs: list
    mean_fn: object
    sigma: float
    seed: int
    fold: np.ndarray = field(default=None)
    nfold: int = 0
    name: str = ""

    @property
    def n(self):
        return self.offs.shape[0] - 1

    @property
    def P(self):
        return int(np.prod(self.m))


def _scores(rng, n, lam):
    return rng.standard_normal((n, lam.shape[0])) * np.sqrt(lam)[None, :]


def make_dense(d, m, n, lam, n_comp=None, sigma=0.5, mean="sincos", seed=0,
               domain="full", dropout=0.0, name=""):
    """Draw n surfaces on the full grid ``m`` and mask them.

    domain  'full' | 'disk' (cells whose centre lies within 0.5 of (.5,...,.5))
    dropout i.i.d. Bernoulli probability of dropping a remaining point.
    """
    rng = np.random.default_rng(seed)
    lam = np.asarray(lam, dtype=np.float64)
    specs = fourier_basis_specs(d, lam.shape[0] if n_comp is None else n_comp)
    mean_fn = {"sincos": mean_sincos, "exp": mean_exp, "1d": mean_1d, "zero":
               (lambda p: np.zeros(p.shape[0]))}[mean]
    c = grid_centres(m)
    P = c.shape[0]
    phi = np.stack([eval_fourier(s, c) for s in specs], axis=1)
    xi = _scores(rng, n, lam)
    y = mean_fn(c)[None, :] + xi @ phi.T + sigma * rng.standard_normal((n, P))
    inside = np.ones(P, dtype=bool)
    if domain == "disk":
        inside = np.sum((c - 0.5) ** 2, axis=1) <= 0.25
    mask = np.broadcast_to(inside, (n, P)).copy()
    if dropout > 0:
        mask &= rng.random((n, P)) >= dropout
    return DenseData(d=d, m=tuple(m), y=y, mask=mask.astype(np.uint8), lam=lam, specs=specs,
                     mean_fn=mean_fn, sigma=sigma, seed=seed, name=name)


def make_sparse(d, m, n, lam, nmin=5, nmax=20, sigma=0.5, mean="sincos", seed=0,
                nfold=5, name=""):
    """Draw n subjects with Uniform{nmin..nmax} points uniform on [0,1]^d."""
    rng = np.random.default_rng(seed)
    lam = np.asarray(lam, dtype=np.float64)
    specs = fourier_basis_specs(d, lam.shape[0])
    mean_fn = {"sincos": mean_sincos, "exp": mean_exp, "1d": mean_1d}[mean]
    Ni = rng.integers(nmin, nmax + 1, size=n)
    offs = np.zeros(n + 1, dtype=np.int64)
    offs[1:] = np.cumsum(Ni)
    N = int(offs[-1])
    t = rng.random((N, d))
    xi = _scores(rng, n, lam)
    phi = np.stack([eval_fourier(s, t) for s in specs], axis=1)
    subj = np.repeat(np.arange(n), Ni)
    y = mean_fn(t) + np.sum(xi[subj] * phi, axis=1) + sigma * rng.standard_normal(N)
    fold = None
    if nfold > 0:
        fold = (rng.permutation(n) % nfold).astype(np.int32)
    return SparseData(d=d, m=tuple(m), offs=offs, t=t, y=y, lam=lam, specs=specs,
                      mean_fn=mean_fn, sigma=sigma, seed=seed, fold=fold, nfold=nfold,
                      name=name)


def gaussian_test_matrix(P, l, seed):
    """Omega: P x l standard normal test matrix of the random projection."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((P, l))


# ----------------------------------------------------------------------------
# the named workloads
# ----------------------------------------------------------------------------

def dense_2d_full(seed_offset=0, n=50):
    """n=50 surfaces on a full 16x16 grid: lambda=(8,4,2,1), var(eps)=0.25."""
    return make_dense(2, (16, 16), n, [8.0, 4.0, 2.0, 1.0], sigma=0.5, mean="sincos",
                      seed=SEED_BASE + 0 + seed_offset, name="dense_2d_full_16x16_n50")


def dense_2d_disk(seed_offset=0, n=1000, m=64):
    """n=1000 surfaces on 64x64, disk domain, 10% dropout, 8 components, sigma=.5."""
    lam = [8.0 * 2.0 ** (-k) for k in range(8)]
    return make_dense(2, (m, m), n, lam, sigma=0.5, mean="sincos",
                      seed=SEED_BASE + 1 + seed_offset, domain="disk", dropout=0.1,
                      name=f"dense_2d_disk_{m}x{m}_n{n}")


def sparse_2d(seed_offset=0, n=20000, m=64):
    """n=20000 subjects, Uniform{5..20} points on [0,1]^2, 6 components, sigma=.5."""
    lam = [8.0 * 2.0 ** (-k) for k in range(6)]
    return make_sparse(2, (m, m), n, lam, sigma=0.5, mean="sincos",
                       seed=SEED_BASE + 2 + seed_offset, nfold=5,
                       name=f"sparse_2d_{m}x{m}_n{n}")


def dense_3d(seed_offset=0, n=2000, m=32):
    """n=2000 volumes on 32^3, 10 components with lambda_k=10/k, sigma=.3."""
    lam = [10.0 / (k + 1) for k in range(10)]
    return make_dense(3, (m, m, m), n, lam, sigma=0.3, mean="exp",
                      seed=SEED_BASE + 3 + seed_offset, name=f"dense_3d_{m}^3_n{n}")


def cv_bandwidth_grid(nh=16, lo=0.03, hi=0.3):
    """16 isotropic bandwidths log-spaced over [0.03, 0.3]."""
    return np.exp(np.linspace(math.log(lo), math.log(hi), nh))
