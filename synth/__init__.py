"""Seeded synthetic inputs shared by the oracle, the tests and the bench.

This module holds problem *data* only: node coordinates and triangles of the
structured meshes, Dirichlet masks and values, initial fields, the wind
function, the random log-diffusion field and the instance list of the batched
workload.  It contains none of the method's arithmetic (no assembly, no
Butcher tables, no solver); both the FP64 oracle and the CUDA path consume
what it returns, each with its own code.

Problems (the paper's test problems, Section 3):
  * heat  u_t = Lap u on the unit square, zero Dirichlet (Eq. testProblemHeat);
  * double glazing  u_t + w.grad u - eps Lap u = 0 on [-1,1]^2, u = 1 on the
    east wall, 0 on the other walls (Eq. testProblemAD), circulating wind
    w = (2y(1-x^2), -2x(1-y^2)).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "Mesh", "MeshP2", "structured_mesh", "structured_mesh_p2", "heat_u0", "double_glazing_wind",
    "double_glazing_boundary", "grf_log_kappa", "random_smooth_u0",
    "batch_instance_sizes", "random_stage_block",
]


class Mesh:
    """Structured triangulation of a rectangle.

    Node (i, j), 0 <= i, j <= N, has index j*(N+1) + i and coordinates
    (x0 + i*hx, y0 + j*hy).  Square (i, j) is cut along its lower-left to
    upper-right diagonal into the counter-clockwise triangles
    ((i,j), (i+1,j), (i+1,j+1)) and ((i,j), (i+1,j+1), (i,j+1)).
    Unknowns are the interior nodes, numbered row by row (i fastest), so the
    stage vectors have n = (N-1)^2 entries.
    """

    def __init__(self, N: int, lo=(0.0, 0.0), hi=(1.0, 1.0)):
        if N < 2:
            raise ValueError("need N >= 2")
        self.N = int(N)
        self.lo = (float(lo[0]), float(lo[1]))
        self.hi = (float(hi[0]), float(hi[1]))
        n1 = N + 1
        ii, jj = np.meshgrid(np.arange(n1), np.arange(n1), indexing="xy")
        ii = ii.ravel()
        jj = jj.ravel()
        hx = (self.hi[0] - self.lo[0]) / N
        hy = (self.hi[1] - self.lo[1]) / N
        self.hx, self.hy = hx, hy
        self.xy = np.stack([self.lo[0] + ii * hx, self.lo[1] + jj * hy], axis=1)
        # exact boundary coordinates (no rounding drift on the far walls)
        self.xy[ii == N, 0] = self.hi[0]
        self.xy[jj == N, 1] = self.hi[1]
        sq_i, sq_j = np.meshgrid(np.arange(N), np.arange(N), indexing="xy")
        a = (sq_j * n1 + sq_i).ravel()
        b = a + 1
        c = a + n1 + 1
        d = a + n1
        t1 = np.stack([a, b, c], axis=1)
        t2 = np.stack([a, c, d], axis=1)
        # interleave so that triangles 2q, 2q+1 belong to square q
        self.tri = np.empty((2 * N * N, 3), dtype=np.int32)
        self.tri[0::2] = t1
        self.tri[1::2] = t2
        self.boundary = (ii == 0) | (ii == N) | (jj == 0) | (jj == N)
        self.dof = np.full(n1 * n1, -1, dtype=np.int32)
        interior = np.flatnonzero(~self.boundary)
        self.dof[interior] = np.arange(interior.size, dtype=np.int32)
        self.interior = interior

    @property
    def n_nodes(self) -> int:
        return self.xy.shape[0]

    @property
    def n_tri(self) -> int:
        return self.tri.shape[0]

    @property
    def n(self) -> int:
        return self.interior.size


class MeshP2:
    """The same triangulation with quadratic (6-node) elements.

    Nodes are the (2N+1)^2 points of the twice-refined lattice: node (I, J),
    0 <= I, J <= 2N, has index J*(2N+1) + I and coordinates (x0 + I*hx/2,
    y0 + J*hy/2); element vertices sit at even (I, J), edge midpoints at the
    others.  Each triangle lists its nodes as (a, b, c, ab, bc, ca): the three
    counter-clockwise vertices of the P1 mesh, then the midpoints of the edges
    a-b, b-c, c-a.  Unknowns are the interior nodes, numbered row by row, so
    n = (2N-1)^2 (the degrees of freedom per stage of the paper's P2 runs)."""

    order = 2

    def __init__(self, N: int, lo=(0.0, 0.0), hi=(1.0, 1.0)):
        if N < 1:
            raise ValueError("need N >= 1")
        self.N = int(N)
        self.lo = (float(lo[0]), float(lo[1]))
        self.hi = (float(hi[0]), float(hi[1]))
        m = 2 * N + 1
        ii, jj = np.meshgrid(np.arange(m), np.arange(m), indexing="xy")
        ii = ii.ravel()
        jj = jj.ravel()
        hx = (self.hi[0] - self.lo[0]) / N
        hy = (self.hi[1] - self.lo[1]) / N
        self.hx, self.hy = hx, hy
        self.xy = np.stack([self.lo[0] + ii * (0.5 * hx), self.lo[1] + jj * (0.5 * hy)], axis=1)
        self.xy[ii == 2 * N, 0] = self.hi[0]
        self.xy[jj == 2 * N, 1] = self.hi[1]
        sq_i, sq_j = np.meshgrid(np.arange(N), np.arange(N), indexing="xy")
        I0 = (2 * sq_i).ravel()
        J0 = (2 * sq_j).ravel()

        def node(di, dj):
            return (J0 + dj) * m + (I0 + di)

        t1 = np.stack([node(0, 0), node(2, 0), node(2, 2), node(1, 0), node(2, 1), node(1, 1)], axis=1)
        t2 = np.stack([node(0, 0), node(2, 2), node(0, 2), node(1, 1), node(1, 2), node(0, 1)], axis=1)
        self.tri = np.empty((2 * N * N, 6), dtype=np.int32)
        self.tri[0::2] = t1
        self.tri[1::2] = t2
        self.boundary = (ii == 0) | (ii == 2 * N) | (jj == 0) | (jj == 2 * N)
        self.dof = np.full(m * m, -1, dtype=np.int32)
        interior = np.flatnonzero(~self.boundary)
        self.dof[interior] = np.arange(interior.size, dtype=np.int32)
        self.interior = interior

    @property
    def n_nodes(self) -> int:
        return self.xy.shape[0]

    @property
    def n_tri(self) -> int:
        return self.tri.shape[0]

    @property
    def n(self) -> int:
        return self.interior.size


def structured_mesh_p2(N: int) -> MeshP2:
    """N x N squares of the unit square, each cut into two 6-node triangles."""
    return MeshP2(N)


def structured_mesh(N: int, domain: str = "unit") -> Mesh:
    """N x N squares cut into right triangles; domain 'unit' = [0,1]^2,
    'box' = [-1,1]^2 (double glazing)."""
    if domain == "unit":
        return Mesh(N)
    if domain == "box":
        return Mesh(N, lo=(-1.0, -1.0), hi=(1.0, 1.0))
    raise ValueError(domain)


def heat_u0(mesh: Mesh) -> np.ndarray:
    """u0 = sin(pi x) sin(pi y) at the interior nodes (length n)."""
    x = mesh.xy[mesh.interior, 0]
    y = mesh.xy[mesh.interior, 1]
    return np.sin(np.pi * x) * np.sin(np.pi * y)


def double_glazing_wind(x, y):
    """Circulating cavity wind w = (2y(1-x^2), -2x(1-y^2))."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    return np.stack([2.0 * y * (1.0 - x * x), -2.0 * x * (1.0 - y * y)], axis=-1)


def double_glazing_boundary(mesh: Mesh) -> np.ndarray:
    """Dirichlet values at every node: 1 on the east wall x = 1 (corners
    included), 0 elsewhere.  Interior entries are 0 (the initial field u0 = 0
    away from the hot wall)."""
    ub = np.zeros(mesh.n_nodes)
    east = mesh.boundary & (mesh.xy[:, 0] == mesh.hi[0])
    ub[east] = 1.0
    return ub


def grf_log_kappa(mesh: Mesh, sigma: float = 0.5, ell: float = 0.1,
                  seed: int = 0) -> np.ndarray:
    """Per-element log-diffusion sampled from a stationary Gaussian random
    field with covariance sigma^2 exp(-r^2 / (2 ell^2)), evaluated at the
    triangle centroids.

    Sampling: circulant embedding on a periodic grid of spacing h/3 padded to
    twice the domain (centroids of both triangle orientations fall on that
    grid); negative embedding eigenvalues are clipped to zero.
    """
    N = mesh.N
    L = mesh.hi[0] - mesh.lo[0]
    g = 3 * N                       # grid points per domain length
    P = 2 * g                       # padded periodic size
    hg = L / g
    k = np.arange(P)
    d = np.minimum(k, P - k) * hg
    r2 = d[:, None] ** 2 + d[None, :] ** 2
    cov = sigma * sigma * np.exp(-r2 / (2.0 * ell * ell))
    lam = np.real(np.fft.fft2(cov))
    lam = np.clip(lam, 0.0, None)
    rng = np.random.default_rng(seed)
    xi = rng.standard_normal((P, P)) + 1j * rng.standard_normal((P, P))
    field = np.real(np.fft.ifft2(np.sqrt(lam) * xi)) * P  # unit-variance scaling
    # centroids: square (i,j): tri 1 at (3i+2, 3j+1), tri 2 at (3i+1, 3j+2)
    si, sj = np.meshgrid(np.arange(N), np.arange(N), indexing="xy")
    si = si.ravel()
    sj = sj.ravel()
    out = np.empty(2 * N * N)
    out[0::2] = field[3 * sj + 1, 3 * si + 2]
    out[1::2] = field[3 * sj + 2, 3 * si + 1]
    return out


def random_smooth_u0(mesh: Mesh, seed: int = 0, kmax: int = 8) -> np.ndarray:
    """u0 = sum_{k,l<=kmax} xi_kl sin(k pi x) sin(l pi y) / (k^2 + l^2) at the
    interior nodes of a unit-square mesh, xi_kl ~ N(0,1) seeded."""
    rng = np.random.default_rng(10_000 + seed)
    xi = rng.standard_normal((kmax, kmax))
    x = mesh.xy[mesh.interior, 0]
    y = mesh.xy[mesh.interior, 1]
    u = np.zeros(x.shape)
    for k in range(1, kmax + 1):
        sx = np.sin(k * np.pi * x)
        for l in range(1, kmax + 1):
            u += xi[k - 1, l - 1] * sx * np.sin(l * np.pi * y) / (k * k + l * l)
    return u


def batch_instance_sizes(count: int = 64, n_min: int = 64, n_max: int = 512):
    """Grid sizes of the uneven batch: N_i = 32 * round(2 * 8^(i/(count-1)))
    for the default 64..512 range (geometric, multiples of 32)."""
    ratio = n_max / n_min
    out = []
    for i in range(count):
        v = (n_min / 32.0) * ratio ** (i / max(count - 1, 1))
        out.append(int(32 * round(v)))
    return out


def random_stage_block(n: int, s: int, seed: int) -> np.ndarray:
    """A seeded (s, n) FP64 block with entries N(0,1) (test vectors)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((s, n))
