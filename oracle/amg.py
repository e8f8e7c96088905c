"""Smoothed-aggregation AMG, plain FP64 (oracle; test infrastructure only).

The paper approximates each diagonal-block subsolve (M + h A~_jj F) w_j = v_j
by one AMG V-cycle (Section 4.2) using smoothed aggregation from IFISS
(Section 5).  The paper gives no further parameters; this module follows the
reading fixed in the design notes, step by step:

  strength   i ~ j strong iff  (c_ij + c_ji)/2 >= theta_l sqrt(|a_ii a_jj|) with
             c_ij = |a_ij| (default; max(-a_ij, 0) as an option), symmetrised
             so that nonsymmetric blocks give an undirected graph; theta_l starts at theta (0.08) on every level and is
             halved, at most 6 times, while more than a quarter of the level's
             nodes have no strong coupling (isotropic or mass-dominated blocks
             whose couplings all sit just below the threshold).
  roots      a maximal distance-2 independent set of the strength graph,
             chosen greedily in decreasing priority; priority of node i on
             level l is the 64-bit key (fmix32(i ^ (0x9E3779B9*(l+1))) << 32) | i
             where fmix32 is the MurmurHash3 32-bit finaliser.
  aggregates each root and its strong neighbours form an aggregate (phase 1);
             every other node joins the aggregate of its phase-1 strong
             neighbour of largest priority (phase 2).  Aggregates are
             numbered by increasing root index.
  P          tentative piecewise constant P_t (entries 1), smoothed by
             p_smooth damped-Jacobi steps (default 2) on every level:
             P = (I - omega D^{-1} A)^steps P_t, omega = 4 / (3 rho), rho the
             estimate of the spectral radius of D^{-1} A by 20 steps of the
             power iteration on the similar S = |D|^{-1/2} A |D|^{-1/2} from
             the +-1 vector x_i = +1 iff fmix32(i ^ 0x68E31DA4) is odd:
             x <- S x / ||x||, rho = ||S x_19|| / ||x_19||.
  SUPG       with a streamline-diffusion matrix T and the block coefficient c
             (block M + c F of a SUPG problem), every coarse level adds the
             streamline diffusion of its larger mesh size:
             A_c = P^T A P + c (f_c - f) T_c, T_c = P^T T P, f = sqrt(n_0 / n)
             (the coarse-level stabilisation of Section 5); the stabilised A_c
             is the one that is coarsened further.
  coarse     A_c = P^T A P (Galerkin, R = P^T), until n <= coarse_max (2048) or
             coarsening stalls (the next level would keep more than 90% of the
             rows); the coarsest level is solved directly (dense LU) when it
             has at most coarse_max rows, otherwise by 4 smoothing sweeps from
             zero.
  smoother   l1-Jacobi x <- x + D_l1^{-1} (b - A x), D_l1 = diag(sum_j |a_ij|),
             or Chebyshev of degree k on the l1-scaled operator D_l1^{-1} A,
             whose spectrum lies in (0, 1] for symmetric A (D_l1 - A is
             diagonally dominant); the interval [lo, 1] (lo = 0.1) is fixed, so
             no eigenvalue estimate is needed.  The Chebyshev recurrence is
             the classical three-term one (Saad, Iterative Methods, Alg. 12.1):
               theta = (1+lo)/2, delta = (1-lo)/2, sigma = theta/delta,
               rho_0 = 1/sigma, d_0 = D^{-1}(b - A x_0)/theta, x_1 = x_0 + d_0,
               rho_k = 1/(2 sigma - rho_{k-1}),
               d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k/delta) D^{-1}(b - A x_k),
               x_{k+1} = x_k + d_k.
             V(nu1, nu2) cycle from a zero initial guess (each sweep is one
             l1-Jacobi step or one Chebyshev polynomial of degree k).
  cycle      "V" (the paper's one V-cycle per subsolve, default) or "Wc": the
             finest level is visited once as in the V-cycle, and every coarser
             level l >= 1 whose next level is not the coarsest applies the
             coarse-grid correction twice (residual, restriction, recursion,
             prolongation, then the same again) between its pre- and
             post-smoothing, i.e. a W-cycle below the finest level.  A level
             whose next level is the coarsest corrects once (with the exact
             coarsest solve a second correction would be zero).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

M32 = 0xFFFFFFFF


def fmix32(x: int) -> int:
    """MurmurHash3 32-bit finaliser (Appleby), on a Python int."""
    x &= M32
    x ^= x >> 16
    x = (x * 0x85EBCA6B) & M32
    x ^= x >> 13
    x = (x * 0xC2B2AE35) & M32
    x ^= x >> 16
    return x


def priority_keys(n: int, level: int) -> np.ndarray:
    """64-bit priority keys of nodes 0..n-1 on ``level`` (unique)."""
    salt = (0x9E3779B9 * (level + 1)) & M32
    x = (np.arange(n, dtype=np.uint64) ^ np.uint64(salt)) & np.uint64(M32)
    x ^= x >> np.uint64(16)
    x = (x * np.uint64(0x85EBCA6B)) & np.uint64(M32)
    x ^= x >> np.uint64(13)
    x = (x * np.uint64(0xC2B2AE35)) & np.uint64(M32)
    x ^= x >> np.uint64(16)
    return (x << np.uint64(32)) | np.arange(n, dtype=np.uint64)


def strength_graph(A: sp.csr_matrix, theta: float, negative: bool = False) -> sp.csr_matrix:
    """Boolean symmetric strength graph (no diagonal) as CSR with sorted
    indices.  negative: couplings measured by max(-a_ij, 0) (the off-diagonal
    entries that carry the smooth error in an M-matrix-like block; quadratic
    elements have positive ones), else by |a_ij|."""
    A = A.tocsr()
    A.sort_indices()
    n = A.shape[0]
    d = np.abs(A.diagonal())
    absA = (-A).maximum(0) if negative else abs(A)
    S = 0.5 * (absA + absA.T)          # (c_ij + c_ji) / 2
    S = S.tocoo()
    keep = (S.row != S.col) & (S.data >= theta * np.sqrt(d[S.row] * d[S.col]))
    G = sp.csr_matrix((np.ones(int(keep.sum()), dtype=np.int8),
                       (S.row[keep], S.col[keep])), shape=(n, n))
    G.sort_indices()
    return G


def mis2_roots(G: sp.csr_matrix, level: int) -> np.ndarray:
    """Greedy maximal distance-2 independent set in decreasing priority."""
    n = G.shape[0]
    key = priority_keys(n, level)
    order = np.argsort(key)[::-1]
    ip, ix = G.indptr, G.indices
    UND, ROOT, OUT = 0, 1, 2
    state = np.zeros(n, dtype=np.int8)
    for v in order:
        if state[v] != UND:
            continue
        state[v] = ROOT
        nb1 = ix[ip[v]:ip[v + 1]]
        for u in nb1:
            if state[u] == UND:
                state[u] = OUT
            for w in ix[ip[u]:ip[u + 1]]:
                if state[w] == UND:
                    state[w] = OUT
    return state == ROOT


def aggregate(G: sp.csr_matrix, level: int):
    """Aggregate index per node (0..nc-1) and the root mask."""
    n = G.shape[0]
    root = mis2_roots(G, level)
    key = priority_keys(n, level)
    agg = np.full(n, -1, dtype=np.int64)
    roots = np.flatnonzero(root)
    agg[roots] = np.arange(roots.size)
    ip, ix = G.indptr, G.indices
    phase1 = agg.copy()
    for r in roots:
        for u in ix[ip[r]:ip[r + 1]]:
            phase1[u] = agg[r]
    agg = phase1.copy()
    for v in np.flatnonzero(phase1 < 0):
        nb = ix[ip[v]:ip[v + 1]]
        cand = nb[phase1[nb] >= 0]
        if cand.size == 0:
            raise RuntimeError("node without an aggregated strong neighbour")
        u = cand[np.argmax(key[cand])]
        agg[v] = phase1[u]
    return agg, root


POWER_SALT = 0x68E31DA4
POWER_STEPS = 20


def power_start_vector(n: int) -> np.ndarray:
    """The +-1 start vector of the power iteration: +1 where the MurmurHash3
    finaliser of i ^ POWER_SALT is odd, else -1."""
    x = (np.arange(n, dtype=np.uint64) ^ np.uint64(POWER_SALT)) & np.uint64(M32)
    x ^= x >> np.uint64(16)
    x = (x * np.uint64(0x85EBCA6B)) & np.uint64(M32)
    x ^= x >> np.uint64(13)
    x = (x * np.uint64(0xC2B2AE35)) & np.uint64(M32)
    x ^= x >> np.uint64(16)
    return np.where((x & np.uint64(1)) == 1, 1.0, -1.0)


def spectral_radius_estimate(A: sp.csr_matrix, steps: int = POWER_STEPS) -> float:
    """Estimate of rho(D^{-1} A) (D = diag A): the power iteration on the
    similar matrix S = |D|^{-1/2} A |D|^{-1/2}, normalising every step,
    x_{k+1} = S x_k / ||x_k||_2; returns ||S x_{steps-1}|| / ||x_{steps-1}||.
    For symmetric A this never exceeds rho and rises with ``steps``."""
    d = np.sqrt(np.abs(A.diagonal()))
    x = power_start_vector(A.shape[0])
    nx = np.linalg.norm(x)
    ny = 0.0
    for _ in range(steps):
        y = (A @ ((x / nx) / d)) / d
        ny = np.linalg.norm(y)
        x, nx = y, ny
    return float(ny)


def smoothed_prolongator(A: sp.csr_matrix, agg: np.ndarray, nc: int, steps: int = 2):
    """P = (I - omega D^{-1} A)^steps P_t, one damped-Jacobi step at a time,
    omega = 4 / (3 rho) with rho the power-iteration estimate of rho(D^{-1} A)."""
    n = A.shape[0]
    Pt = sp.csr_matrix((np.ones(n), (np.arange(n), agg)), shape=(n, nc))
    diag = A.diagonal()
    rho = spectral_radius_estimate(A)
    omega = 4.0 / (3.0 * rho)
    Dinv = sp.diags(1.0 / diag)
    P = Pt
    for _ in range(steps):
        P = (P - omega * (Dinv @ (A @ P))).tocsr()
    P.sort_indices()
    return P, omega


class Level:
    def __init__(self, A):
        self.A = A.tocsr()
        self.A.sort_indices()
        self.n = A.shape[0]
        self.dl1 = np.asarray(abs(self.A).sum(axis=1)).ravel()
        self.P = None
        self.R = None
        self.agg = None
        self.lu = None


class Hierarchy:
    """AMG hierarchy of one diagonal block."""

    def __init__(self, A, theta=0.08, coarse_max=2048, max_levels=12,
                 nu_pre=1, nu_post=1, smoother="chebyshev", cheb_degree=4,
                 cheb_lo=0.1, p_smooth=2, strength_negative=False, stab=None,
                 cycle="V"):
        if cycle not in ("V", "Wc"):
            raise ValueError(cycle)
        self.cycle = cycle
        self.theta = theta
        self.nu_pre = nu_pre
        self.nu_post = nu_post
        if smoother not in ("l1jacobi", "chebyshev"):
            raise ValueError(smoother)
        self.smoother = smoother
        self.cheb_degree = cheb_degree
        self.cheb_lo = cheb_lo
        self.levels = [Level(A)]
        T, c_stab = (None, 0.0) if stab is None else stab
        n0 = self.levels[0].n
        f_prev = 1.0
        while True:
            lev = self.levels[-1]
            lvl = len(self.levels) - 1
            if lev.n <= coarse_max or len(self.levels) >= max_levels:
                break
            th = theta
            G = strength_graph(lev.A, th, strength_negative)
            for _ in range(6):
                if 4 * int(np.sum(np.diff(G.indptr) == 0)) <= lev.n:
                    break
                th *= 0.5
                G = strength_graph(lev.A, th, strength_negative)
            agg, _ = aggregate(G, lvl)
            nc = int(agg.max()) + 1
            if 10 * nc > 9 * lev.n:
                break
            P, _ = smoothed_prolongator(lev.A, agg, nc, p_smooth)
            lev.P = P
            lev.R = P.T.tocsr()
            lev.agg = agg
            Ac = (lev.R @ lev.A @ P).tocsr()
            if T is not None:
                T = (lev.R @ T @ P).tocsr()
                f = float(np.sqrt(n0 / nc))
                Ac = (Ac + (c_stab * (f - f_prev)) * T).tocsr()
                f_prev = f
            self.levels.append(Level(Ac))
        last = self.levels[-1]
        self.coarse_max = coarse_max
        if last.n <= coarse_max:
            last.lu = sla.lu_factor(last.A.toarray())

    def sizes(self):
        return [lev.n for lev in self.levels]

    def smooth(self, lev, b, x):
        """One smoothing sweep on level ``lev``."""
        if self.smoother == "l1jacobi":
            return x + (b - lev.A @ x) / lev.dl1
        lo = self.cheb_lo
        theta = 0.5 * (1.0 + lo)
        delta = 0.5 * (1.0 - lo)
        sigma = theta / delta
        rho = 1.0 / sigma
        d = ((b - lev.A @ x) / lev.dl1) / theta
        x = x + d
        for _ in range(1, self.cheb_degree):
            rho_new = 1.0 / (2.0 * sigma - rho)
            d = rho_new * rho * d + (2.0 * rho_new / delta) * ((b - lev.A @ x) / lev.dl1)
            x = x + d
            rho = rho_new
        return x

    def vcycle(self, b, l=0):
        lev = self.levels[l]
        if lev.lu is not None:
            return sla.lu_solve(lev.lu, b)
        if l == len(self.levels) - 1:          # stalled coarsest level: smoothing only
            x = np.zeros_like(b)
            for _ in range(4):
                x = self.smooth(lev, b, x)
            return x
        x = np.zeros_like(b)
        for _ in range(self.nu_pre):
            x = self.smooth(lev, b, x)
        corrections = 1
        if self.cycle == "Wc" and l >= 1 and l + 2 < len(self.levels):
            corrections = 2
        for _ in range(corrections):
            r = b - lev.A @ x
            e = self.vcycle(lev.R @ r, l + 1)
            x = x + lev.P @ e
        for _ in range(self.nu_post):
            x = self.smooth(lev, b, x)
        return x
