"""The IRK stage system, its block preconditioners, flexible GMRES, the time
step and the discrete adjoint (oracle; test infrastructure only).

Stage vectors are (s, n) arrays: row i is the stage block K_i of the paper's
block vector [K_1; ...; K_s] (Eq. block_coeff_mtx).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import butcher as bt
from .amg import Hierarchy


# ----------------------------------------------------------------------------
# Section 4: the Kronecker operator  A = I_s (x) M + h A (x) F
# ----------------------------------------------------------------------------

def apply_operator(M, F, A, h, z):
    """w_i = M z_i + h sum_j a_ij F z_j, i.e. (I (x) M + h A (x) F) z."""
    Mz = np.stack([M @ z[j] for j in range(z.shape[0])])
    Fz = np.stack([F @ z[j] for j in range(z.shape[0])])
    return Mz + h * (A @ Fz)


def kron_matrix(M, F, A, h):
    """The assembled sN x sN sparse matrix I_s (x) M + h A (x) F."""
    s = A.shape[0]
    return (sp.kron(sp.identity(s), M) + h * sp.kron(sp.csr_matrix(A), F)).tocsc()


def solve_stages_eig(M, F, A, h, rhs):
    """Exact solve of (I_s (x) M + h A (x) F) k = rhs for a diagonalisable
    Butcher matrix (the Radau IIA tables have distinct eigenvalues), by the
    eigendecomposition A = S diag(lam) S^-1: multiplying by S^-1 (x) I
    decouples the stages into the s sparse systems
        (M + h lam_j F) y_j = sum_i (S^-1)_ji rhs_i,   k = (S (x) I) y.
    A real A has eigenvalues in conjugate pairs whose solutions are conjugate,
    so each pair takes one complex sparse LU.  For sizes where the assembled
    sN x sN system is too large for a direct solve."""
    s = A.shape[0]
    lam, S = np.linalg.eig(A)
    R = np.linalg.solve(S, rhs.astype(complex))
    Y = np.zeros((s, rhs.shape[1]), dtype=complex)
    done = [False] * s
    for j in range(s):
        if done[j]:
            continue
        Bj = (M + (h * lam[j]) * F).tocsc()
        Y[j] = spla.splu(Bj).solve(R[j])
        done[j] = True
        if abs(lam[j].imag) > 0.0:
            for q in range(s):
                if not done[q] and abs(lam[q] - np.conj(lam[j])) <= 1e-12 * abs(lam[j]):
                    Y[q] = np.conj(Y[j])     # real A, real rhs: R_q = conj(R_j)
                    done[q] = True
                    break
    return np.real(S @ Y)


def stage_rhs(F, g, u, s):
    """Right-hand side -(1_s (x) (F u_n + g)) of Eq. block_coeff_mtx
    (g = F_IB u_B is the Dirichlet lift, zero for the heat problem)."""
    r = -(F @ u + g)
    return np.tile(r, (s, 1))


# ----------------------------------------------------------------------------
# Section 4.2: applying P = I_s (x) M + h A~ (x) F
# ----------------------------------------------------------------------------

class BlockPreconditioner:
    """z = P^{-1} v by the substitutions of Section 4.2.

    kind J: s independent subsolves (M + h A~_jj F) w_j = v_j.
    kind GSL / GSL_OPT / LD (A~ lower): forward substitution,
        (M + h A~_jj F) w_j = v_j - sum_{k<j} h A~_jk F w_k.
    kind DU (A~ upper): backward substitution,
        (M + h A~_jj F) w_j = v_j - sum_{k>j} h A~_jk F w_k.
    Each subsolve is exact (sparse LU, ``subsolve='direct'``) or one AMG
    V-cycle on the block (``subsolve='amg'``); ``stab`` (a SUPG problem's
    streamline matrix T) stabilises the coarse AMG levels of the block
    M + h A~_jj F with c = h A~_jj.
    ``transpose=True`` applies P^T = I (x) M^T + h A~^T (x) F^T, whose
    substitution runs in the opposite direction with the transposed blocks.
    """

    def __init__(self, M, F, A, h, kind="LD", subsolve="amg", Atilde=None,
                 amg_opts=None, transpose=False, stab=None):
        self.kind = kind.upper()
        self.At = np.array(Atilde if Atilde is not None else bt.atilde(A, self.kind))
        direction = bt.sweep_direction(self.kind)
        if transpose:
            self.At = self.At.T.copy()
            direction = {"diag": "diag", "forward": "backward",
                         "backward": "forward"}[direction]
        self.direction = direction
        if transpose:
            M, F = M.T.tocsr(), F.T.tocsr()
        self.M, self.F, self.h = M, F, h
        self.s = self.At.shape[0]
        self.subsolve = subsolve
        amg_opts = amg_opts or {}
        self.blocks = []
        self.solvers = []
        for j in range(self.s):
            Bj = (M + (h * self.At[j, j]) * F).tocsr()
            self.blocks.append(Bj)
            if subsolve == "direct":
                self.solvers.append(spla.splu(Bj.tocsc()))
            elif subsolve == "amg":
                st = None if stab is None else (stab, h * self.At[j, j])
                self.solvers.append(Hierarchy(Bj, stab=st, **amg_opts))
            else:
                raise ValueError(subsolve)

    def _solve(self, j, rhs):
        S = self.solvers[j]
        if self.subsolve == "direct":
            return S.solve(rhs)
        return S.vcycle(rhs)

    def apply(self, v):
        s, h, F, At = self.s, self.h, self.F, self.At
        w = np.zeros_like(v)
        if self.direction == "diag":
            order = range(s)
        elif self.direction == "forward":
            order = range(s)
        else:
            order = range(s - 1, -1, -1)
        done = []
        for j in order:
            rhs = v[j].copy()
            if self.direction != "diag":
                for k in done:
                    if At[j, k] != 0.0:
                        rhs -= h * At[j, k] * (F @ w[k])
            w[j] = self._solve(j, rhs)
            done.append(j)
        return w


# ----------------------------------------------------------------------------
# Right-preconditioned restarted flexible GMRES (modified Gram-Schmidt)
# ----------------------------------------------------------------------------

class GmresResult:
    def __init__(self, x, iterations, restarts, resid, converged, history):
        self.x = x
        self.iterations = iterations
        self.restarts = restarts
        self.resid = resid
        self.converged = converged
        self.history = history


def fgmres(apply_A, apply_Pinv, b, m=30, rtol=1e-10, max_it=1000, record=None):
    """Solve A x = b from x0 = 0; stop when ||b - A x||_2 <= rtol ||b||_2.
    ``record`` (a dict, tests only) receives the first cycle's V, Z, the
    Hessenberg matrix before the Givens rotations, its width k and the final
    residual estimate |g_k|.

    Each cycle: v_0 = r / ||r||; for j: z_j = P^{-1} v_j (stored, flexible),
    w = A z_j, MGS against v_0..v_j, Givens rotations on the Hessenberg
    column, residual estimate |g_{j+1}|.  The cycle ends at j = m or when the
    estimate meets the tolerance; x += Z y and the true residual decides.
    Returns the total number of inner iterations."""
    shape = b.shape
    bv = b.ravel()
    bnorm = np.linalg.norm(bv)
    x = np.zeros_like(bv)
    if bnorm == 0.0:
        return GmresResult(x.reshape(shape), 0, 0, 0.0, True, [])
    r = bv.copy()
    it = 0
    restarts = 0
    history = []
    while True:
        beta = np.linalg.norm(r)
        history.append(beta / bnorm)
        if beta <= rtol * bnorm:
            return GmresResult(x.reshape(shape), it, restarts, beta / bnorm, True, history)
        if it >= max_it:
            return GmresResult(x.reshape(shape), it, restarts, beta / bnorm, False, history)
        V = np.zeros((m + 1, bv.size))
        Z = np.zeros((m, bv.size))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            Z[j] = apply_Pinv(V[j].reshape(shape)).ravel()
            w = apply_A(Z[j].reshape(shape)).ravel()
            for i in range(j + 1):
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            if record is not None and restarts == 0:
                record.setdefault("H", np.zeros((m + 1, m)))[:j + 2, j] = H[:j + 2, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k = j + 1
            if abs(g[j + 1]) <= rtol * bnorm or it >= max_it:
                break
        if record is not None and restarts == 0:
            record.update(V=V[:k + 1].copy(), Z=Z[:k].copy(), k=k, estimate=abs(g[k]))
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + Z[:k].T @ y
        r = bv - apply_A(x.reshape(shape)).ravel()
        restarts += 1


def gmres_left(apply_A, apply_Pinv, b, m=30, rtol=1e-10, max_it=1000):
    """Left-preconditioned restarted GMRES on P^{-1} A x = P^{-1} b from x0 = 0
    (the left-preconditioned runs of Section 5): stop when the preconditioned
    residual ||P^{-1}(b - A x)||_2 <= rtol ||P^{-1} b||_2.

    Each cycle: r = P^{-1}(b - A x) formed explicitly, v_0 = r / ||r||; for j:
    w = P^{-1} A v_j, MGS against v_0..v_j, Givens rotations, estimate
    |g_{j+1}|; the cycle ends at j = m or when the estimate meets the
    tolerance; x += V y.  `history` holds the explicit preconditioned
    residual at every cycle start."""
    shape = b.shape
    bv = b.ravel()
    r = apply_Pinv(b).ravel()
    bnorm = np.linalg.norm(r)
    x = np.zeros_like(bv)
    if bnorm == 0.0:
        return GmresResult(x.reshape(shape), 0, 0, 0.0, True, [])
    it = 0
    restarts = 0
    history = []
    while True:
        beta = np.linalg.norm(r)
        history.append(beta / bnorm)
        if beta <= rtol * bnorm:
            return GmresResult(x.reshape(shape), it, restarts, beta / bnorm, True, history)
        if it >= max_it:
            return GmresResult(x.reshape(shape), it, restarts, beta / bnorm, False, history)
        V = np.zeros((m + 1, bv.size))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            w = apply_Pinv(apply_A(V[j].reshape(shape))).ravel()
            for i in range(j + 1):
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k = j + 1
            if abs(g[j + 1]) <= rtol * bnorm or it >= max_it:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + V[:k].T @ y
        r = apply_Pinv((bv - apply_A(x.reshape(shape)).ravel()).reshape(shape)).ravel()
        restarts += 1


# ----------------------------------------------------------------------------
# Section 2: one IRK step  u_{n+1} = u_n + h sum_i b_i K_i
# ----------------------------------------------------------------------------

class StepResult:
    def __init__(self, u, k, iterations, resid):
        self.u = u
        self.k = k
        self.iterations = iterations
        self.resid = resid


class IRKSolver:
    """One problem (M, F, g), one Butcher table, one time step h."""

    def __init__(self, prob, A, b, h, kind="LD", subsolve="amg", m=30,
                 rtol=1e-10, amg_opts=None, Atilde=None, side="right"):
        self.M, self.F, self.g = prob.M, prob.F, prob.g
        self.A = np.asarray(A, dtype=np.float64)
        self.b = np.asarray(b, dtype=np.float64)
        self.h = float(h)
        self.s = self.A.shape[0]
        self.m, self.rtol = m, rtol
        self.kind = kind
        if side not in ("right", "left"):
            raise ValueError("side must be 'right' or 'left'")
        self.side = side
        self.subsolve = subsolve
        self.amg_opts = amg_opts
        self.pc = None
        if kind is not None:
            self.pc = BlockPreconditioner(self.M, self.F, self.A, self.h, kind,
                                          subsolve, Atilde=Atilde, amg_opts=amg_opts,
                                          stab=getattr(prob, "T", None))
        self._pcT = None

    def op(self, z):
        return apply_operator(self.M, self.F, self.A, self.h, z)

    def opT(self, z):
        """The transposed stage operator I (x) M^T + h A^T (x) F^T."""
        return apply_operator(self.M.T.tocsr(), self.F.T.tocsr(), self.A.T, self.h, z)

    def solve_stages(self, rhs):
        solver = gmres_left if self.side == "left" else fgmres
        return solver(self.op, self.pc.apply, rhs, m=self.m, rtol=self.rtol)

    def solve_stages_direct(self, rhs):
        K = kron_matrix(self.M, self.F, self.A, self.h)
        return spla.spsolve(K, rhs.ravel()).reshape(rhs.shape)

    def step(self, u, direct=False):
        rhs = stage_rhs(self.F, self.g, u, self.s)
        if direct:
            k = self.solve_stages_direct(rhs)
            its, resid = 0, 0.0
        else:
            res = self.solve_stages(rhs)
            k, its, resid = res.x, res.iterations, res.resid
        unew = u + self.h * (self.b @ k)
        return StepResult(unew, k, its, resid)

    def run(self, u0, nsteps, direct=False):
        u = np.array(u0, dtype=np.float64)
        out = [u]
        its = []
        for _ in range(nsteps):
            r = self.step(u, direct=direct)
            u = r.u
            out.append(u)
            its.append(r.iterations)
        return out, its

    # ------------------------------------------------------------------
    # Discrete adjoint of the time loop (FP64, direct or preconditioned)
    # ------------------------------------------------------------------
    def adjoint_step(self, lam_next, direct=True):
        """mu solves A^T mu = h (b (x) lam_{n+1}); lam_n = lam_{n+1} -
        F^T sum_i mu_i.  Returns (lam_n, mu)."""
        s = self.s
        rhs = self.h * np.outer(self.b, lam_next)
        if direct:
            KT = kron_matrix(self.M, self.F, self.A, self.h).T.tocsc()
            mu = spla.spsolve(KT, rhs.ravel()).reshape(s, -1)
        else:
            if self._pcT is None:
                self._pcT = BlockPreconditioner(self.M, self.F, self.A, self.h,
                                                self.kind, self.subsolve,
                                                amg_opts=self.amg_opts,
                                                transpose=True)
            mu = fgmres(self.opT, self._pcT.apply, rhs, m=self.m, rtol=self.rtol).x
        lam = lam_next - self.F.T @ mu.sum(axis=0)
        return lam, mu


def misfit(M, u, d):
    """L = 1/2 (u - d)^T M (u - d)."""
    e = u - d
    return 0.5 * e @ (M @ e)


def adjoint_gradients(solver, Ke_int, elem_dofs, u0, nsteps, d, direct=True):
    """Gradient of L(u_N) w.r.t. u_0 and the per-element kappa, for the heat
    problem with F = sum_e kappa_e K_e.

    dL/dkappa_e = - sum_n sum_i mu_{n,i}[e]^T K_e U_{n,i}[e], where
    U_{n,i} = u_n + h sum_j a_ij k_{n,j} is the stage value and [e] gathers
    the element's three vertices (Dirichlet vertices contribute zero).
    Ke_int: (nt, 3, 3) element stiffness for kappa = 1; elem_dofs (nt, 3)
    interior index per vertex or -1."""
    us, _ = solver.run(u0, nsteps, direct=direct)
    ks = []
    u = us[0]
    for n in range(nsteps):
        rhs = stage_rhs(solver.F, solver.g, us[n], solver.s)
        if direct:
            ks.append(solver.solve_stages_direct(rhs))
        else:
            ks.append(solver.solve_stages(rhs).x)
    lam = solver.M @ (us[-1] - d)
    nt = Ke_int.shape[0]
    gk = np.zeros(nt)
    mask = elem_dofs >= 0
    idx = np.where(mask, elem_dofs, 0)
    for n in range(nsteps - 1, -1, -1):
        lam_prev, mu = solver.adjoint_step(lam, direct=direct)
        U = us[n][None, :] + solver.h * (solver.A @ ks[n])     # (s, n)
        for i in range(solver.s):
            mu_e = np.where(mask, mu[i][idx], 0.0)              # (nt, 3)
            U_e = np.where(mask, U[i][idx], 0.0)
            gk -= np.einsum("ea,eab,eb->e", mu_e, Ke_int, U_e)
        lam = lam_prev
    return lam, gk, misfit(solver.M, us[-1], d)
