"""Butcher tables, the LDU factorisation and the preconditioner coefficient
matrices (oracle; test infrastructure only).

* Radau IIA (Section 2, Table 1: order 2s-1, L-stable): collocation method
  whose nodes c_i are the zeros of P_s(2x-1) - P_{s-1}(2x-1) (P_k Legendre;
  c_s = 1), with a_ij = int_0^{c_i} l_j and b_j = int_0^1 l_j (l_j the
  Lagrange basis on the nodes).
* Lobatto IIIC (Table 1: order 2s-2, L-stable): Lobatto nodes (zeros of
  x(1-x) P'_{s-1}(2x-1)), b_j = int_0^1 l_j, first column a_i1 = b_1 for
  every i, and the other s-1 columns fixed by the simplifying conditions
  C(s-1): sum_j a_ij c_j^{q-1} = c_i^q / q, q = 1..s-1.
* LDU without pivoting (Section 4.1): A = L D U, L unit lower, U unit upper.
* A~ of Eq. PrecForm: J = diag(A), GSL = tril(A), DU, LD (Eq. PLDandPDU),
  and the optimised GSL of Eq. GSLopt (min kappa_2(A~^{-1} A) over lower
  triangular A~ with diag(A~) = diag(A)), recomputed by Nelder-Mead from
  tril(A) since the optimised coefficients are not printed in the paper.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as L


def _refine_roots(coef, x, iters=4):
    """Newton steps on the Legendre series ``coef`` (variable t in [-1,1])."""
    d = L.legder(coef)
    for _ in range(iters):
        x = x - L.legval(x, coef) / L.legval(x, d)
    return x


def _lagrange_integrals(c, upper):
    """I[i, j] = int_0^{upper[i]} l_j(tau) dtau, by an s-point Gauss rule on
    [0, upper[i]] (exact: l_j has degree s-1)."""
    s = c.size
    t, w = L.leggauss(s)
    I = np.zeros((upper.size, s))
    for i, ub in enumerate(upper):
        tau = 0.5 * ub * (t + 1.0)
        wt = 0.5 * ub * w
        for j in range(s):
            lj = np.ones_like(tau)
            for m in range(s):
                if m != j:
                    lj *= (tau - c[m]) / (c[j] - c[m])
            I[i, j] = np.dot(wt, lj)
    return I


def radau_iia(s: int):
    """(A, b, c) of the s-stage Radau IIA method."""
    if s < 1:
        raise ValueError("s >= 1")
    coef = np.zeros(s + 1)
    coef[s] = 1.0
    coef[s - 1] = -1.0
    t = np.sort(np.real(L.legroots(coef)))
    t = _refine_roots(coef, t)
    c = 0.5 * (t + 1.0)
    c[-1] = 1.0
    A = _lagrange_integrals(c, c)
    b = _lagrange_integrals(c, np.array([1.0]))[0]
    return A, b, c


def lobatto_iiic(s: int):
    """(A, b, c) of the s-stage Lobatto IIIC method (s >= 2)."""
    if s < 2:
        raise ValueError("s >= 2")
    # interior nodes: zeros of P'_{s-1}(t)
    coef = np.zeros(s)
    coef[s - 1] = 1.0
    dcoef = L.legder(coef)
    if s > 2:
        ti = np.sort(np.real(L.legroots(dcoef)))
        ti = _refine_roots(dcoef, ti)
    else:
        ti = np.zeros(0)
    t = np.concatenate([[-1.0], ti, [1.0]])
    c = 0.5 * (t + 1.0)
    b = _lagrange_integrals(c, np.array([1.0]))[0]
    A = np.zeros((s, s))
    A[:, 0] = b[0]
    # C(s-1) for columns 2..s: sum_{j>=2} a_ij c_j^{q-1} = c_i^q/q - b_1 c_1^{q-1}
    V = np.array([[c[j] ** (q - 1) for j in range(1, s)] for q in range(1, s)])
    for i in range(s):
        rhs = np.array([c[i] ** q / q - b[0] * c[0] ** (q - 1) for q in range(1, s)])
        A[i, 1:] = np.linalg.solve(V, rhs)
    return A, b, c


def ldu(A):
    """Doolittle-style A = L D U without pivoting.  Raises ZeroDivisionError
    on a vanishing leading principal minor."""
    A = np.asarray(A, dtype=np.float64)
    s = A.shape[0]
    Lm = np.eye(s)
    Um = np.eye(s)
    d = np.zeros(s)
    for k in range(s):
        d[k] = A[k, k] - sum(Lm[k, m] * d[m] * Um[m, k] for m in range(k))
        if d[k] == 0.0:
            raise ZeroDivisionError(f"zero pivot at {k}")
        for i in range(k + 1, s):
            Lm[i, k] = (A[i, k] - sum(Lm[i, m] * d[m] * Um[m, k] for m in range(k))) / d[k]
        for j in range(k + 1, s):
            Um[k, j] = (A[k, j] - sum(Lm[k, m] * d[m] * Um[m, j] for m in range(k))) / d[k]
    return Lm, np.diag(d), Um


def kappa2(X):
    sv = np.linalg.svd(X, compute_uv=False)
    return sv[0] / sv[-1]


def gsl_optimized(A, iters=20000):
    """Eq. GSLopt: lower-triangular A~ with diag(A~) = diag(A) minimising
    kappa_2(A~^{-1} A); Nelder-Mead started from tril(A)."""
    from scipy.optimize import minimize
    s = A.shape[0]
    idx = np.tril_indices(s, -1)
    if idx[0].size == 0:
        return np.tril(A)

    def build(p):
        At = np.diag(np.diag(A)).astype(np.float64)
        At[idx] = p
        return At

    def obj(p):
        return kappa2(np.linalg.solve(build(p), A))

    p0 = np.tril(A)[idx]
    best = minimize(obj, p0, method="Nelder-Mead",
                    options={"maxiter": iters, "maxfev": iters, "xatol": 1e-10,
                             "fatol": 1e-12, "adaptive": True})
    return build(best.x)


def atilde(A, kind: str, gsl_opt=None):
    """Preconditioner coefficient matrix of Eq. PrecForm."""
    kind = kind.upper()
    if kind == "J":
        return np.diag(np.diag(A))
    if kind == "GSL":
        return np.tril(A)
    if kind == "GSL_OPT":
        return gsl_opt if gsl_opt is not None else gsl_optimized(A)
    Lm, D, Um = ldu(A)
    if kind == "DU":
        return D @ Um
    if kind == "LD":
        return Lm @ D
    if kind == "FULL":          # A~ = A: the preconditioner is the operator
        return np.array(A, dtype=np.float64)
    raise ValueError(kind)


def sweep_direction(kind: str) -> str:
    """'diag', 'forward' (lower triangular A~) or 'backward' (upper)."""
    kind = kind.upper()
    if kind == "J":
        return "diag"
    if kind in ("GSL", "GSL_OPT", "LD"):
        return "forward"
    if kind == "DU":
        return "backward"
    raise ValueError(kind)


def stability_function(A, b, z):
    """R(z) = 1 + z b^T (I - z A)^{-1} 1."""
    s = A.shape[0]
    return 1.0 + z * b @ np.linalg.solve(np.eye(s) - z * A, np.ones(s))
