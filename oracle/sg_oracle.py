"""Plain FP64 CPU oracle of the SG-GMRES method of arXiv 1910.11505 (test infrastructure only).

Problem (Sec. 2, Eq. Strong_PS): -div(a grad u) = f on D = [0,1]^2, u = 0 on the boundary, with
a lognormal coefficient a = a_min + exp(gamma) (Eqs. 3-6).  gamma is truncated to M Karhunen-Loeve
(KL) terms (Eq. aKL) of the separable exponential covariance (Eq. standard_deviation); a is
projected on normalised Hermite chaos of total degree q (Eq. dataProjection); the solution uses
total degree p (Eq. u_discrete).  The stochastic Galerkin matrix is K = sum_q G_q (x) A_q
(Eqs. A_q, stochastic_matrix).  Preconditioners: mean-based block diagonal (Sec. 1, cited) and the
field-split block lower triangular P of Eq. P_preconditioner (block Gauss-Seidel) plus its block
diagonal (block Jacobi) variant, the diagonal blocks approximated by ILU(0); both wrapped in the
Richardson level solver of Eq. level_solver.  The outer solver is restarted GMRES (Sec. 3).

Readings where the paper is silent (numbered as in the design notes):
  R1  element quadrature: 3x3 Gauss-Legendre per Q1 cell.
  R2  KL order: eigenvalues descending, ties broken by the lexicographic (i, j) of the 1-D modes,
      signs as in the closed forms below.
  R3  multi-index order: lexicographic, last index fastest.
  R4  Dirichlet nodes kept: rows and columns zeroed in every A_q, A_0[b, b] = 1, F[b, :] = 0.
  R5  ILU(0), natural node order, no pivoting.
  R6  ``inner_iters`` Richardson steps per diagonal block, ``outer_sweeps`` steps of Eq. level_solver.
  R7  right-preconditioned GMRES(restart), classical Gram-Schmidt applied twice (CGS2), Givens
      rotations, stop on the true relative residual ||F - K x|| / ||F||.
  R8  mean-based preconditioner = I (x) ILU0(A_0), A_0 the stiffness of E[a].
  R18 ILU(0) ordering (the paper names none): natural order by default; a four-colour ordering
      (colour (x mod 2) + 2 (y mod 2)) is the alternative, whose triangular solves run one colour
      at a time with every node of a colour independent.
  R20 ILU(0) of a block of K with several fields (the whole K of G-I / G-M-I, a split of
      G-M-Fg-I): unknowns node-major (a node's fields together), nodes in the four-colour order,
      the pattern every field of a node coupled to every field of its 9-point neighbours.  With
      q = 2p that is K's own pattern; scalar ILU(0) on it equals block ILU(0) with exact dense
      LU of the diagonal blocks.
  R21 G-M-Fg-I splits (Sec. 3, Eq. P_group): fields grouped by the first index of their
      multi-index; in order, a group that holds a multi-index with all indices equal opens a
      new split, any other group joins the preceding split.

Layout conventions: a nodal field over the chaos basis is an N x P float64 array X with
X[j, b] = u_b(node j); node id = i + m*j for grid point (i/n, j/n), m = n + 1.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.optimize
import scipy.sparse
import scipy.sparse.linalg

__all__ = [
    "kl_modes_1d", "kl_eval_1d", "KLModes", "kl_modes_2d", "kl_fields",
    "multi_indices", "hermite_triple_1d", "triple_products",
    "chaos_coefficients", "gauss_legendre_3", "q1_local_stiffness_stack",
    "SGProblem", "build_problem", "stack_rows_dense", "sg_matvec", "sg_matvec_rows",
    "ilu0", "ilu0_solve", "mean_precond", "fs_blocks", "fs_precond", "gmres", "boundary_mask",
    "prolongation", "mg_levels", "mg_setup", "mg_vcycle", "color4_order",
    "fg_splits", "block_pattern_matrix", "bilu0", "bilu0_solve", "fg_blocks", "fg_precond",
]


# ----------------------------------------------------------------------------------------------
# Karhunen-Loeve expansion of the separable exponential covariance (Sec. 2.1, Eqs. gen_eigen,
# standard_deviation).  In one dimension, on t = x - 1/2 in [-1/2, 1/2] with c = 1/ell, the
# integral operator with kernel exp(-c|s - t|) has eigenpairs
#   even:  c cos(w/2) - w sin(w/2) = 0,  f(t) = cos(w t) / sqrt(1/2 + sin(w)/(2w))
#   odd :  w cos(w/2) + c sin(w/2) = 0,  f(t) = sin(w t) / sqrt(1/2 - sin(w)/(2w))
#   eigenvalue mu = 2c / (w^2 + c^2).
# The 2-D covariance sigma^2 exp(-(|x1-y1| + |x2-y2|)/ell) is the product of two 1-D kernels,
# so its eigenpairs are lambda = sigma^2 mu_i mu_j, b = f_i(x1) f_j(x2).
# ----------------------------------------------------------------------------------------------

_HALF = 0.5


def kl_modes_1d(ell: float, count: int):
    """First ``count`` 1-D KL modes (omega, parity, mu, norm) in decreasing mu (= increasing omega).

    The even root of branch k lies in (2k pi, (2k+1) pi), the odd root in ((2k+1) pi, (2k+2) pi)
    (for the half-width 1/2 used here), so the modes alternate even, odd, even, ...
    """
    c = 1.0 / ell
    modes = []
    k = 0
    while len(modes) < count:
        if len(modes) % 2 == 0:  # even branch k
            lo, hi = 2 * k * math.pi, (2 * k + 1) * math.pi
            fn = lambda w: c * math.cos(w * _HALF) - w * math.sin(w * _HALF)  # noqa: E731
            parity = 0
        else:  # odd branch k
            lo, hi = (2 * k + 1) * math.pi, (2 * k + 2) * math.pi
            fn = lambda w: w * math.cos(w * _HALF) + c * math.sin(w * _HALF)  # noqa: E731
            parity = 1
        # the smooth forms above have exactly one sign change inside each open bracket
        eps = 1e-14 * hi
        w = scipy.optimize.brentq(fn, lo + eps, hi - eps, xtol=1e-300, rtol=4 * np.finfo(float).eps,
                                  maxiter=500)
        if parity == 0:
            norm = math.sqrt(_HALF + math.sin(w) / (2.0 * w))
        else:
            norm = math.sqrt(_HALF - math.sin(w) / (2.0 * w))
            k += 1
        modes.append((w, parity, 2.0 * c / (w * w + c * c), norm))
    return modes


def kl_eval_1d(mode, x):
    """Normalised 1-D eigenfunction f(t), t = x - 1/2, of a mode returned by kl_modes_1d."""
    w, parity, _mu, norm = mode
    t = np.asarray(x, dtype=np.float64) - _HALF
    return (np.cos(w * t) if parity == 0 else np.sin(w * t)) / norm


@dataclass
class KLModes:
    """Top-M 2-D KL modes: eigenvalue lam[n] = sigma^2 mu_i mu_j and 1-D factor indices (i, j)."""
    sigma: float
    ell: float
    modes1d: list
    lam: np.ndarray
    ij: list


def kl_modes_2d(sigma: float, ell: float, M: int) -> KLModes:
    """Largest M eigenpairs of the 2-D covariance (Eq. standard_deviation), ordered by reading R2:
    eigenvalue descending, ties by lexicographic (i, j), i the x1 factor."""
    m1 = kl_modes_1d(ell, M + 1)
    cand = []
    for i in range(len(m1)):
        for j in range(len(m1)):
            cand.append((-(m1[i][2] * m1[j][2]), i, j))
    cand.sort()
    top = cand[:M]
    lam = np.array([sigma * sigma * (-v) for v, _, _ in top])
    return KLModes(sigma, ell, m1, lam, [(i, j) for _, i, j in top])


def kl_fields(kl: KLModes, x1, x2):
    """g_n(x) = sqrt(lambda_n) b_n(x) for n = 1..M (Eq. aKL); returns an (M, len(x)) array."""
    x1 = np.asarray(x1, dtype=np.float64)
    x2 = np.asarray(x2, dtype=np.float64)
    out = np.empty((len(kl.lam),) + x1.shape)
    for n, (i, j) in enumerate(kl.ij):
        out[n] = math.sqrt(kl.lam[n]) * kl_eval_1d(kl.modes1d[i], x1) * kl_eval_1d(kl.modes1d[j], x2)
    return out


# ----------------------------------------------------------------------------------------------
# Hermite chaos (Sec. 2.2): index sets J(p) = {p in N^M : sum p_n <= p}, normalised probabilists'
# Hermite polynomials psi_p(y) = prod He_{p_n}(y_n) / sqrt(p_n!), orthonormal under N(0, I).
# ----------------------------------------------------------------------------------------------

def multi_indices(M: int, p: int) -> np.ndarray:
    """J(p) of total degree <= p in M variables, lexicographic with the last index fastest (R3).

    Its size is (M + p)! / (M! p!) (Sec. 2.2)."""
    out = []

    def rec(prefix, left, depth):
        if depth == M:
            out.append(tuple(prefix))
            return
        for d in range(left + 1):
            rec(prefix + [d], left - d, depth + 1)

    rec([], p, 0)
    return np.array(out, dtype=np.int64).reshape(len(out), M)


def hermite_triple_1d(i: int, j: int, k: int) -> float:
    """E[psi_i psi_j psi_k] for normalised 1-D Hermite polynomials under N(0, 1).

    With s = (i + j + k) / 2: zero unless s is an integer with s >= max(i, j, k); otherwise
    sqrt(i! j! k!) / ((s-i)! (s-j)! (s-k)!)."""
    t = i + j + k
    if t % 2:
        return 0.0
    s = t // 2
    if s < i or s < j or s < k:
        return 0.0
    num = math.factorial(i) * math.factorial(j) * math.factorial(k)
    den = math.factorial(s - i) * math.factorial(s - j) * math.factorial(s - k)
    return math.sqrt(num) / den


def triple_products(Jq: np.ndarray, Jp: np.ndarray) -> np.ndarray:
    """Dense G[k, a, b] = E[psi_{q_k} psi_{p_a} psi_{p_b}] (Sec. 2.2, definition of G_q).

    The M-variate expectation factorises over the independent y_n."""
    L, P = len(Jq), len(Jp)
    G = np.zeros((L, P, P))
    for k in range(L):
        for a in range(P):
            for b in range(P):
                v = 1.0
                for n in range(Jq.shape[1]):
                    v *= hermite_triple_1d(int(Jq[k, n]), int(Jp[a, n]), int(Jp[b, n]))
                    if v == 0.0:
                        break
                G[k, a, b] = v
    return G


def chaos_coefficients(g: np.ndarray, Jq: np.ndarray, a_min: float, mu: float) -> np.ndarray:
    """a_q(x) = E[a_KL(x, y) psi_q(y)] (Eq. dataProjection) for a_KL of Eq. KL_gamma.

    With y ~ N(0, I): E[exp(g.y) psi_q(y)] = exp(|g|^2 / 2) prod_n g_n^{q_n} / sqrt(q_n!), so
    a_q = a_min delta_{q,0} + exp(mu + |g|^2 / 2) prod_n g_n^{q_n} / sqrt(q_n!).
    ``g`` is (M, npts); returns (L, npts)."""
    base = np.exp(mu + 0.5 * np.sum(g * g, axis=0))
    out = np.empty((len(Jq),) + g.shape[1:])
    for k, q in enumerate(Jq):
        v = base.copy()
        for n, qn in enumerate(q):
            v = v * g[n] ** int(qn) / math.sqrt(math.factorial(int(qn)))
        out[k] = v
    if np.all(Jq[0] == 0):
        out[0] += a_min
    return out


# ----------------------------------------------------------------------------------------------
# Q1 finite elements on the uniform n x n mesh of [0,1]^2 (the configs use bilinear elements;
# the entries [A_q]_{jj'} = int a_q grad phi_j . grad phi_j' of Eq. A_q are computed with the
# 3x3 Gauss-Legendre rule, reading R1).
# ----------------------------------------------------------------------------------------------

def gauss_legendre_3():
    """3-point Gauss-Legendre nodes and weights on [0, 1]."""
    r = math.sqrt(3.0 / 5.0)
    return np.array([0.5 - 0.5 * r, 0.5, 0.5 + 0.5 * r]), np.array([5.0, 8.0, 5.0]) / 18.0


def _q1_ref():
    """Reference-square Gauss points (9), weights and the gradients / values of the 4 bilinear
    shape functions; local node order (0,0), (1,0), (0,1), (1,1)."""
    t, w = gauss_legendre_3()
    pts, wts, grads, vals = [], [], [], []
    for jy in range(3):
        for ix in range(3):
            xi, eta = t[ix], t[jy]
            pts.append((xi, eta))
            wts.append(w[ix] * w[jy])
            grads.append([(-(1 - eta), -(1 - xi)), ((1 - eta), -xi), (-eta, (1 - xi)), (eta, xi)])
            vals.append([(1 - xi) * (1 - eta), xi * (1 - eta), (1 - xi) * eta, xi * eta])
    return np.array(pts), np.array(wts), np.array(grads), np.array(vals)


def q1_local_stiffness_stack(n: int, elems: np.ndarray, kl: KLModes, Jq, a_min, mu):
    """Element matrices sum_gp w a_q(x_gp) gradphi_a . gradphi_b for each listed cell
    (index ex + n*ey) and every chaos index q: an (ncell, L, 4, 4) array.  On a square cell of
    side h the Jacobian factors h^2 and 1/h^2 cancel."""
    pts, wts, grads, _ = _q1_ref()
    h = 1.0 / n
    ex = elems % n
    ey = elems // n
    x1 = (ex[:, None] + pts[None, :, 0]) * h  # (ncell, 9)
    x2 = (ey[:, None] + pts[None, :, 1]) * h
    g = kl_fields(kl, x1.ravel(), x2.ravel())
    aq = chaos_coefficients(g, Jq, a_min, mu).reshape(len(Jq), len(elems), 9)
    gg = np.einsum("gad,gbd->gab", grads, grads)  # (9, 4, 4)
    return np.einsum("g,kcg,gab->ckab", wts, aq, gg)


def _local_nodes(n: int, elems: np.ndarray) -> np.ndarray:
    m = n + 1
    ex = elems % n
    ey = elems // n
    base = ex + m * ey
    return np.stack([base, base + 1, base + m, base + m + 1], axis=1)


@dataclass
class SGProblem:
    """Everything the oracle assembles for one SG system."""
    n: int
    M: int
    p: int
    q: int
    sigma: float
    ell: float
    a_min: float
    mu: float
    f: float
    kl: KLModes
    Jp: np.ndarray
    Jq: np.ndarray
    G: np.ndarray                      # (L, P, P)
    A: list                            # L scipy CSR matrices (N x N), Dirichlet applied
    F: np.ndarray                      # (N, P)
    boundary: np.ndarray               # bool (N,)
    extra: dict = field(default_factory=dict)

    @property
    def N(self):
        return (self.n + 1) ** 2

    @property
    def P(self):
        return len(self.Jp)

    @property
    def L(self):
        return len(self.Jq)


def boundary_mask(n: int) -> np.ndarray:
    m = n + 1
    i = np.arange(m * m) % m
    j = np.arange(m * m) // m
    return (i == 0) | (j == 0) | (i == n) | (j == n)


def build_problem(n, M, p, q=None, sigma=0.5, ell=1.0, a_min=0.0, mu=0.0, f=1.0) -> SGProblem:
    """Assemble the SG system K u = F (Eqs. linear_algebraic_2, stochastic_matrix) for the full
    mesh.  ``q`` defaults to 2p, for which K = E[A(y) psi psi^T] holds exactly."""
    if q is None or q <= 0:
        q = 2 * p
    kl = kl_modes_2d(sigma, ell, M)
    Jp = multi_indices(M, p)
    Jq = multi_indices(M, q)
    G = triple_products(Jq, Jp)
    m = n + 1
    N = m * m
    elems = np.arange(n * n)
    loc = q1_local_stiffness_stack(n, elems, kl, Jq, a_min, mu)  # (ne, L, 4, 4)
    nodes = _local_nodes(n, elems)
    rows = np.repeat(nodes[:, :, None], 4, axis=2).reshape(len(elems), 16)
    cols = np.repeat(nodes[:, None, :], 4, axis=1).reshape(len(elems), 16)
    bnd = boundary_mask(n)
    A = []
    for k in range(len(Jq)):
        Ak = scipy.sparse.coo_matrix((loc[:, k].reshape(len(elems), 16).ravel(),
                                      (rows.ravel(), cols.ravel())), shape=(N, N)).tocsr()
        Ak.sum_duplicates()
        A.append(_apply_dirichlet(Ak, bnd, k == 0))
    F = np.zeros((N, len(Jp)))
    _, wts, _, vals = _q1_ref()
    h = 1.0 / n
    load_local = f * h * h * (wts @ vals)  # int f phi_a over one cell, a = 0..3
    np.add.at(F[:, 0], nodes.ravel(), np.tile(load_local, len(elems)))
    F[bnd, :] = 0.0
    return SGProblem(n, M, p, q, sigma, ell, a_min, mu, f, kl, Jp, Jq, G, A, F, bnd)


def _apply_dirichlet(Ak, bnd, is_mean):
    """Reading R4: zero boundary rows and columns; unit diagonal on the mean block."""
    keep = scipy.sparse.diags((~bnd).astype(np.float64))
    out = (keep @ Ak @ keep).tocsr()
    if is_mean:
        out = (out + scipy.sparse.diags(bnd.astype(np.float64))).tocsr()
    out.sort_indices()
    return out


def stack_rows_dense(n, rows, kl: KLModes, Jq, a_min, mu):
    """Rows ``rows`` of every A_q without assembling the full stack (for sampled parity at sizes
    where the whole stack does not fit the host): returns cols (list per row) and values
    (len(rows), L, ncols) built from the cells around each row node, Dirichlet applied."""
    m = n + 1
    bnd = boundary_mask(n)
    out_cols, out_vals = [], []
    for r in rows:
        i, j = r % m, r // m
        cells = []
        for ey in (j - 1, j):
            for ex in (i - 1, i):
                if 0 <= ex < n and 0 <= ey < n:
                    cells.append(ex + n * ey)
        cells = np.array(cells, dtype=np.int64)
        loc = q1_local_stiffness_stack(n, cells, kl, Jq, a_min, mu)
        nodes = _local_nodes(n, cells)
        acc = {}
        for c in range(len(cells)):
            a = int(np.nonzero(nodes[c] == r)[0][0])
            for b in range(4):
                col = int(nodes[c, b])
                acc[col] = acc.get(col, 0.0) + loc[c, :, a, b]
        cols = sorted(acc)
        vals = np.stack([acc[c] for c in cols], axis=1)  # (L, ncols)
        if bnd[r]:
            vals[:] = 0.0
            vals[0, cols.index(r)] = 1.0
        else:
            for ci, col in enumerate(cols):
                if bnd[col]:
                    vals[:, ci] = 0.0
        out_cols.append(np.array(cols))
        out_vals.append(vals)
    return out_cols, out_vals


# ----------------------------------------------------------------------------------------------
# SG operator (Eqs. stochastic_matrix, K_matrix): (K u)_a = sum_b sum_q G_q[a, b] A_q u_b, i.e.
# Y = sum_q A_q X G_q^T for the N x P array X.
# ----------------------------------------------------------------------------------------------

def sg_matvec(prob: SGProblem, X: np.ndarray) -> np.ndarray:
    Y = np.zeros_like(X)
    for k in range(prob.L):
        Gk = prob.G[k]
        if not Gk.any():
            continue
        Y += (prob.A[k] @ X) @ Gk.T
    return Y


def sg_matvec_rows(n, rows, kl, Jq, G, a_min, mu, X):
    """Rows ``rows`` of Y = sum_q A_q X G_q^T, each from its own stiffness rows (sampled parity)."""
    cols, vals = stack_rows_dense(n, rows, kl, Jq, a_min, mu)
    out = np.zeros((len(rows), X.shape[1]))
    for t in range(len(rows)):
        T = vals[t] @ X[cols[t]]             # (L, P): sum_j A_q[r, j] X[j, b]
        out[t] = np.einsum("kab,kb->a", G, T)
    return out


# ----------------------------------------------------------------------------------------------
# ILU(0) (reading R5) and the preconditioners.
# ----------------------------------------------------------------------------------------------

def color4_order(n: int) -> np.ndarray:
    """Four-colour ordering of the nodes of the n x n mesh (reading R18): colour (x mod 2) +
    2 (y mod 2), colours in turn, natural order inside a colour.  No two nodes of one colour are
    neighbours in the 9-point stencil."""
    m = n + 1
    x = np.arange(m * m) % m
    y = np.arange(m * m) // m
    return np.lexsort((np.arange(m * m), (x % 2) + 2 * (y % 2)))


def ilu0(A: scipy.sparse.csr_matrix, order=None):
    """Incomplete LU with zero fill on the pattern of A, no pivoting (the IKJ form: for each
    row i, for each k < i in its pattern, l_ik = a_ik / u_kk and a_ij -= l_ik u_kj for j > k
    present in both rows), in natural order (reading R5) or, with ``order`` (a permutation of the
    rows), of A permuted symmetrically into that order.  Returns (unit lower L, upper U) as CSR,
    with the permutation appended when one was given."""
    if order is not None:
        order = np.asarray(order)
        Ap = A.tocsr()[order][:, order].tocsr()
        Lo, Up = ilu0(Ap)
        return Lo, Up, order
    A = A.tocsr().copy()
    A.sort_indices()
    indptr, indices, data = A.indptr, A.indices, A.data.astype(np.float64).copy()
    n = A.shape[0]
    pos = [dict(zip(indices[indptr[i]:indptr[i + 1]].tolist(), range(indptr[i], indptr[i + 1])))
           for i in range(n)]
    diag = [pos[i][i] for i in range(n)]
    for i in range(n):
        row = pos[i]
        for kk in range(indptr[i], indptr[i + 1]):
            k = indices[kk]
            if k >= i:
                break
            data[kk] = data[kk] / data[diag[k]]
            lik = data[kk]
            for kj in range(diag[k] + 1, indptr[k + 1]):
                j = indices[kj]
                t = row.get(j)
                if t is not None:
                    data[t] -= lik * data[kj]
    LU = scipy.sparse.csr_matrix((data, indices, indptr), shape=A.shape)
    Lo = scipy.sparse.tril(LU, k=-1, format="csr") + scipy.sparse.identity(n, format="csr")
    Up = scipy.sparse.triu(LU, k=0, format="csr")
    return Lo.tocsr(), Up.tocsr()


def ilu0_solve(LU, R):
    """(L U)^{-1} R for a vector or a column block R (in the factorisation's ordering)."""
    if len(LU) == 3:
        Lo, Up, order = LU
        Rp = np.asarray(R)[order]
        Y = scipy.sparse.linalg.spsolve_triangular(Lo, Rp, lower=True, unit_diagonal=True)
        Zp = scipy.sparse.linalg.spsolve_triangular(Up, Y, lower=False)
        Z = np.empty_like(Zp)
        Z[order] = Zp
        return Z
    Lo, Up = LU
    Y = scipy.sparse.linalg.spsolve_triangular(Lo, R, lower=True, unit_diagonal=True)
    return scipy.sparse.linalg.spsolve_triangular(Up, Y, lower=False)


def _richardson(apply_A, LU, rhs, iters):
    """``iters`` steps z <- z + ILU^{-1}(rhs - A z) from z = 0 (the block form of Eq. level_solver)."""
    z = ilu0_solve(LU, rhs)
    for _ in range(iters - 1):
        z = z + ilu0_solve(LU, rhs - apply_A(z))
    return z


def _order(prob, ordering):
    return None if ordering in (None, "natural") else color4_order(prob.n)


def mean_precond(prob: SGProblem, R: np.ndarray, inner_iters: int = 1, LU=None,
                 ordering=None) -> np.ndarray:
    """Mean-based block-diagonal preconditioner (reading R8): every chaos column of R is solved
    with ILU0(A_0) (natural or four-colour ordering), ``inner_iters`` Richardson steps."""
    if LU is None:
        LU = ilu0(prob.A[0], _order(prob, ordering))
    A0 = prob.A[0]
    return _richardson(lambda z: A0 @ z, LU, R, inner_iters)


def fs_blocks(prob: SGProblem, ordering=None):
    """Diagonal blocks K_aa = sum_q G_q[a, a] A_q (Eq. K_matrix) and their ILU(0) factors
    (natural or four-colour ordering)."""
    blocks, facs = [], []
    for a in range(prob.P):
        Kaa = None
        for k in range(prob.L):
            c = prob.G[k, a, a]
            if c != 0.0:
                Kaa = c * prob.A[k] if Kaa is None else Kaa + c * prob.A[k]
        Kaa = Kaa.tocsr()
        Kaa.sort_indices()
        blocks.append(Kaa)
        facs.append(ilu0(Kaa, _order(prob, ordering)))
    return blocks, facs


def _offdiag_apply(prob: SGProblem, a: int, Z: np.ndarray, bs, coupling=None) -> np.ndarray:
    """sum over b in bs of K_ab z_b, K_ab = sum_q G_q[a, b] A_q (``coupling`` replaces the A_q,
    e.g. by copies rounded to a storage precision)."""
    A = prob.A if coupling is None else coupling
    out = np.zeros(Z.shape[0])
    for b in bs:
        for k in range(prob.L):
            c = prob.G[k, a, b]
            if c != 0.0:
                out += c * (A[k] @ Z[:, b])
    return out


def fs_precond(prob: SGProblem, R: np.ndarray, mode: str = "gs", inner_iters: int = 1,
               outer_sweeps: int = 1, blocks=None, coupling=None) -> np.ndarray:
    """Field-split preconditioner: ``outer_sweeps`` steps of Eq. level_solver from zero with P the
    block lower triangle of K (Eq. P_preconditioner, mode 'gs') or its block diagonal
    (mode 'jacobi'); each diagonal block solved by ``inner_iters`` ILU(0)-Richardson steps."""
    if blocks is None:
        blocks = fs_blocks(prob)
    Kd, facs = blocks
    P = prob.P
    Z = np.zeros_like(R)
    for sweep in range(outer_sweeps):
        res = R if sweep == 0 else R - sg_matvec(prob, Z)
        D = np.zeros_like(R)
        for a in range(P):
            rhs = res[:, a].copy()
            if mode == "gs" and a > 0:
                rhs -= _offdiag_apply(prob, a, D, range(a), coupling)
            D[:, a] = _richardson(lambda z, A=Kd[a]: A @ z, facs[a], rhs, inner_iters)
        Z = Z + D
    return Z


# ----------------------------------------------------------------------------------------------
# ILU(0) of multi-field blocks of K and the grouped field split (G-I, G-M-I, G-M-Fg-I; Sec. 3).
# ----------------------------------------------------------------------------------------------

def fg_splits(Jp: np.ndarray, rule: str = "paper"):
    """Field ranges [start, end) of the splits (Sec. 3, Eq. P_group; reading R21).  Fields are
    grouped by the first index of their multi-index (the groups are consecutive ranges in the
    R3 order).  rule 'paper': a group opens a new split when one of its multi-indices has all
    indices equal, else it joins the preceding split; 'groups': every group is a split; 'whole':
    one split of all fields (G-I / G-M-I); 'fields': one split per field (G-F-I / G-M-F-I)."""
    Jp = np.asarray(Jp)
    P = Jp.shape[0]
    if rule == "whole":
        return [(0, P)]
    if rule == "fields":
        return [(a, a + 1) for a in range(P)]
    groups = []
    for a in range(P):
        if not groups or Jp[a, 0] != Jp[groups[-1][0], 0]:
            groups.append([a, a + 1])
        else:
            groups[-1][1] = a + 1
    if rule == "groups":
        return [tuple(g) for g in groups]
    if rule != "paper":
        raise ValueError("unknown split rule")
    splits = []
    for g0, g1 in groups:
        all_equal = any(np.all(Jp[a] == Jp[a, 0]) for a in range(g0, g1))
        if all_equal or not splits:
            splits.append([g0, g1])
        else:
            splits[-1][1] = g1
    return [tuple(sp) for sp in splits]


def block_pattern_matrix(prob: SGProblem, f0: int, f1: int) -> scipy.sparse.csr_matrix:
    """K restricted to the fields f0..f1-1, unknowns node-major (index node * Q + field - f0), on
    the pattern of reading R20: every field of a node coupled to every field of each 9-point
    neighbour, explicit zeros kept."""
    n, Q = prob.n, f1 - f0
    m = n + 1
    Knm = sum(scipy.sparse.kron(prob.A[k], prob.G[k][f0:f1, f0:f1], format="csr")
              for k in range(prob.L)).tocsr()
    Knm.sort_indices()
    indptr, indices, data = [0], [], []
    for node in range(m * m):
        x, y = node % m, node // m
        nbs = [xx + m * yy for yy in range(y - 1, y + 2) for xx in range(x - 1, x + 2)
               if 0 <= xx < m and 0 <= yy < m]
        for a in range(Q):
            r = node * Q + a
            row = dict(zip(Knm.indices[Knm.indptr[r]:Knm.indptr[r + 1]].tolist(),
                           Knm.data[Knm.indptr[r]:Knm.indptr[r + 1]].tolist()))
            for j in nbs:
                for b in range(Q):
                    c = j * Q + b
                    indices.append(c)
                    data.append(row.get(c, 0.0))
            indptr.append(len(indices))
    return scipy.sparse.csr_matrix((np.array(data), np.array(indices), np.array(indptr)),
                                   shape=(m * m * Q, m * m * Q))


def bilu0(prob: SGProblem, f0: int, f1: int, ordering="color4"):
    """ILU(0) of the block of K on fields f0..f1-1 (reading R20): the scalar IKJ ILU(0) of
    ``ilu0`` on the node-major block pattern, nodes in the four-colour (or natural) order, each
    node's fields in order."""
    Q = f1 - f0
    A = block_pattern_matrix(prob, f0, f1)
    nodes = color4_order(prob.n) if ordering == "color4" else np.arange(prob.N)
    order = (nodes[:, None] * Q + np.arange(Q)[None, :]).ravel()
    return ilu0(A, order)


def bilu0_solve(LU, R: np.ndarray) -> np.ndarray:
    """(L U)^{-1} R for R of shape N x Q (node-major flattening)."""
    N, Q = R.shape
    return ilu0_solve(LU, R.reshape(N * Q)).reshape(N, Q)


def fg_blocks(prob: SGProblem, splits, ordering="color4"):
    """The ILU(0) factors of every split's diagonal block (reading R20)."""
    return [bilu0(prob, f0, f1, ordering) for f0, f1 in splits]


def fg_precond(prob: SGProblem, R: np.ndarray, splits, facs=None, mode: str = "gs",
               coupling=None) -> np.ndarray:
    """Grouped field split (Sec. 3, Eq. P_group): block Gauss-Seidel over the splits (or block
    Jacobi, mode 'jacobi'), split s solved with the ILU(0) of its diagonal block K_ss after
    subtracting sum_{t<s} K_st z_t.  Singleton splits give the field split of Eq.
    P_preconditioner; one split of all fields gives ILU(0) of K (G-I)."""
    if facs is None:
        facs = fg_blocks(prob, splits)
    Z = np.zeros_like(R)
    for s, (f0, f1) in enumerate(splits):
        rhs = R[:, f0:f1].copy()
        if mode == "gs" and s > 0:
            prev = range(0, f0)
            for a in range(f0, f1):
                rhs[:, a - f0] -= _offdiag_apply(prob, a, Z, prev, coupling)
        Z[:, f0:f1] = bilu0_solve(facs[s], rhs)
    return Z


# ----------------------------------------------------------------------------------------------
# Restarted, right-preconditioned GMRES with CGS2 Arnoldi and Givens rotations (reading R7).
# ----------------------------------------------------------------------------------------------

def gmres(apply_K, apply_M, F, x0=None, restart=30, rtol=1e-10, atol=0.0, max_iters=1000,
          flexible=False):
    """Solve K x = F.  Vectors are flattened N*P arrays.  Returns (x, info) with info keys
    iters, restarts, rel_resid (true residual), converged, history (Givens estimates)."""
    F = np.asarray(F, dtype=np.float64).ravel()
    x = np.zeros_like(F) if x0 is None else np.asarray(x0, dtype=np.float64).ravel().copy()
    bnorm = float(np.linalg.norm(F))
    target = max(rtol * bnorm, atol)
    if bnorm == 0.0:
        return np.zeros_like(F), dict(iters=0, restarts=0, rel_resid=0.0, converged=True, history=[])
    r = F - apply_K(x)
    beta = float(np.linalg.norm(r))
    iters, restarts, history = 0, 0, []
    m = restart
    while beta > target and iters < max_iters:
        V = np.zeros((m + 1, F.size))
        Z = np.zeros((m, F.size)) if flexible else None
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            z = apply_M(V[j])
            if flexible:
                Z[j] = z
            w = apply_K(z)
            h = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h
            h2 = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h2
            h = h + h2
            hn = float(np.linalg.norm(w))
            H[:j + 1, j] = h
            H[j + 1, j] = hn
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = math.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            iters += 1
            k = j + 1
            history.append(abs(g[j + 1]) / bnorm)
            if hn > 0.0:
                V[j + 1] = w / hn
            if abs(g[j + 1]) <= target or iters >= max_iters or hn == 0.0:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        if flexible:
            x = x + Z[:k].T @ y
        else:
            x = x + apply_M(V[:k].T @ y)
        r = F - apply_K(x)
        beta = float(np.linalg.norm(r))
        restarts += 1
    return x, dict(iters=iters, restarts=restarts, rel_resid=beta / bnorm,
                   converged=beta <= target, history=history)


# ----------------------------------------------------------------------------------------------
# Geometric multigrid V-cycle (Sec. 3: GMRES preconditioned by MG, the level solver of
# Eq. level_solver as smoother with i_max = 1 pre- and post-smoothing step, a direct solve on the
# coarsest level; Sec. 4: V-cycle on the midpoint-refined hierarchy that starts from 2 x 2 cells).
# Readings where the paper is silent:
#   R16 each level is the same SG problem discretised on its own mesh (the paper's FE library
#       assembles every level); the coarse space is the nested Q1 space, so the prolongation is
#       bilinear interpolation and the restriction its transpose; boundary nodes carry no coarse
#       unknowns (the coarse space keeps the zero Dirichlet condition).
#   R17 pre- and post-smoothing are one step each of Eq. level_solver with the chosen block
#       preconditioner (mean-based, field-split Gauss-Seidel or Jacobi), from zero for the
#       pre-smoothing step.
# ----------------------------------------------------------------------------------------------

def prolongation(nc: int) -> scipy.sparse.csr_matrix:
    """Bilinear interpolation from the nc x nc mesh to the 2nc x 2nc mesh (reading R16): an
    (N_fine x N_coarse) matrix whose columns of coarse boundary nodes are zero."""
    mc, mf = nc + 1, 2 * nc + 1
    bc = boundary_mask(nc)
    rows, cols, vals = [], [], []
    for jf in range(mf):
        for i_f in range(mf):
            # coarse nodes around the fine node and their bilinear weights
            xs = [(i_f // 2, 1.0)] if i_f % 2 == 0 else [(i_f // 2, 0.5), (i_f // 2 + 1, 0.5)]
            ys = [(jf // 2, 1.0)] if jf % 2 == 0 else [(jf // 2, 0.5), (jf // 2 + 1, 0.5)]
            for ic, wx in xs:
                for jc, wy in ys:
                    c = ic + mc * jc
                    if not bc[c]:
                        rows.append(i_f + mf * jf)
                        cols.append(c)
                        vals.append(wx * wy)
    return scipy.sparse.csr_matrix((vals, (rows, cols)), shape=(mf * mf, mc * mc))


def mg_levels(n, M, p, coarse=2, **kw):
    """The SG problem on every mesh of the hierarchy coarse, 2 coarse, ..., n (reading R16),
    coarsest first."""
    sizes = [n]
    while sizes[-1] > coarse:
        if sizes[-1] % 2:
            raise ValueError("n must be coarse times a power of two")
        sizes.append(sizes[-1] // 2)
    if sizes[-1] != coarse:
        raise ValueError("n must be coarse times a power of two")
    return [build_problem(s, M, p, **kw) for s in reversed(sizes)]


def mg_setup(levels, smoother="fs_gs", ordering=None):
    """Per level: smoother data (ILU(0) factors in natural or four-colour ordering), the
    prolongation from the level below, and the dense coarsest-level operator for the direct
    solve.  Smoothers: 'fs_gs', 'fs_jacobi', 'mean', and 'fg' / 'fg:<rule>' (the grouped field
    split with the split rule of ``fg_splits``; 'fg:whole' is G-M-I)."""
    data = []
    for li, prob in enumerate(levels):
        d = {"P": prolongation(levels[li - 1].n) if li > 0 else None}
        if li == 0:
            d["K"] = sum(np.kron(prob.G[k], prob.A[k].toarray()) for k in range(prob.L))
        elif smoother == "mean":
            d["LU"] = ilu0(prob.A[0], _order(prob, ordering))
        elif smoother.startswith("fg"):
            rule = smoother.split(":")[1] if ":" in smoother else "paper"
            d["splits"] = fg_splits(prob.Jp, rule)
            d["fg"] = fg_blocks(prob, d["splits"], ordering or "color4")
        else:
            d["blocks"] = fs_blocks(prob, ordering)
        data.append(d)
    return data


def _smooth(prob, d, smoother, r):
    if smoother == "mean":
        return mean_precond(prob, r, LU=d["LU"])
    if smoother.startswith("fg"):
        return fg_precond(prob, r, d["splits"], d["fg"])
    return fs_precond(prob, r, mode="gs" if smoother == "fs_gs" else "jacobi", blocks=d["blocks"])


def mg_vcycle(levels, data, b, smoother="fs_gs", level=None):
    """One V-cycle for K u = b on ``level`` (default: finest) from u = 0 (Sec. 3): pre-smoothing,
    restriction of the residual, the V-cycle of the level below, prolongation of its correction,
    post-smoothing; the direct solve on the coarsest level."""
    if level is None:
        level = len(levels) - 1
    prob, d = levels[level], data[level]
    if level == 0:
        x = np.linalg.solve(d["K"], b.T.ravel())          # mode-major unknown vector
        return x.reshape(prob.P, prob.N).T
    u = _smooth(prob, d, smoother, b)                     # Eq. level_solver from zero
    r = b - sg_matvec(prob, u)
    bc = d["P"].T @ r                                      # restriction = transpose
    uc = mg_vcycle(levels, data, bc, smoother, level - 1)
    u = u + d["P"] @ uc
    return u + _smooth(prob, d, smoother, b - sg_matvec(prob, u))
