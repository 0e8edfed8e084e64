"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each test checks one oracle function against something the paper or the mathematics fixes: a
golden value the paper prints, a closed form, an independent quadrature, brute force on a tiny
case, or a defining property.  They are chosen so that a dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of them.
"""

import itertools
import math
import os

import numpy as np
import scipy.linalg
import pytest
import scipy.sparse
import scipy.sparse.linalg
from numpy.polynomial import hermite_e as He

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _psi(k, y):
    """Normalised probabilists' Hermite polynomial, evaluated by numpy's own series code."""
    c = np.zeros(k + 1)
    c[k] = 1.0
    return He.hermeval(y, c) / math.sqrt(math.factorial(k))


def _gh(npts):
    """Gauss-Hermite rule for the N(0, 1) density."""
    x, w = He.hermegauss(npts)
    return x, w / math.sqrt(2.0 * math.pi)


# ------------------------------------------------------------------ multi-indices (Sec. 2.2)

def test_multi_index_counts_golden():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "multi_index_counts.txt"))
            if l.strip() and not l.startswith("#")]
    for N, p, Mp in rows:
        assert len(O.multi_indices(int(N), int(p))) == int(Mp)


def test_multi_index_set_is_the_total_degree_set_in_stated_order():
    for M, p in [(1, 4), (2, 3), (3, 2), (4, 3)]:
        J = O.multi_indices(M, p)
        brute = sorted(t for t in itertools.product(range(p + 1), repeat=M) if sum(t) <= p)
        # lexicographic with the last index fastest is exactly Python's tuple order
        assert [tuple(r) for r in J] == brute
        assert tuple(J[0]) == (0,) * M


# ------------------------------------------------------------------ triple products (Sec. 2.2)

def test_hermite_triple_1d_against_gauss_hermite():
    y, w = _gh(30)
    for i, j, k in itertools.product(range(9), repeat=3):
        q = float(np.sum(w * _psi(i, y) * _psi(j, y) * _psi(k, y)))
        assert abs(O.hermite_triple_1d(i, j, k) - q) < 1e-10 * max(1.0, abs(q)), (i, j, k)


def test_triple_product_tensor_against_multivariate_quadrature():
    M, p = 2, 2
    Jp, Jq = O.multi_indices(M, p), O.multi_indices(M, 2 * p)
    G = O.triple_products(Jq, Jp)
    y, w = _gh(12)
    Y1, Y2 = np.meshgrid(y, y, indexing="ij")
    W = np.outer(w, w)

    def psi(idx):
        return _psi(int(idx[0]), Y1) * _psi(int(idx[1]), Y2)

    for k in range(len(Jq)):
        for a in range(len(Jp)):
            for b in range(len(Jp)):
                q = np.sum(W * psi(Jq[k]) * psi(Jp[a]) * psi(Jp[b]))
                assert abs(G[k, a, b] - q) < 1e-12, (k, a, b)
    assert np.allclose(G[0], np.eye(len(Jp)), atol=0, rtol=0)  # psi_0 = 1: orthonormality
    assert np.array_equal(G, G.transpose(0, 2, 1))


# ------------------------------------------------------------------ chaos coefficients (Eq. dataProjection)

def test_chaos_coefficients_against_quadrature():
    rng = np.random.default_rng(7)
    M, q = 2, 6
    Jq = O.multi_indices(M, q)
    g = rng.normal(scale=0.6, size=(M, 5))
    a_min, mu = 0.01, 0.2
    got = O.chaos_coefficients(g, Jq, a_min, mu)
    y, w = _gh(60)
    Y1, Y2 = np.meshgrid(y, y, indexing="ij")
    W = np.outer(w, w)
    for t in range(g.shape[1]):
        a = a_min + np.exp(mu + g[0, t] * Y1 + g[1, t] * Y2)
        for k, idx in enumerate(Jq):
            ref = np.sum(W * a * _psi(int(idx[0]), Y1) * _psi(int(idx[1]), Y2))
            assert abs(got[k, t] - ref) < 1e-12 * max(1.0, abs(ref)), (t, k)


def test_chaos_parseval_1d():
    # sum_q a_q^2 -> E[a^2] = exp(2 mu + 2 g^2) for a = exp(mu + g y)
    g = np.array([[0.7]])
    mu = -0.1
    Jq = O.multi_indices(1, 40)
    aq = O.chaos_coefficients(g, Jq, 0.0, mu)
    assert abs(np.sum(aq ** 2) - math.exp(2 * mu + 2 * 0.49)) < 1e-12


# ------------------------------------------------------------------ KL (Eqs. gen_eigen, standard_deviation)

def test_kl_1d_against_nystrom_and_orthonormality():
    for ell in (0.5, 1.0, 2.0):
        modes = O.kl_modes_1d(ell, 6)
        npts = 4000
        x = (np.arange(npts) + 0.5) / npts
        C = np.exp(-np.abs(x[:, None] - x[None, :]) / ell) / npts
        ev = np.sort(np.linalg.eigvalsh(C))[::-1][:6]
        mus = np.array([m[2] for m in modes])
        assert np.all(np.diff(mus) < 0)
        assert np.allclose(mus, ev, rtol=2e-5, atol=0)
        t, w = np.polynomial.legendre.leggauss(200)
        xs, ws = 0.5 + 0.5 * t, 0.5 * w
        F = np.array([O.kl_eval_1d(m, xs) for m in modes])
        gram = (F * ws) @ F.T
        assert np.allclose(gram, np.eye(6), atol=1e-12)
        # eigen-equation at a few points: int C(x, s) f(s) ds = mu f(x), split at s = x
        for xv in (0.1, 0.37, 0.8):
            for mode in modes[:4]:
                lhs = 0.0
                for lo, hi in ((0.0, xv), (xv, 1.0)):
                    ss = lo + (hi - lo) * (0.5 + 0.5 * t)
                    lhs += np.sum(0.5 * (hi - lo) * w * np.exp(-np.abs(xv - ss) / ell)
                                  * O.kl_eval_1d(mode, ss))
                assert abs(lhs - mode[2] * O.kl_eval_1d(mode, xv)) < 1e-12


def _galerkin_kl(n, sigma, ell, M):
    """The paper's Galerkin KL (Sec. 2.1): Q1 on an n x n mesh of the unit square, the covariance
    integrated with 3 x 3 Gauss points per cell, C v = lam Mass v; top M eigenpairs (vectors at
    the nodes, Mass-orthonormal)."""
    g = np.array([-np.sqrt(0.6), 0.0, np.sqrt(0.6)])
    w = np.array([5.0, 8.0, 5.0]) / 9.0
    h, m = 1.0 / n, n + 1
    pts, wts, cols, vals = [], [], [], []
    for ey in range(n):
        for ex in range(n):
            for a in range(3):
                for b in range(3):
                    s, t = (g[a] + 1) / 2, (g[b] + 1) / 2
                    pts.append(((ex + s) * h, (ey + t) * h))
                    wts.append(w[a] * w[b] * h * h / 4)
                    cols.append([ex + m * ey, ex + 1 + m * ey, ex + m * (ey + 1), ex + 1 + m * (ey + 1)])
                    vals.append([(1 - s) * (1 - t), s * (1 - t), (1 - s) * t, s * t])
    pts, wts = np.array(pts), np.array(wts)
    Phi = np.zeros((len(pts), m * m))
    for q in range(len(pts)):
        Phi[q, cols[q]] = vals[q]
    dx = np.abs(pts[:, None, 0] - pts[None, :, 0]) + np.abs(pts[:, None, 1] - pts[None, :, 1])
    WP = wts[:, None] * Phi
    lam, V = scipy.linalg.eigh(WP.T @ (sigma ** 2 * np.exp(-dx / ell)) @ WP, WP.T @ Phi)
    return lam[::-1][:M], V[:, ::-1][:, :M]


def test_kl_closed_form_is_the_limit_of_the_galerkin_kl():
    # the paper computes the KL modes by a Galerkin FE eigenproblem; for the separable exponential
    # covariance the closed form is its mesh limit: eigenvalues converge at O(h^2) and the first
    # eigenfunction agrees at the nodes (reading R9: the closed form stands for the Galerkin KL)
    kl = O.kl_modes_2d(1.0, 0.5, 6)
    errs = [np.abs(_galerkin_kl(n, 1.0, 0.5, 6)[0] - kl.lam) / kl.lam for n in (4, 8, 16)]
    assert np.all(errs[2] < 3e-3)
    assert 3.0 < errs[0][0] / errs[1][0] < 5.0 and 3.0 < errs[1][0] / errs[2][0] < 5.0
    _, V = _galerkin_kl(16, 1.0, 0.5, 1)
    x = np.arange(17) / 16.0
    X1, X2 = np.meshgrid(x, x)          # node id = x1 index + 17 * x2 index
    b1 = O.kl_fields(kl, X1.ravel(), X2.ravel())[0] / np.sqrt(kl.lam[0])
    v = V[:, 0] * np.sign(V[:, 0] @ b1)
    assert np.abs(v - b1).max() <= 5e-3 * np.abs(b1).max()


def test_kl_trace_sums_to_one():
    # trace of the 1-D operator on [0, 1] is int C(x, x) dx = 1
    modes = O.kl_modes_1d(0.5, 4000)
    s = sum(m[2] for m in modes)
    assert 0.999 < s < 1.0


def test_kl_2d_ordering_and_ties():
    kl = O.kl_modes_2d(0.5, 1.0, 6)
    assert kl.ij[0] == (0, 0)
    assert kl.ij[1] == (0, 1) and kl.ij[2] == (1, 0)  # equal eigenvalues: lexicographic
    assert kl.lam[1] == kl.lam[2]
    assert np.all(np.diff(kl.lam) <= 0)
    mu0 = kl.modes1d[0][2]
    assert abs(kl.lam[0] - 0.25 * mu0 * mu0) < 1e-16


def _gl01(npts, lo=0.0, hi=1.0):
    t, w = np.polynomial.legendre.leggauss(npts)
    return lo + (hi - lo) * (0.5 + 0.5 * t), 0.5 * (hi - lo) * w


def test_kl_fields_are_sqrt_lambda_scaled_2d_eigenfunctions():
    # Eq. aKL with Eq. standard_deviation: g_n = sqrt(lambda_n) b_n with b_n orthonormal on
    # [0,1]^2 and C b_n = lambda_n b_n for C(x, y) = sigma^2 exp(-(|x1-y1| + |x2-y2|)/ell).
    # So int g_n g_m = lambda_n delta_nm (fixes the sqrt(lambda) scaling), and the 2-D
    # eigen-equation holds for g_n as written out from the covariance, not from the 1-D factors.
    sigma, ell, M = 0.7, 0.5, 6
    kl = O.kl_modes_2d(sigma, ell, M)
    xs, ws = _gl01(60)
    X1, X2 = np.meshgrid(xs, xs, indexing="ij")
    W2 = np.outer(ws, ws)
    g = O.kl_fields(kl, X1.ravel(), X2.ravel()).reshape(M, 60, 60)
    gram = np.einsum("nij,mij,ij->nm", g, g, W2)
    assert np.allclose(gram, np.diag(kl.lam), rtol=0, atol=1e-13)
    for x in [(0.2, 0.7), (0.55, 0.31), (0.9, 0.05)]:
        lhs = np.zeros(M)
        # the kernel has kinks at y = x: split both directions there
        for lo1, hi1 in ((0.0, x[0]), (x[0], 1.0)):
            for lo2, hi2 in ((0.0, x[1]), (x[1], 1.0)):
                y1, w1 = _gl01(40, lo1, hi1)
                y2, w2 = _gl01(40, lo2, hi2)
                Y1, Y2 = np.meshgrid(y1, y2, indexing="ij")
                C = sigma ** 2 * np.exp(-(np.abs(x[0] - Y1) + np.abs(x[1] - Y2)) / ell)
                gy = O.kl_fields(kl, Y1.ravel(), Y2.ravel()).reshape(M, *Y1.shape)
                lhs += np.einsum("ij,nij->n", C * np.outer(w1, w2), gy)
        gx = O.kl_fields(kl, [x[0]], [x[1]])[:, 0]
        assert np.allclose(lhs, kl.lam * gx, rtol=0, atol=1e-12)


def test_kl_fields_orientation_of_reading_r2():
    # Reading R2 puts the first 1-D factor on x1.  The first 1-D mode is even about 1/2 and the
    # second odd, so the mode with factors (0, 1) is even in x1 and odd in x2, and (1, 0) the
    # reverse; a swap of x1 and x2 anywhere in the oracle flips these parities.
    kl = O.kl_modes_2d(1.0, 1.0, 3)
    assert kl.ij[1] == (0, 1) and kl.ij[2] == (1, 0)
    rng = np.random.default_rng(5)
    x1, x2 = rng.random(20), rng.random(20)
    g = O.kl_fields(kl, x1, x2)
    g_m1 = O.kl_fields(kl, 1.0 - x1, x2)
    g_m2 = O.kl_fields(kl, x1, 1.0 - x2)
    assert np.allclose(g_m1[1], g[1], atol=1e-14) and np.allclose(g_m2[1], -g[1], atol=1e-14)
    assert np.allclose(g_m1[2], -g[2], atol=1e-14) and np.allclose(g_m2[2], g[2], atol=1e-14)
    assert np.abs(g[1]).max() > 0.1 and np.abs(g[2]).max() > 0.1


def test_kl_fields_mercer_partial_sums():
    # Mercer: sum_n g_n(x)^2 -> C(x, x) = sigma^2 from below; the remainder is
    # sum_{n>M} lambda_n b_n(x)^2 <= max|b|^2 (sigma^2 - sum_{n<=M} lambda_n).
    sigma, ell = 0.8, 0.5
    rng = np.random.default_rng(9)
    x1, x2 = rng.random(15), rng.random(15)
    prev = None
    for M in (10, 60, 300):
        kl = O.kl_modes_2d(sigma, ell, M)
        s = np.sum(O.kl_fields(kl, x1, x2) ** 2, axis=0)
        tail = sigma ** 2 - kl.lam.sum()
        # |f| <= 1 / sqrt(1/2 - 1/(2 w)) for the normalised 1-D modes, so |b|^2 <= 4 here
        assert np.all(s <= sigma ** 2 + 1e-12)
        assert np.all(sigma ** 2 - s <= 4.0 * tail + 1e-12), (M, (sigma ** 2 - s).max(), tail)
        if prev is not None:
            assert np.all(s >= prev - 1e-14)
        prev = s
    assert tail < 0.03 * sigma ** 2


# ------------------------------------------------------------------ FE assembly (Eq. A_q) and boundary data

def test_sigma_zero_gives_q1_laplacian_stencil():
    n = 6
    prob = O.build_problem(n, M=2, p=2, sigma=0.0, ell=1.0)
    A0 = prob.A[0].toarray()
    m = n + 1
    i = 3 + m * 3  # interior node
    row = A0[i]
    assert abs(row[i] - 8.0 / 3.0) < 1e-14
    for d in (-m - 1, -m, -m + 1, -1, 1, m - 1, m, m + 1):
        assert abs(row[i + d] + 1.0 / 3.0) < 1e-14
    for k in range(1, prob.L):
        assert abs(prob.A[k]).max() == 0.0
    # load vector: f h^2 at interior nodes, mode 0 only
    assert abs(prob.F[i, 0] - 1.0 / n ** 2) < 1e-15
    assert np.all(prob.F[:, 1:] == 0)


def _series_centre(terms=400):
    s = 0.0
    for i in range(1, terms, 2):
        for j in range(1, terms, 2):
            s += 16.0 / (math.pi ** 4 * i * j * (i * i + j * j)) * math.sin(i * math.pi / 2) * math.sin(j * math.pi / 2)
    return s


def test_deterministic_limit_converges_at_second_order():
    exact = _series_centre()
    errs = []
    for n in (8, 16, 32):
        prob = O.build_problem(n, M=2, p=1, sigma=0.0)
        u = scipy.sparse.linalg.spsolve(prob.A[0].tocsc(), prob.F[:, 0])
        m = n + 1
        errs.append(abs(u[n // 2 + m * (n // 2)] - exact))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5, errs


# ------------------------------------------------------------------ SG operator (Eqs. stochastic_matrix, K_matrix)

def _dense_K(prob):
    return sum(np.kron(prob.G[k], prob.A[k].toarray()) for k in range(prob.L))


def test_sg_matvec_equals_kronecker_sum():
    prob = O.build_problem(3, M=2, p=2, sigma=0.7, ell=0.8, a_min=0.01, mu=0.1)
    K = _dense_K(prob)
    rng = np.random.default_rng(3)
    X = rng.normal(size=(prob.N, prob.P))
    Y = O.sg_matvec(prob, X)
    ref = (K @ X.T.ravel()).reshape(prob.P, prob.N).T  # mode-major unknown vector
    assert np.allclose(Y, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    assert np.allclose(K, K.T, atol=1e-14)
    assert np.all(np.linalg.eigvalsh(K) > 0)


def _stiffness_with_coefficient(n, coef):
    """Q1 stiffness for a coefficient given at the 9 Gauss points of every cell (test-side
    assembly, written independently of the oracle)."""
    t = [0.5 - 0.5 * math.sqrt(0.6), 0.5, 0.5 + 0.5 * math.sqrt(0.6)]
    w = [5 / 18, 8 / 18, 5 / 18]
    m = n + 1
    A = np.zeros((m * m, m * m))
    for ey in range(n):
        for ex in range(n):
            nodes = [ex + m * ey, ex + 1 + m * ey, ex + m * (ey + 1), ex + 1 + m * (ey + 1)]
            c = ex + n * ey
            for gy in range(3):
                for gx in range(3):
                    xi, eta = t[gx], t[gy]
                    grads = np.array([[eta - 1, xi - 1], [1 - eta, -xi], [-eta, 1 - xi], [eta, xi]])
                    A[np.ix_(nodes, nodes)] += w[gx] * w[gy] * coef[c, gy * 3 + gx] * grads @ grads.T
    return A


def test_sg_blocks_equal_expectation_over_y():
    # K_ab = E[A(y) psi_a psi_b] exactly when q = 2p (Eq. linear_algebraic): checks the chaos
    # coefficients, the triple products and the contraction order together, with the Dirichlet
    # treatment applied on both sides.
    n, M, p = 3, 2, 2
    sigma, ell, a_min, mu = 0.6, 0.7, 0.02, 0.1
    prob = O.build_problem(n, M, p, sigma=sigma, ell=ell, a_min=a_min, mu=mu)
    tt = [0.5 - 0.5 * math.sqrt(0.6), 0.5, 0.5 + 0.5 * math.sqrt(0.6)]
    gp = np.array([[(ex + tt[gx]) / n, (ey + tt[gy]) / n] for ey in range(n) for ex in range(n)
                   for gy in range(3) for gx in range(3)])
    g = O.kl_fields(prob.kl, gp[:, 0], gp[:, 1]).reshape(M, n * n, 9)
    y, w = _gh(40)
    N, P = prob.N, prob.P
    Kref = np.zeros((P * N, P * N))
    for i1, y1 in enumerate(y):
        for i2, y2 in enumerate(y):
            coef = a_min + np.exp(mu + g[0] * y1 + g[1] * y2)
            Ay = _stiffness_with_coefficient(n, coef)
            ps = np.array([_psi(int(ix[0]), y1) * _psi(int(ix[1]), y2) for ix in prob.Jp])
            Kref += w[i1] * w[i2] * np.kron(np.outer(ps, ps), Ay)
    bnd = prob.boundary
    keep = np.tile(~bnd, P)
    Kref[~keep, :] = 0.0
    Kref[:, ~keep] = 0.0
    Kref[np.diag_indices_from(Kref)] += (~keep).astype(float)
    K = _dense_K(prob)
    assert np.allclose(K, Kref, rtol=0, atol=1e-11 * np.abs(Kref).max())


# ------------------------------------------------------------------ ILU(0) and preconditioners

def test_ilu0_defining_property():
    prob = O.build_problem(5, M=2, p=1, sigma=0.5)
    A = prob.A[0]
    Lo, Up = O.ilu0(A)
    LU = (Lo @ Up).toarray()
    pat = A.toarray() != 0
    pat |= np.eye(A.shape[0], dtype=bool)
    Ad = A.toarray()
    assert np.allclose(LU[pat], Ad[pat], atol=1e-13)
    assert set(zip(*Lo.nonzero())) | set(zip(*Up.nonzero())) <= set(zip(*np.nonzero(pat)))


def test_ilu0_of_tridiagonal_is_exact():
    n = 40
    T = scipy.sparse.diags([-np.ones(n - 1), 2.5 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="csr")
    b = np.arange(n, dtype=float)
    x = O.ilu0_solve(O.ilu0(T), b)
    assert np.allclose(T @ x, b, atol=1e-12)


def _small_problem():
    return O.build_problem(4, M=2, p=2, sigma=0.8, ell=0.7)


def test_mean_precond_richardson_converges_to_mean_inverse():
    prob = _small_problem()
    rng = np.random.default_rng(5)
    R = rng.normal(size=(prob.N, prob.P))
    Z1 = O.mean_precond(prob, R, inner_iters=1)
    Lo, Up = O.ilu0(prob.A[0])
    assert np.allclose((Lo @ Up) @ Z1, R, atol=1e-12)
    Zinf = O.mean_precond(prob, R, inner_iters=200)
    ref = scipy.sparse.linalg.spsolve(prob.A[0].tocsc(), R)
    assert np.allclose(Zinf, ref, atol=1e-11 * np.abs(ref).max())


def _dense_blocks(prob, facs, mode):
    N, P = prob.N, prob.P
    Pm = np.zeros((N * P, N * P))
    for a in range(P):
        for b in range(P):
            if b > a or (b < a and mode == "jacobi"):
                continue
            if a == b:
                Lo, Up = facs[a]
                blk = (Lo @ Up).toarray()
            else:
                blk = sum(prob.G[k, a, b] * prob.A[k].toarray() for k in range(prob.L))
            Pm[a * N:(a + 1) * N, b * N:(b + 1) * N] = blk
    return Pm


@pytest.mark.parametrize("mode", ["gs", "jacobi"])
def test_field_split_solves_its_block_triangular_matrix(mode):
    prob = _small_problem()
    blocks = O.fs_blocks(prob)
    rng = np.random.default_rng(11)
    R = rng.normal(size=(prob.N, prob.P))
    Pm = _dense_blocks(prob, blocks[1], mode)
    # one sweep: Z = Ptilde^{-1} R (Eq. P_preconditioner with ILU diagonal blocks)
    Z = O.fs_precond(prob, R, mode=mode, blocks=blocks)
    assert np.allclose(Pm @ Z.T.ravel(), R.T.ravel(), atol=1e-12)
    # three sweeps follow Eq. level_solver from zero
    K = _dense_K(prob)
    z = np.zeros(prob.N * prob.P)
    r = R.T.ravel()
    for _ in range(3):
        z = z + np.linalg.solve(Pm, r - K @ z)
    Z3 = O.fs_precond(prob, R, mode=mode, outer_sweeps=3, blocks=blocks)
    assert np.allclose(Z3.T.ravel(), z, atol=1e-11 * np.abs(z).max())


def test_field_split_diagonal_blocks_are_sums_of_stack():
    prob = _small_problem()
    Kd, _ = O.fs_blocks(prob)
    K = _dense_K(prob)
    N = prob.N
    for a in range(prob.P):
        assert np.allclose(Kd[a].toarray(), K[a * N:(a + 1) * N, a * N:(a + 1) * N], atol=1e-14)


# ------------------------------------------------------------------ GMRES (Sec. 3)

def test_gmres_iterates_minimise_over_the_krylov_space():
    prob = _small_problem()
    K = _dense_K(prob)
    F = prob.F.T.ravel()
    blocks = O.fs_blocks(prob)
    Pm = _dense_blocks(prob, blocks[1], "jacobi")
    Minv = np.linalg.inv(Pm)
    for k in range(1, 6):
        x, info = O.gmres(lambda v: K @ v, lambda v: Minv @ v, F, restart=k, max_iters=k, rtol=1e-30)
        # brute force: x = M^{-1} V c with V spanning {F, (K M^{-1}) F, ...}
        B = K @ Minv
        basis = [F]
        for _ in range(k - 1):
            basis.append(B @ basis[-1])
        V = np.linalg.qr(np.array(basis).T)[0]
        c = np.linalg.lstsq(K @ Minv @ V, F, rcond=None)[0]
        ref = Minv @ (V @ c)
        assert np.allclose(x, ref, atol=1e-9 * np.abs(ref).max()), k
        assert info["iters"] == k


def test_gmres_converges_to_direct_solution_with_monotone_estimates():
    prob = _small_problem()
    K = _dense_K(prob)
    F = prob.F.T.ravel()
    blocks = O.fs_blocks(prob)

    def M(v):
        return O.fs_precond(prob, v.reshape(prob.P, prob.N).T, blocks=blocks).T.ravel()

    x, info = O.gmres(lambda v: K @ v, M, F, restart=5, rtol=1e-13)
    ref = np.linalg.solve(K, F)
    assert info["converged"] and info["restarts"] > 1
    assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)
    h = info["history"]
    assert all(h[i + 1] <= h[i] * (1 + 1e-8) + 1e-15 for i in range(len(h) - 1))


# ------------------------------------------------------------------ whole SG solve vs collocation of E[u]

def test_sg_moments_converge_to_gauss_hermite_collocation():
    # E[u] and E[u^2] of the discrete problem with the truncated-KL lognormal coefficient,
    # by tensor Gauss-Hermite collocation over y (one deterministic FE solve per node), must be
    # matched by the SG solution's mode 0 and sum of squared modes, increasingly well in p.
    n, M = 6, 2
    sigma, ell = 0.5, 1.0
    base = O.build_problem(n, M, 1, sigma=sigma, ell=ell)
    tt = [0.5 - 0.5 * math.sqrt(0.6), 0.5, 0.5 + 0.5 * math.sqrt(0.6)]
    gp = np.array([[(ex + tt[gx]) / n, (ey + tt[gy]) / n] for ey in range(n) for ex in range(n)
                   for gy in range(3) for gx in range(3)])
    g = O.kl_fields(base.kl, gp[:, 0], gp[:, 1]).reshape(M, n * n, 9)
    y, w = _gh(24)
    keep = ~base.boundary
    Eu = np.zeros(base.N)
    Eu2 = np.zeros(base.N)
    for i1, y1 in enumerate(y):
        for i2, y2 in enumerate(y):
            A = _stiffness_with_coefficient(n, np.exp(g[0] * y1 + g[1] * y2))
            u = np.zeros(base.N)
            u[keep] = np.linalg.solve(A[np.ix_(keep, keep)], base.F[keep, 0])
            Eu += w[i1] * w[i2] * u
            Eu2 += w[i1] * w[i2] * u * u
    errs = []
    for p in (1, 2, 3, 4):
        prob = O.build_problem(n, M, p, sigma=sigma, ell=ell)
        K = _dense_K(prob)
        X = np.linalg.solve(K, prob.F.T.ravel()).reshape(prob.P, prob.N).T
        errs.append((np.abs(X[:, 0] - Eu).max(), np.abs((X ** 2).sum(1) - Eu2).max()))
    for (e1, e2), (f1, f2) in zip(errs, errs[1:]):
        assert f1 < 0.5 * e1 and f2 < 0.5 * e2, errs
    assert errs[-1][0] < 2e-6 * np.abs(Eu).max(), errs


@pytest.mark.parametrize("n", [3, 4, 5, 6, 7, 8])
def test_sampled_rows_equal_rows_of_the_assembled_operator(n):
    # the row-sampled operator (built from the cells around each node) must reproduce every row
    # of the pinned full operator: corner, edge, next-to-boundary and interior rows
    prob = O.build_problem(n, M=2, p=2, sigma=0.6, ell=0.7, a_min=0.02, mu=0.05)
    rng = np.random.default_rng(n)
    X = rng.normal(size=(prob.N, prob.P))
    Y = O.sg_matvec(prob, X)
    rows = np.arange(prob.N)
    got = O.sg_matvec_rows(n, rows, prob.kl, prob.Jq, prob.G, prob.a_min, prob.mu, X)
    assert np.allclose(got, Y, rtol=0, atol=1e-13 * np.abs(Y).max())
    cols, vals = O.stack_rows_dense(n, rows, prob.kl, prob.Jq, prob.a_min, prob.mu)
    for r in rows:
        for k in range(prob.L):
            dense = prob.A[k].getrow(r).toarray()[0]
            ref = np.zeros_like(dense)
            ref[cols[r]] = vals[r][k]
            assert np.allclose(dense, ref, rtol=0, atol=1e-14), (r, k)


# ------------------------------------------------------------------ multigrid V-cycle (Sec. 3, Sec. 4)

def test_prolongation_reproduces_the_coarse_finite_element_function():
    # the fine nodal values of a coarse Q1 function are its values at the fine nodes; the coarse
    # function is written out with hat functions, boundary nodes carrying zero (reading R16)
    nc = 4
    mc, mf, H = nc + 1, 2 * nc + 1, 1.0 / nc
    rng = np.random.default_rng(2)
    uc = rng.normal(size=mc * mc)
    uc[O.boundary_mask(nc)] = 0.0
    xf = (np.arange(mf * mf) % mf) / (2 * nc)
    yf = (np.arange(mf * mf) // mf) / (2 * nc)
    ref = np.zeros(mf * mf)
    for c in range(mc * mc):
        xc, yc = (c % mc) * H, (c // mc) * H
        hat = np.clip(1 - np.abs(xf - xc) / H, 0, None) * np.clip(1 - np.abs(yf - yc) / H, 0, None)
        ref += uc[c] * hat
    assert np.allclose(O.prolongation(nc) @ uc, ref, rtol=0, atol=1e-15)


def test_restricted_fine_stiffness_is_the_coarse_stiffness_for_constant_coefficient():
    # Galerkin property of nested conforming spaces: with a constant coefficient (sigma = 0) the
    # 3x3 Gauss rule integrates the Q1 stiffness exactly, so P^T A_h P = A_H on interior nodes
    for nc in (2, 3, 5):
        fine = O.build_problem(2 * nc, 1, 0, sigma=0.0, mu=0.3)
        coarse = O.build_problem(nc, 1, 0, sigma=0.0, mu=0.3)
        Pm = O.prolongation(nc)
        galerkin = (Pm.T @ fine.A[0] @ Pm).toarray()
        inner = ~O.boundary_mask(nc)
        ref = coarse.A[0].toarray()[np.ix_(inner, inner)]
        assert np.allclose(galerkin[np.ix_(inner, inner)], ref, rtol=0, atol=1e-13)


def test_one_level_vcycle_is_the_direct_solve():
    levels = O.mg_levels(2, 2, 2, coarse=2, sigma=0.6, ell=0.8)
    data = O.mg_setup(levels)
    prob = levels[0]
    b = np.random.default_rng(4).normal(size=(prob.N, prob.P))
    b[prob.boundary] = 0.0
    u = O.mg_vcycle(levels, data, b)
    assert np.allclose(O.sg_matvec(prob, u), b, rtol=0, atol=1e-13 * np.abs(b).max())


@pytest.mark.parametrize("smoother,sigma", [("fs_gs", 0.5), ("fs_jacobi", 0.3), ("mean", 0.2)])
def test_vcycle_iteration_contracts_independently_of_the_mesh(smoother, sigma):
    # the V-cycle as a stationary iteration u <- u + V(F - K u): its error contraction per step
    # must stay well below one and not degrade as the mesh is refined (Table 1's trend).  The
    # mean-based smoother ignores the stochastic coupling, so it is checked at a smaller sigma.
    rates = []
    for n in (8, 16, 32):
        levels = O.mg_levels(n, 2, 2, sigma=sigma, ell=0.7)
        data = O.mg_setup(levels, smoother)
        prob = levels[-1]
        u = np.zeros_like(prob.F)
        ref = scipy.sparse.linalg.spsolve(
            scipy.sparse.csr_matrix(sum(scipy.sparse.kron(prob.G[k], prob.A[k])
                                        for k in range(prob.L))).tocsc(),
            prob.F.T.ravel()).reshape(prob.P, prob.N).T
        errs = []
        for _ in range(6):
            u = u + O.mg_vcycle(levels, data, prob.F - O.sg_matvec(prob, u), smoother)
            errs.append(np.linalg.norm(u - ref))
        rates.append((errs[-1] / errs[1]) ** 0.25)
    assert max(rates) < 0.5, rates
    assert rates[-1] < rates[0] + 0.1, rates


def test_mg_preconditioned_gmres_iterations_stay_flat_in_the_mesh():
    its = []
    for n in (8, 16, 32):
        levels = O.mg_levels(n, 2, 2, sigma=0.5, ell=0.7)
        data = O.mg_setup(levels, "fs_gs")
        prob = levels[-1]

        def apply_M(v, prob=prob, levels=levels, data=data):
            V = v.reshape(prob.N, prob.P)
            return O.mg_vcycle(levels, data, V).ravel()

        _, info = O.gmres(lambda v, prob=prob: O.sg_matvec(prob, v.reshape(prob.N, prob.P)).ravel(),
                          apply_M, prob.F, rtol=1e-10, restart=30)
        assert info["converged"]
        its.append(info["iters"])
    assert max(its) - min(its) <= 2, its
    assert max(its) <= 12, its


# ------------------------------------------------------------------ four-colour ILU(0) (reading R18)

def test_color4_order_separates_stencil_neighbours():
    for n in (2, 3, 6, 9):
        order = O.color4_order(n)
        m = n + 1
        assert sorted(order.tolist()) == list(range(m * m))
        x, y = order % m, order // m
        col = (x % 2) + 2 * (y % 2)
        assert np.all(np.diff(col) >= 0)               # colours in turn
        A = O.build_problem(n, 1, 0, sigma=0.0).A[0]
        c_of = np.empty(m * m, int)
        c_of[order] = col
        rows, cols = A.nonzero()
        off = rows != cols
        assert np.all(c_of[rows[off]] != c_of[cols[off]])  # no coupling inside a colour


def test_color4_ilu0_defining_property_and_solve():
    prob = O.build_problem(7, 2, 1, sigma=0.6, ell=0.8, a_min=0.02)
    A = prob.A[0]
    LU = O.ilu0(A, O.color4_order(7))
    Lo, Up, order = LU
    Ap = A[order][:, order].toarray()
    prod = (Lo @ Up).toarray()
    pat = Ap != 0
    assert np.allclose(prod[pat], Ap[pat], rtol=0, atol=1e-13)
    # L couples a node only to earlier colours: its strictly lower part has no entry inside a
    # colour block; the unit diagonal is implicit in the stored factor
    m = 8
    col = ((order % m) % 2) + 2 * ((order // m) % 2)
    Ls = scipy.sparse.tril(Lo, k=-1).tocoo()
    assert np.all(col[Ls.row] > col[Ls.col])
    # the solve inverts L U in the original ordering
    r = np.random.default_rng(2).normal(size=A.shape[0])
    z = O.ilu0_solve(LU, r)
    M = np.zeros_like(prod)
    M[np.ix_(order, order)] = prod
    assert np.allclose(M @ z, r, atol=1e-12)


def test_mg_with_color4_smoother_is_mesh_independent():
    its = []
    for n in (8, 16, 32):
        levels = O.mg_levels(n, 2, 2, sigma=0.5, ell=0.7)
        data = O.mg_setup(levels, "fs_gs", ordering="color4")
        prob = levels[-1]
        _, info = O.gmres(lambda v, prob=prob: O.sg_matvec(prob, v.reshape(prob.N, prob.P)).ravel(),
                          lambda v, prob=prob, levels=levels, data=data:
                          O.mg_vcycle(levels, data, v.reshape(prob.N, prob.P)).ravel(),
                          prob.F, rtol=1e-10, restart=30)
        assert info["converged"]
        its.append(info["iters"])
    assert max(its) - min(its) <= 3 and max(its) <= 16, its
