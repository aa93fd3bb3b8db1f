"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

No GPU. Each test ties one oracle function to something other than itself:
closed-form eigenpairs, Chebyshev polynomials, interpolation exactness, the
finite-element nesting property, the Woodbury identity with an exact inverse,
brute-force dense solves, and the m = 0 / m = 1 special cases.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from numpy.polynomial import chebyshev as npcheb

from oracle import discretization as disc
from oracle import multigrid as mg
from oracle import woodbury as wb
from oracle import ccg


# --------------------------------------------------------------------------
# P2: closed-form cosine eigenpairs of the grid operators
# --------------------------------------------------------------------------

@pytest.mark.parametrize("nx,ny,hx,hy", [(7, 5, 1 / 6, 1 / 4), (9, 9, 0.125, 0.125), (4, 11, 0.3, 0.07)])
def test_q1_generalized_eigenpairs(nx, ny, hx, hy):
    """(K + Ml) v = lam Ml v with v = cos(k pi i/(nx-1)) cos(l pi j/(ny-1)) and
    lam = mu_k nu_l + nu_k mu_l + 1, mu = (2 - 2 cos t)/h^2, nu = 1 - h^2 mu / 6."""
    K, _, Ml = disc.q1_assemble(nx, ny, hx, hy)
    i = np.arange(nx)
    j = np.arange(ny)
    for k in range(nx):
        for l in range(ny):
            tk, tl = k * np.pi / (nx - 1), l * np.pi / (ny - 1)
            v = np.outer(np.cos(tl * j), np.cos(tk * i)).ravel()
            mux, muy = (2 - 2 * np.cos(tk)) / hx ** 2, (2 - 2 * np.cos(tl)) / hy ** 2
            nux, nuy = 1 - hx ** 2 * mux / 6, 1 - hy ** 2 * muy / 6
            lam = mux * nuy + nux * muy + 1.0
            res = K @ v + Ml * v - lam * Ml * v
            assert np.linalg.norm(res) <= 1e-11 * lam * np.linalg.norm(Ml * v)


def test_q1_lumped_mass_values():
    """Row-sum lumping of the Q1 mass: h^2 inside, h^2/2 on edges, h^2/4 at corners."""
    n, h = 6, 0.2
    _, _, Ml = disc.q1_assemble(n, n, h, h)
    Ml = Ml.reshape(n, n)
    assert np.isclose(Ml[2, 3], h * h)
    assert np.isclose(Ml[0, 3], h * h / 2)
    assert np.isclose(Ml[0, 0], h * h / 4)
    assert np.isclose(Ml.sum(), 1.0)


@pytest.mark.parametrize("n,h", [((5, 4, 3), (0.2, 0.25, 1 / 3)), ((8, 8, 8), (0.125,) * 3)])
def test_fv_eigenpairs(n, h):
    """FV Neumann: v = prod cos(k_d pi (i_d + 1/2)/n_d), lam = sum T_d (2 - 2 cos(k_d pi/n_d)) + V."""
    K, M = disc.fv_assemble(*n, *h)
    T = (h[1] * h[2] / h[0], h[0] * h[2] / h[1], h[0] * h[1] / h[2])
    V = h[0] * h[1] * h[2]
    rng = np.random.default_rng(3)
    for _ in range(12):
        ks = [int(rng.integers(0, nd)) for nd in n]
        cx = np.cos(ks[0] * np.pi * (np.arange(n[0]) + 0.5) / n[0])
        cy = np.cos(ks[1] * np.pi * (np.arange(n[1]) + 0.5) / n[1])
        cz = np.cos(ks[2] * np.pi * (np.arange(n[2]) + 0.5) / n[2])
        v = (cz[:, None, None] * cy[None, :, None] * cx[None, None, :]).ravel()
        lam = sum(T[d] * (2 - 2 * np.cos(ks[d] * np.pi / n[d])) for d in range(3)) + V
        res = K @ v + M * v - lam * v
        assert np.linalg.norm(res) <= 1e-12 * max(lam, 1.0) * np.linalg.norm(v)


def test_operators_symmetric():
    for A in (disc.regularization_operator("q1", (9, 6), (0.1, 0.2)),
              disc.regularization_operator("fv", (6, 4, 5), (0.1, 0.2, 0.3))):
        assert abs(A - A.T).max() == 0.0


# --------------------------------------------------------------------------
# Chebyshev smoother: error polynomial in closed form
# --------------------------------------------------------------------------

@pytest.mark.parametrize("degree", [1, 2, 3, 4])
def test_chebyshev_error_polynomial(degree):
    """With D = I, the error of x_k is T_k((theta - mu)/delta) / T_k(theta/delta) times
    the initial error for each eigenvalue mu of A."""
    rng = np.random.default_rng(4)
    lam = 1.7
    mu = np.linspace(0.01, lam, 40)
    A = sp.diags(mu).tocsr()
    xs = rng.standard_normal(40)
    b = A @ xs
    x0 = rng.standard_normal(40)
    x = mg.chebyshev(A, np.ones(40), lam, b, x0, 30.0, degree=degree)
    lo, hi = lam / 30.0, lam
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    c = np.zeros(degree + 1)
    c[degree] = 1.0
    factor = npcheb.chebval((theta - mu) / delta, c) / npcheb.chebval(theta / delta, c)
    np.testing.assert_allclose(x - xs, factor * (x0 - xs), rtol=0, atol=1e-12)


# --------------------------------------------------------------------------
# Transfer operators
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [3, 4, 5, 8, 9, 64])
def test_q1_prolongation_reproduces_linears(n):
    P, nc = mg.q1_prolongation_1d(n)
    xf = np.arange(n, dtype=float)
    coarse = list(range(0, n, 2)) + ([n - 1] if (n - 1) % 2 else [])
    xc = np.array(coarse, dtype=float)
    for f in (lambda t: 1.0 + 0 * t, lambda t: 2.5 * t - 1.0):
        np.testing.assert_allclose(P @ f(xc), f(xf), atol=1e-13)
    assert nc == len(coarse)


@pytest.mark.parametrize("n", [4, 6, 16])
def test_fv_prolongation(n):
    """Cell-centred interpolation: constants everywhere, linears away from the boundary."""
    P, nc = mg.fv_prolongation_1d(n)
    xf = (np.arange(n) + 0.5) / n
    xc = (np.arange(nc) + 0.5) / nc
    np.testing.assert_allclose(P @ np.ones(nc), np.ones(n), atol=1e-15)
    lin = P @ (3.0 * xc - 1.0)
    np.testing.assert_allclose(lin[1:-1], (3.0 * xf - 1.0)[1:-1], atol=1e-13)
    assert mg.fv_prolongation_1d(n + 1)[0] is None


def _q1_assemble_tensor_mesh(x, y):
    """Q1 stiffness on a tensor mesh with vertex coordinates x, y (test helper)."""
    nx, ny = len(x), len(y)
    N = nx * ny
    K = np.zeros((N, N))
    for ey in range(ny - 1):
        for ex in range(nx - 1):
            Ke, _ = disc.q1_element_matrices(x[ex + 1] - x[ex], y[ey + 1] - y[ey])
            nodes = [(ey + a // 2) * nx + ex + a % 2 for a in range(4)]
            K[np.ix_(nodes, nodes)] += Ke
    return K


@pytest.mark.parametrize("nx,ny", [(8, 8), (9, 6), (10, 7)])
def test_q1_galerkin_is_coarse_fe_stiffness(nx, ny):
    """Nested Q1 spaces: P^T K P equals the Q1 stiffness assembled on the coarse
    (possibly non-uniform) mesh."""
    h = (1.0 / (nx - 1), 1.0 / (ny - 1))
    K, _, _ = disc.q1_assemble(nx, ny, *h)
    Px, ncx = mg.q1_prolongation_1d(nx)
    Py, ncy = mg.q1_prolongation_1d(ny)
    P = sp.kron(Py, Px).tocsr()
    coarse = lambda n: np.array(list(range(0, n, 2)) + ([n - 1] if (n - 1) % 2 else []), dtype=float)
    Kc = _q1_assemble_tensor_mesh(coarse(nx) * h[0], coarse(ny) * h[1])
    np.testing.assert_allclose((P.T @ K @ P).toarray(), Kc, atol=1e-12)


# --------------------------------------------------------------------------
# V-cycle: exact on a single level, symmetric positive definite, good
# --------------------------------------------------------------------------

def test_vcycle_single_level_is_exact_inverse():
    H = mg.build_hierarchy("fv", (8, 8, 8), (0.125,) * 3)
    assert len(H.levels) == 1
    A = H.levels[0].A.toarray()
    b = np.random.default_rng(5).standard_normal(512)
    np.testing.assert_allclose(mg.vcycle(H, b), np.linalg.solve(A, b), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("case", [("q1", (29, 23), (1 / 28, 1 / 22)), ("q1", (24, 24), (1 / 23,) * 2),
                                  ("fv", (16, 8, 12), (1 / 16, 1 / 8, 1 / 12))])
def test_vcycle_symmetric_positive(case):
    d, n, h = case
    H = mg.build_hierarchy(d, n, h)
    assert len(H.levels) >= 2
    B = mg.vcycle_matrix(H)
    assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
    A = H.levels[0].A.toarray()
    # spectrum of B A: positive; for Galerkin (Q1) levels it lies in (0, 1].
    ev = np.sort(np.linalg.eigvals(B @ A).real)
    assert ev[0] > 0.05
    if d == "q1":
        assert ev[-1] <= 1.0 + 1e-10
    else:
        assert ev[-1] < 2.0


def test_hierarchy_shapes():
    Hq = mg.build_hierarchy("q1", (64, 64), (1 / 63,) * 2)
    assert [lv.n for lv in Hq.levels] == [(64, 64), (33, 33), (17, 17)]
    Hf = mg.build_hierarchy("fv", (32, 16, 24), (1 / 32, 1 / 16, 1 / 24))
    assert [lv.n for lv in Hf.levels] == [(32, 16, 24), (16, 8, 12), (8, 4, 6)]


# --------------------------------------------------------------------------
# P1: Woodbury exactness with an exact Laplace inverse; P6: m = 0, m = 1
# --------------------------------------------------------------------------

def _tiny(disc_name="q1"):
    rng = np.random.default_rng(7)
    if disc_name == "q1":
        A = disc.regularization_operator("q1", (9, 7), (1 / 8, 1 / 6)).toarray()
    else:
        A = disc.regularization_operator("fv", (4, 5, 3), (0.25, 0.2, 1 / 3)).toarray()
    N = A.shape[0]
    J = rng.standard_normal((6, N)) / np.sqrt(N)
    b = rng.standard_normal(N)
    return A, J, b


@pytest.mark.parametrize("d", ["q1", "fv"])
@pytest.mark.parametrize("alpha", [1e-4, 1e-2, 1.0])
def test_woodbury_exact_inverse_is_direct_solve(d, alpha):
    A, J, b = _tiny(d)
    Aop = alpha * A + J.T @ J
    x_direct = np.linalg.solve(Aop, b)
    x_w = wb.woodbury_direct(A, J, alpha, b)
    assert np.linalg.norm(x_w - x_direct) <= 1e-11 * np.linalg.norm(x_direct)
    # PCG with the ideal preconditioner converges in one iteration
    Ainv = np.linalg.inv(A)
    P = wb.WoodburyPreconditioner(lambda v: Ainv @ v, J, alpha)
    x, it, rel = wb.pcg(lambda v: Aop @ v, P, b, 1e-10, 50)
    assert it == 1 and rel <= 1e-10


def test_woodbury_m0_is_scaled_laplace_preconditioner():
    A, J, b = _tiny("q1")
    H = mg.build_hierarchy("q1", (9, 7), (1 / 8, 1 / 6))
    P = wb.WoodburyPreconditioner(lambda v: mg.vcycle(H, v), J[:0], 0.3)
    np.testing.assert_allclose(P(b), mg.vcycle(H, b) / 0.3, rtol=1e-14)


def test_woodbury_m1_sherman_morrison():
    """m = 1: (alpha A + j j^T)^-1 r = y - y_j (j.y) / (1 + j.y_j), y = (alpha A)^-1 r."""
    A, J, b = _tiny("fv")
    j = J[0]
    alpha = 0.05
    Ainv = np.linalg.inv(A)
    y = Ainv @ b / alpha
    yj = Ainv @ j / alpha
    expect = y - yj * (j @ y) / (1.0 + j @ yj)
    P = wb.WoodburyPreconditioner(lambda v: Ainv @ v, J[:1], alpha)
    np.testing.assert_allclose(P(b), expect, rtol=1e-12)


def test_woodbury_preconditioner_symmetric_spd():
    A, J, b = _tiny("q1")
    H = mg.build_hierarchy("q1", (9, 7), (1 / 8, 1 / 6))
    P = wb.WoodburyPreconditioner(lambda v: mg.vcycle(H, v), J, 1e-3)
    N = A.shape[0]
    Pm = np.stack([P(np.eye(N)[k]) for k in range(N)], axis=1)
    assert np.abs(Pm - Pm.T).max() <= 1e-10 * np.abs(Pm).max()
    assert np.linalg.eigvalsh(0.5 * (Pm + Pm.T)).min() > 0


# --------------------------------------------------------------------------
# P4: brute force; P7/P8: iteration counts
# --------------------------------------------------------------------------

def test_c1_pcg_matches_dense_solve():
    from paper_2209_02815_gb300.inputs import small_c1_problem
    pr = small_c1_problem()
    A = disc.regularization_operator("q1", (pr.nx, pr.ny), pr.h)
    Aop = pr.alpha * A.toarray() + pr.J.T @ pr.J
    x_ref = np.linalg.solve(Aop, pr.b)
    H = mg.build_hierarchy("q1", (pr.nx, pr.ny), pr.h)
    P = wb.WoodburyPreconditioner(lambda v: mg.vcycle(H, v), pr.J, pr.alpha)
    x, it, rel = wb.pcg(lambda v: wb.apply_operator(A, pr.alpha, pr.J, v), P, pr.b, 1e-12, 200)
    assert rel <= 1e-12
    assert np.linalg.norm(x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    assert it <= 20


def test_c_oracle_cg_matches_dense_solve():
    A = disc.regularization_operator("fv", (6, 5, 4), (1 / 6, 1 / 5, 1 / 4))
    rng = np.random.default_rng(11)
    N = A.shape[0]
    J = rng.standard_normal((5, N)) / np.sqrt(N)
    b = rng.standard_normal(N)
    alpha = 0.1
    op = ccg.CsrOperator(A, alpha, J)
    p = rng.standard_normal(N)
    np.testing.assert_allclose(op.apply(p), alpha * (A @ p) + J.T @ (J @ p), rtol=1e-13, atol=1e-14)
    x, it, rel = op.cg(b, 1e-13, 10000)
    x_ref = np.linalg.solve(alpha * A.toarray() + J.T @ J, b)
    assert rel <= 1e-13
    assert np.linalg.norm(x - x_ref) <= 1e-10 * np.linalg.norm(x_ref)


@pytest.mark.parametrize("alpha", [1e-4, 1e-1])
def test_woodbury_pcg_iterations_bounded_by_mg_pcg(alpha):
    """kappa(P^-1 A) <= kappa(L-hat^-1 (K+M)): the Woodbury-PCG count stays near the
    MG-PCG count for K + M alone, for any alpha and m."""
    from paper_2209_02815_gb300.inputs import gaussian_problem
    pr = gaussian_problem(33, 33, 24, alpha)
    A = disc.regularization_operator("q1", (pr.nx, pr.ny), pr.h)
    H = mg.build_hierarchy("q1", (pr.nx, pr.ny), pr.h)
    V = lambda v: mg.vcycle(H, v)
    _, it_mg, _ = wb.pcg(lambda v: A @ v, V, pr.b, 1e-8, 200)
    P = wb.WoodburyPreconditioner(V, pr.J, alpha)
    _, it_w, rel = wb.pcg(lambda v: wb.apply_operator(A, alpha, pr.J, v), P, pr.b, 1e-8, 200)
    assert rel <= 1e-8
    assert it_w <= it_mg + 2


@pytest.mark.parametrize("d", ["q1", "fv"])
def test_laplace_only_exact_inverse_terminates_within_m_plus_1(d):
    """The preconditioner without the capacitance matrix, alpha^-1 A^-1 (the paper's
    comparison variant): P^-1 (alpha A + J^T J) = I + alpha^-1 A^-1 J^T J is the identity
    plus a rank-m term, so it has at most m + 1 distinct eigenvalues and CG stops within
    m + 1 iterations, where the Woodbury preconditioner needs one. (The bound is one of
    exact arithmetic; with alpha = 1 the spectrum is narrow enough that rounding does not
    delay it, while at alpha = 1e-3 the oracle takes m + 2.)"""
    A, J, b = _tiny(d)
    alpha = 1.0
    Aop = alpha * A + J.T @ J
    Ainv = np.linalg.inv(A)
    x, it, rel = wb.pcg(lambda v: Aop @ v, lambda v: Ainv @ v / alpha, b, 1e-10, 50)
    assert 1 < it <= J.shape[0] + 1 and rel <= 1e-10, it


# --------------------------------------------------------------------------
# Gauss-Newton right-hand side (Eq. 2.9 scaled by beta, with the mass term)
# --------------------------------------------------------------------------

def _gn_rhs_case(disc_kind):
    if disc_kind == "q1":
        n, h = (7, 6), (1 / 6, 1 / 5)
    else:
        n, h = (5, 4, 3), (0.2, 0.25, 1 / 3)
    A = disc.regularization_operator(disc_kind, n, h)
    N = A.shape[0]
    rng = np.random.default_rng(31)
    m = 5
    J = rng.standard_normal((m, N))
    dm = rng.standard_normal(N)
    d = rng.standard_normal(m)
    return A, J, dm, d, 0.37


@pytest.mark.parametrize("disc_kind", ["q1", "fv"])
def test_gn_rhs_is_minus_the_gradient_of_the_linearized_objective(disc_kind):
    """b is minus the gradient at dm' = 0 of the quadratic model
    Q(dm') = 1/2 ||d + J dm'||^2 + alpha/2 (dm + dm')^T (K + M) (dm + dm'):
    central differences of Q (exact for a quadratic up to rounding) along random
    directions v give -b . v. A sign slip or a dropped term in either part fails."""
    A, J, dm, d, alpha = _gn_rhs_case(disc_kind)
    b = wb.gn_rhs(A, alpha, dm, J, d)

    def Q(step):
        r = d + J @ step
        u = dm + step
        return 0.5 * float(r @ r) + 0.5 * alpha * float(u @ (A @ u))

    rng = np.random.default_rng(32)
    for _ in range(6):
        v = rng.standard_normal(dm.size)
        eps = 1e-3
        fd = (Q(eps * v) - Q(-eps * v)) / (2 * eps)
        assert abs(fd + float(b @ v)) <= 1e-9 * (abs(fd) + np.linalg.norm(b) * np.linalg.norm(v))


@pytest.mark.parametrize("disc_kind", ["q1", "fv"])
def test_gn_rhs_from_the_stacked_least_squares_problem(disc_kind):
    """With K + M = R^T R (numpy Cholesky), the linearized step solves the stacked
    least-squares problem min ||[J; sqrt(alpha) R] s - y||, y = -[d; sqrt(alpha) R dm];
    its normal-equation right-hand side [J; sqrt(alpha) R]^T y is b."""
    A, J, dm, d, alpha = _gn_rhs_case(disc_kind)
    R = np.linalg.cholesky(A.toarray()).T
    S = np.vstack([J, np.sqrt(alpha) * R])
    y = -np.concatenate([d, np.sqrt(alpha) * (R @ dm)])
    want = S.T @ y
    b = wb.gn_rhs(A, alpha, dm, J, d)
    assert np.abs(b - want).max() <= 1e-12 * np.abs(want).max()
    # and the step it gives is the least-squares minimizer (QR)
    step = np.linalg.solve(S.T @ S, b)
    ls = np.linalg.lstsq(S, y, rcond=None)[0]
    assert np.abs(step - ls).max() <= 1e-9 * np.abs(ls).max()
