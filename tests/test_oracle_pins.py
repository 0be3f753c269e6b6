"""Pins for the FP64 oracle: closed forms, brute force and textbook special cases.

Each test checks the oracle against something other than itself: the discrete
Laplacian symbol (Eq. discrete_symbol), hand-assembled sparse / Kronecker
matrices, a separately written textbook shifted-Laplacian multigrid
(Appendix A.3), exact linear algebra on tiny grids, and literal values.
"""
import math

import numpy as np
import pytest
import scipy.ndimage
import scipy.sparse as sp

from oracle import mcmg_oracle as O
from paper_2606_30495_b300 import inputs as I


def rng(seed=0):
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------
# problem definition
# --------------------------------------------------------------------------

def test_sponge_profile_literal_values():
    # N = 10, width 3, gamma_max 2: depths 3,2,1,0,0,0,0,1,2,3 along an axis.
    g = O.sponge_gamma((10,), 3, 2.0)
    want = np.array([2.0, 2 * 4 / 9, 2 / 9, 0, 0, 0, 0, 2 / 9, 2 * 4 / 9, 2.0])
    np.testing.assert_allclose(g, want, rtol=0, atol=1e-15)
    g2 = O.sponge_gamma((10, 10), 3, 2.0)
    assert g2[0, 4] == 2.0 and g2[5, 5] == 0.0
    assert abs(g2[1, 2] - 2 * 4 / 9) < 1e-15      # max over axes, not sum
    assert O.sponge_gamma((8, 8), 0, 1.0).max() == 0.0


def test_wavenumber_coef_literal():
    c = np.full((8, 8), 2.0)
    q = O.wavenumber_coef(c, omega=16.0, width=2, gamma_max=1.0)
    # k h = omega h / c = 16 / 8 / 2 = 1 ; corner gamma = 1 -> q = 1 - i
    assert abs(q[4, 4] - 1.0) < 1e-15
    assert abs(q[0, 0] - (1.0 - 1.0j)) < 1e-15


@pytest.mark.parametrize("shape,modes", [((12, 9), [(1, 1), (3, 5), (8, 2)]),
                                         ((6, 5, 7), [(1, 1, 1), (2, 4, 3)])])
def test_dirichlet_sine_modes_are_eigenvectors(shape, modes):
    """Discrete Laplacian symbol (Eq. discrete_symbol): with zero Dirichlet
    truncation, prod_a sin(pi p_a (i_a+1)/(N_a+1)) is an eigenvector of h^2 A
    with eigenvalue sum_a 4 sin^2(pi p_a / (2 (N_a+1))) - (k h)^2."""
    kh2 = 0.37
    q = np.full(shape, kh2, dtype=np.complex128)
    for p in modes:
        u = np.ones(shape)
        lam = -kh2
        for ax, (n, pa) in enumerate(zip(shape, p)):
            i = np.arange(n)
            sh = [1] * len(shape)
            sh[ax] = n
            u = u * np.sin(math.pi * pa * (i + 1) / (n + 1)).reshape(sh)
            lam += 4 * math.sin(math.pi * pa / (2 * (n + 1))) ** 2
        Au = O.apply_A(q, u.astype(np.complex128))
        assert np.max(np.abs(Au - lam * u)) < 1e-13


def test_plane_wave_on_discrete_dispersion_shell():
    """A plane wave exp(i xi.x) with 4 sin^2(xi_x/2) + 4 sin^2(xi_y/2) = (kh)^2
    solves the homogeneous discrete equation at every interior node."""
    kh = 2 * math.pi / 10
    xi_x = 0.3
    s = (kh ** 2 - 4 * math.sin(xi_x / 2) ** 2) / 4
    xi_y = 2 * math.asin(math.sqrt(s))
    n = 16
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    u = np.exp(1j * (xi_x * xx + xi_y * yy))
    q = np.full((n, n), kh ** 2, dtype=np.complex128)
    Au = O.apply_A(q, u)
    assert np.max(np.abs(Au[1:-1, 1:-1])) < 1e-13
    assert np.max(np.abs(Au[0])) > 1e-3        # the truncated boundary is not exact


def _laplacian_sparse(shape):
    """-Delta_h h^2 with zero Dirichlet truncation, by Kronecker sums of 1D tridiagonals."""
    mats = [sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1])
            for n in shape]
    total = None
    for ax in range(len(shape)):
        term = None
        for bx in range(len(shape)):
            m = mats[bx] if bx == ax else sp.identity(shape[bx])
            term = m if term is None else sp.kron(term, m)
        total = term if total is None else total + term
    return total.toarray()


@pytest.mark.parametrize("shape", [(7, 6), (4, 5, 3)])
def test_operator_matches_sparse_assembly(shape):
    q = I.complex_normal(shape, rng(1))
    Adense = O.dense_matrix(lambda u: O.apply_A(q, u), shape)
    want = _laplacian_sparse(shape) - np.diag(q.reshape(-1))
    assert np.max(np.abs(Adense - want)) < 1e-14


# --------------------------------------------------------------------------
# multi-channel pieces against Kronecker (dense) forms
# --------------------------------------------------------------------------

def _shift_matrix(shape, off):
    """S with (S u)[p] = u[p + off], zero outside, built from 1D shifted identities."""
    m = None
    for n, o in zip(shape, off):
        s1 = np.eye(n, k=o)
        m = s1 if m is None else np.kron(m, s1)
    return m


def _select_matrix(shape, off):
    """Sel with (Sel u)[J] = u[2J + off] over a coarse grid of half the size."""
    m = None
    for n, o in zip(shape, off):
        s1 = np.zeros((n // 2, n))
        for J in range(n // 2):
            i = 2 * J + o
            if 0 <= i < n:
                s1[J, i] = 1.0
        m = s1 if m is None else np.kron(m, s1)
    return m


@pytest.mark.parametrize("shape,C", [((6, 4), 3), ((4, 4, 2), 2)])
def test_neural_operator_and_smoother_kronecker(shape, C):
    d = len(shape)
    g = rng(2)
    T = 2 * d + 1
    lv = dict(W=I.complex_normal((T, C, C), g), KA=I.complex_normal((C, C), g),
              KS=I.complex_normal((C, C), g), Wsm=I.complex_normal((3, C, C), g))
    a = I.complex_normal(shape + (C,), g)
    s = I.complex_normal(shape + (C,), g)
    x = I.complex_normal(shape + (C,), g)
    n = int(np.prod(shape))
    Ad = sum(np.kron(_shift_matrix(shape, off), lv["W"][t])
             for t, off in enumerate(O.stencil_offsets(d)))
    Ad = Ad + np.diag(a.reshape(-1)) @ np.kron(np.eye(n), lv["KA"])
    got = O.op_A(lv, a, x).reshape(-1)
    assert np.max(np.abs(got - Ad @ x.reshape(-1))) < 1e-12
    Sd = np.kron(np.eye(n), lv["Wsm"][2]) @ np.diag(s.reshape(-1)) @ np.kron(np.eye(n), lv["KS"])
    got = O.op_S(lv, s, 2, x).reshape(-1)
    assert np.max(np.abs(got - Sd @ x.reshape(-1))) < 1e-12


def test_stencil_tap_order():
    """Tap 1 reads the -x neighbour, tap 3 the -y neighbour (x fastest)."""
    x = np.zeros((4, 4, 1), dtype=np.complex128)
    x[2, 1, 0] = 1.0
    W = np.zeros((5, 1, 1), dtype=np.complex128)
    W[1] = 1.0
    y = O.stencil_conv(W, x)
    assert y[2, 2, 0] == 1.0 and abs(y).sum() == 1.0
    W[:] = 0
    W[3] = 1.0
    y = O.stencil_conv(W, x)
    assert y[3, 1, 0] == 1.0 and abs(y).sum() == 1.0


@pytest.mark.parametrize("shape,C,Cn", [((6, 8), 2, 3), ((4, 4, 6), 2, 2)])
def test_transfer_kronecker_and_transpose_identity(shape, C, Cn):
    d = len(shape)
    g = rng(3)
    T3 = 3 ** d
    R = I.complex_normal((T3, Cn, C), g)
    x = I.complex_normal(shape + (C,), g)
    Rd = sum(np.kron(_select_matrix(shape, off), R[t]) for t, off in enumerate(O.transfer_offsets(d)))
    assert np.max(np.abs(O.restrict(R, x).reshape(-1) - Rd @ x.reshape(-1))) < 1e-12
    # transpose identity <R x, y> = <x, P y> with P[o] = R[o]^T (bilinear pairing)
    P = np.transpose(R, (0, 2, 1))
    cshape = tuple(m // 2 for m in shape)
    y = I.complex_normal(cshape + (Cn,), g)
    lhs = np.sum(O.restrict(R, x) * y)
    rhs = np.sum(x * O.prolong(P, y, shape))
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))
    Pd = sum(np.kron(_select_matrix(shape, off).T, P[t]) for t, off in enumerate(O.transfer_offsets(d)))
    assert np.max(np.abs(O.prolong(P, y, shape).reshape(-1) - Pd @ y.reshape(-1))) < 1e-12


def test_full_weighting_and_bilinear_reproduce_linear_functions():
    n = 16
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    lin = (0.3 + 0.7 * xx - 1.1 * yy)[..., None].astype(np.complex128)
    fw = np.zeros((9, 1, 1), dtype=np.complex128)
    fw[:, 0, 0] = np.array([1, 2, 1, 2, 4, 2, 1, 2, 1]) / 16
    r = O.restrict(fw, lin)[..., 0]
    JJ, II = np.meshgrid(np.arange(n // 2), np.arange(n // 2), indexing="ij")
    want = 0.3 + 0.7 * (2 * II) - 1.1 * (2 * JJ)
    assert np.max(np.abs(r[1:, 1:] - want[1:, 1:])) < 1e-13
    cl = (0.3 + 0.7 * II - 1.1 * JJ)[..., None].astype(np.complex128)
    p = O.prolong(4 * fw, cl, (n, n))[..., 0]
    want_f = 0.3 + 0.7 * (xx / 2) - 1.1 * (yy / 2)
    assert np.max(np.abs(p[:-1, :-1] - want_f[:-1, :-1])) < 1e-13


# --------------------------------------------------------------------------
# setup layers
# --------------------------------------------------------------------------

def test_gelu_literal_values():
    # Phi(1) = 0.8413447460685429 (standard normal CDF)
    v = O.gelu(np.array([0.0, 1.0, -1.0, 3.0]))
    np.testing.assert_allclose(v, [0.0, 0.8413447460685429, -0.15865525393145707,
                                   3 * 0.9986501019683699], rtol=1e-15, atol=1e-16)


@pytest.mark.parametrize("shape", [(9, 8), (5, 6, 4)])
def test_conv3_matches_ndimage_correlate(shape):
    g = rng(4)
    d = len(shape)
    x = g.standard_normal(shape)
    k = g.standard_normal((3,) * d)
    w = k.reshape(1, 1, -1)
    got = O.conv3(w, np.array([0.25]), x[..., None])[..., 0]
    want = scipy.ndimage.correlate(x, k, mode="constant", cval=0.0) + 0.25
    assert np.max(np.abs(got - want)) < 1e-13
    got2 = O.conv3(w, np.array([0.0]), x[..., None], stride=2)[..., 0]
    want2 = scipy.ndimage.correlate(x, k, mode="constant")[tuple(slice(0, None, 2) for _ in shape)]
    want2 = want2[tuple(slice(0, m // 2) for m in shape)]
    assert np.max(np.abs(got2 - want2)) < 1e-13


def test_setup_classical_branch_literal():
    """Degenerate weights: a_1 = -beta q, s_1 = 1/(4 + a_1), a_2 = full weighting of a_1."""
    n = 16
    c = I.grf((n, n), 4.0, 1.0, 3.0, rng(5))
    q = O.wavenumber_coef(c, 30.0, 3, 1.0)
    w = I.make_weights(2, [1, 1, 1], [2, 2, 2], [2, 2, 0], mode="degenerate", seed=0)
    f = O.setup(q, w)
    a1, s1 = f[0][0][..., 0], f[0][1][..., 0]
    beta = complex(*w["sl_shift"])
    assert np.max(np.abs(a1 + beta * q)) < 1e-15
    assert np.max(np.abs(s1 - 1 / (4 - beta * q))) < 1e-15
    a2 = f[1][0][..., 0]
    J, K = 3, 5   # interior coarse node (y, x) <-> fine (6, 10)
    fy, fx = 2 * J, 2 * K
    blk = a1[fy - 1:fy + 2, fx - 1:fx + 2]
    want = (blk * np.array([[1, 2, 1], [2, 4, 2], [1, 2, 1]]) / 16).sum()
    assert abs(a2[J, K] - want) < 1e-14
    s2 = f[1][1][..., 0]
    assert abs(s2[J, K] - 1 / (1.0 + a2[J, K])) < 1e-14


# --------------------------------------------------------------------------
# V-cycle
# --------------------------------------------------------------------------

def _textbook_slmg(q, levels, r, beta):
    """Classical complex-shifted-Laplacian multigrid V-cycle, written out directly.

    M = -Delta_h - beta k^2 (Eq. csl_shift) on every level (fine h^2 units,
    so the Laplacian part of level l carries 1/4^(l-1)); weighted Jacobi 0.66 on
    diag(M), 2 pre + 2 post steps, 2 steps on the coarsest grid, full-weighting
    restriction, bilinear interpolation, coarse k^2 by full weighting.
    """
    def lap(u):
        p = np.pad(u, 1)
        return 4 * u - p[:-2, 1:-1] - p[2:, 1:-1] - p[1:-1, :-2] - p[1:-1, 2:]

    def fw(u):
        p = np.pad(u, 1)
        n0, n1 = u.shape[0] // 2, u.shape[1] // 2
        out = np.zeros((n0, n1), dtype=complex)
        for J in range(n0):
            for K in range(n1):
                y, x = 2 * J + 1, 2 * K + 1
                out[J, K] = (4 * p[y, x] + 2 * (p[y - 1, x] + p[y + 1, x] + p[y, x - 1] + p[y, x + 1])
                             + p[y - 1, x - 1] + p[y - 1, x + 1] + p[y + 1, x - 1] + p[y + 1, x + 1]) / 16
        return out

    def interp(ec, shape):
        e = np.zeros(shape, dtype=complex)
        n0, n1 = ec.shape
        pc = np.pad(ec, ((0, 1), (0, 1)))
        for y in range(shape[0]):
            for x in range(shape[1]):
                J, K = y // 2, x // 2
                if y % 2 == 0 and x % 2 == 0:
                    e[y, x] = pc[J, K]
                elif y % 2 == 0:
                    e[y, x] = 0.5 * (pc[J, K] + pc[J, K + 1])
                elif x % 2 == 0:
                    e[y, x] = 0.5 * (pc[J, K] + pc[J + 1, K])
                else:
                    e[y, x] = 0.25 * (pc[J, K] + pc[J, K + 1] + pc[J + 1, K] + pc[J + 1, K + 1])
        return e

    qs = [q]
    for _ in range(levels - 1):
        qs.append(fw(qs[-1]))

    def M(l, u):
        return lap(u) / 4 ** l - beta * qs[l] * u

    def jacobi(l, u, f, steps):
        dg = 4 / 4 ** l - beta * qs[l]
        for _ in range(steps):
            u = u + 0.66 * (f - M(l, u)) / dg
        return u

    def cycle(l, f):
        u = jacobi(l, np.zeros_like(f), f, 2)
        if l == levels - 1:
            return u
        rc = fw(f - M(l, u))
        u = u + interp(cycle(l + 1, rc), u.shape)
        return jacobi(l, u, f, 2)

    return cycle(0, r)


def test_degenerate_mcmg_equals_textbook_shifted_laplacian_mg():
    n = 16
    c = I.grf((n, n), 4.0, 1.0, 2.0, rng(6))
    q = O.wavenumber_coef(c, 40.0, 3, 1.0)
    w = I.make_weights(2, [1, 1, 1], [2, 2, 2], [2, 2, 0], mode="degenerate", seed=0)
    feats = O.setup(q, w)
    r = I.complex_normal((n, n), rng(7))
    got = O.vcycle(w, feats, r)
    want = _textbook_slmg(q, 3, r, complex(*w["sl_shift"]))
    assert np.max(np.abs(got - want)) < 1e-13 * np.max(np.abs(want))
    w2 = dict(w, sl_shift=(1.0, 1.0))        # the shift as printed in Eq. csl_shift
    got2 = O.vcycle(w2, O.setup(q, w2), r)
    want2 = _textbook_slmg(q, 3, r, 1.0 + 1.0j)
    assert np.max(np.abs(got2 - want2)) < 1e-13 * np.max(np.abs(want2))


def _small_model(mode, seed=0, shape=(8, 8), channels=(2, 3), pre=None, post=None):
    d = len(shape)
    L = len(channels)
    p0, p1 = I.nu_schedule(L)
    pre = p0 if pre is None else pre
    post = p1 if post is None else post
    w = I.make_weights(d, list(channels), pre, post, mode=mode, seed=seed)
    c = I.grf(shape, 3.0, 1.0, 2.0, rng(seed + 11))
    q = O.wavenumber_coef(c, 2.0 * shape[0], 2, 1.0)
    return w, q, O.setup(q, w)


@pytest.mark.parametrize("mode,shape,channels", [("random", (8, 8), (2, 3)),
                                                 ("structured", (16, 8), (3, 2, 4)),
                                                 ("random", (4, 4, 4), (2, 2))])
def test_vcycle_linearity(mode, shape, channels):
    """V(alpha r1 + beta r2) = alpha V(r1) + beta V(r2) for fixed medium (Section 3.2)."""
    w, q, feats = _small_model(mode, shape=shape, channels=channels)
    g = rng(8)
    r1, r2 = I.complex_normal(shape, g), I.complex_normal(shape, g)
    al, be = 0.3 - 1.2j, -0.7 + 0.4j
    lhs = O.vcycle(w, feats, al * r1 + be * r2)
    rhs = al * O.vcycle(w, feats, r1) + be * O.vcycle(w, feats, r2)
    assert np.linalg.norm(lhs - rhs) <= 1e-13 * np.linalg.norm(rhs)


def test_vcycle_step_indexing_special_cases():
    """Zero post-smoother weights == no post-smoothing; zero pre-smoother weights
    leave e_l = 0 after pre-smoothing, so the result equals a cycle with nu1 = 0.
    This pins that post step i uses S^(nu1 + i) (Algorithm 2)."""
    w, q, feats = _small_model("random", shape=(8, 8), channels=(2, 2), pre=[1, 2], post=[2, 0])
    r = I.complex_normal((8, 8), rng(9))
    wz = {**w, "lvl": [dict(lv) for lv in w["lvl"]]}
    wz["lvl"][0]["Wsm"] = w["lvl"][0]["Wsm"].copy()
    wz["lvl"][0]["Wsm"][1:] = 0.0
    ref = {**w, "lvl": [dict(lv) for lv in w["lvl"]], "nu_post": [0, 0]}
    assert np.max(np.abs(O.vcycle(wz, feats, r) - O.vcycle(ref, feats, r))) < 1e-14
    wp = {**w, "lvl": [dict(lv) for lv in w["lvl"]]}
    wp["lvl"][0]["Wsm"] = w["lvl"][0]["Wsm"].copy()
    wp["lvl"][0]["Wsm"][:1] = 0.0
    nopre = {**w, "lvl": [dict(lv) for lv in w["lvl"]], "nu_pre": [0, 2]}
    nopre["lvl"][0]["Wsm"] = w["lvl"][0]["Wsm"][1:]
    assert np.max(np.abs(O.vcycle(wp, feats, r) - O.vcycle(nopre, feats, r))) < 1e-14
    assert np.max(np.abs(O.vcycle(wp, feats, r) - O.vcycle(w, feats, r))) > 1e-6


# --------------------------------------------------------------------------
# outer iterations
# --------------------------------------------------------------------------

def _tiny_problem(n=12, seed=10):
    c = I.grf((n, n), 3.0, 1.0, 2.0, rng(seed))
    q = O.wavenumber_coef(c, 0.6 * n, 3, 1.0)
    return q, (lambda u: O.apply_A(q, u))


def test_fgmres_matches_dense_direct_solve():
    n = 12
    q, A = _tiny_problem(n)
    w = I.make_weights(2, [2, 3], *I.nu_schedule(2), mode="structured", seed=1)
    feats = O.setup(q, w)
    f = I.point_source((n, n))
    u, info = O.fgmres(A, lambda v: O.vcycle(w, feats, v), f, m=8, tol=1e-11)
    Ad = O.dense_matrix(A, (n, n))
    ud = np.linalg.solve(Ad, f.reshape(-1)).reshape(n, n)
    assert info["converged"] and info["rel_residual"] <= 1e-11
    assert np.linalg.norm(u - ud) <= 1e-8 * np.linalg.norm(ud)
    assert info["restarts"] >= 1


def test_fgmres_exact_preconditioner_converges_in_one_step():
    n = 8
    q, A = _tiny_problem(n, seed=12)
    Ad = O.dense_matrix(A, (n, n))
    Ainv = np.linalg.inv(Ad)
    f = I.complex_normal((n, n), rng(13))
    u, info = O.fgmres(A, lambda v: (Ainv @ v.reshape(-1)).reshape(n, n), f, m=5, tol=1e-10)
    assert info["iters"] == 1 and info["converged"]
    u, info = O.stationary_solve(A, lambda v: (Ainv @ v.reshape(-1)).reshape(n, n), f, tol=1e-10)
    assert info["iters"] == 1


def test_fgmres_identity_preconditioner_is_minimal_residual():
    """With M = I and no restart, the implicit residual after j steps equals
    min over the Krylov space K_j(A, f) of ||f - A y|| (brute-force least squares)."""
    n = 6
    q, A = _tiny_problem(n, seed=14)
    Ad = O.dense_matrix(A, (n, n))
    f = I.complex_normal((n, n), rng(15)).reshape(-1)
    fnorm = np.linalg.norm(f)
    _, info = O.fgmres(lambda v: Ad @ v, lambda v: v, f, m=6, tol=1e-30, max_iters=6)
    hist = info["history"][1:7]
    K = [f]
    for j in range(1, 7):
        Kj = np.stack(K, axis=1)
        y, *_ = np.linalg.lstsq(Ad @ Kj, f, rcond=None)
        best = np.linalg.norm(f - Ad @ Kj @ y) / fnorm
        assert abs(hist[j - 1] - best) <= 1e-9 * max(best, 1e-12)
        K.append(Ad @ K[-1])


def test_fgmres_restarted_counts_iterations_and_converges():
    n = 12
    q, A = _tiny_problem(n, seed=16)
    w = I.make_weights(2, [1, 1], [2, 2], [2, 0], mode="degenerate", seed=0)
    feats = O.setup(q, w)
    f = I.point_source((n, n))
    _, info = O.fgmres(A, lambda v: O.vcycle(w, feats, v), f, m=3, tol=1e-8)
    assert info["converged"] and info["restarts"] >= 2
    assert info["iters"] >= 3 * (info["restarts"] - 1)


# ---------------------------------------------------------------------------
# Coarse-basis response (Eq. coarse_basis)
# ---------------------------------------------------------------------------

def _tent(shape, centre, half):
    """Tensor-product hat of half-width `half` (the bilinear / trilinear
    interpolant of a unit spike on a grid `half` times coarser)."""
    out = np.ones(shape)
    for ax, (n, c) in enumerate(zip(shape, centre)):
        t = np.clip(1.0 - np.abs(np.arange(n) - c) / half, 0.0, None)
        out = out * t.reshape([-1 if a == ax else 1 for a in range(len(shape))])
    return out


@pytest.mark.parametrize("shape,levels,level,index", [
    ((32, 32), 3, 2, (4, 3)),
    ((32, 32), 3, 1, (5, 9)),
    ((16, 16, 16), 2, 1, (3, 4, 2)),
])
def test_coarse_basis_of_classical_multigrid_is_the_tent(shape, levels, level, index):
    """With the classical one-channel weights every prolongation is bilinear
    (trilinear) interpolation and g_proj the identity, so the response of a
    spike at coarse node J of level l is the hat of half-width 2^l centred at
    2^l J (interior J, so the zero boundary does not clip it)."""
    d = len(shape)
    pre, post = I.nu_schedule(levels, degenerate=True)
    w = I.make_weights(d, [1] * levels, pre, post, mode="degenerate", seed=0)
    got = O.coarse_basis(w, level, index, 0, shape)
    want = _tent(shape, [i << level for i in index], float(1 << level))
    assert np.max(np.abs(got - want)) < 1e-14


def test_coarse_basis_applies_g_proj_last():
    """g_proj is applied once, last: scaling it scales the response by the
    same complex factor."""
    shape, levels = (16, 16), 2
    pre, post = I.nu_schedule(levels, degenerate=True)
    w = I.make_weights(2, [1] * levels, pre, post, mode="degenerate", seed=0)
    base = O.coarse_basis(w, 1, (3, 4), 0, shape)
    w["proj"] = w["proj"] * (2.5 - 1.0j)
    assert np.max(np.abs(O.coarse_basis(w, 1, (3, 4), 0, shape) - (2.5 - 1.0j) * base)) < 1e-14


# ---------------------------------------------------------------------------
# Born+McMg: discrete Green operator and the Born-series iteration
# ---------------------------------------------------------------------------

def _periodic_background(q0, x):
    """(-Delta_h - q0) x on the periodic grid, written with np.roll (no FFT)."""
    out = 2 * x.ndim * x - q0 * x
    for ax in range(x.ndim):
        out = out - np.roll(x, 1, axis=ax) - np.roll(x, -1, axis=ax)
    return out


@pytest.mark.parametrize("shape", [(12, 10), (6, 8, 5)])
def test_green_operator_inverts_the_periodic_background(shape):
    g = np.random.Generator(np.random.PCG64(70))
    c = 1.0 + 2.0 * g.random(shape)
    q = O.wavenumber_coef(c, 9.0, 2, 1.0)
    q0 = O.born_background(q)
    assert q0.imag < 0 and np.max(np.abs(q - q0.real)) <= -q0.imag + 1e-15
    x = I.complex_normal(shape, g)
    y = O.apply_G(q0, _periodic_background(q0, x))
    assert np.linalg.norm(y - x) <= 1e-12 * np.linalg.norm(x)


def test_green_operator_on_a_plane_wave():
    """A periodic plane wave is an eigenvector of the five-point Laplacian with
    eigenvalue sum_a (2 - 2 cos(2 pi m_a / N_a)): G divides it by that minus q0."""
    shape, m = (16, 12), (3, 5)
    yy, xx = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), indexing="ij")
    e = np.exp(2j * np.pi * (m[0] * yy / shape[0] + m[1] * xx / shape[1]))
    lam = sum(2.0 - 2.0 * np.cos(2 * np.pi * mi / n) for mi, n in zip(m, shape))
    q0 = 0.7 - 0.4j
    assert np.max(np.abs(O.apply_G(q0, e) - e / (lam - q0))) < 1e-12


def test_born_residual_identity_on_the_periodic_grid():
    """G(V u + f) - u = G(f - A u) with V = q - q0 and A = -Delta_h - q (both
    periodic here, where G is the exact background inverse)."""
    g = np.random.Generator(np.random.PCG64(71))
    shape = (10, 14)
    q = O.wavenumber_coef(1.0 + g.random(shape), 12.0, 2, 1.0)
    q0 = O.born_background(q)
    u, f = I.complex_normal(shape, g), I.complex_normal(shape, g)
    A_per = _periodic_background(0.0, u) - q * u
    lhs = O.apply_G(q0, (q - q0) * u + f) - u
    rhs = O.apply_G(q0, f - A_per)
    assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(rhs)


def test_born_solve_with_the_exact_preconditioner_takes_one_step():
    """With MG = (G A)^{-1} one Born+McMg step gives A^{-1} f exactly."""
    g = np.random.Generator(np.random.PCG64(72))
    shape = (6, 5)
    q = O.wavenumber_coef(1.0 + g.random(shape), 7.0, 1, 1.0)
    q0 = O.born_background(q)
    A = lambda v: O.apply_A(q, v)
    G = lambda v: O.apply_G(q0, v)
    GA = O.dense_matrix(lambda v: G(A(v)), shape)
    GAinv = np.linalg.inv(GA)
    M = lambda v: (GAinv @ v.reshape(-1)).reshape(shape)
    f = I.complex_normal(shape, g)
    u, info = O.born_solve(A, G, M, f, tol=1e-10, max_iters=5)
    assert info["iters"] == 1
    Ad = O.dense_matrix(A, shape)
    assert np.linalg.norm(u.reshape(-1) - np.linalg.solve(Ad, f.reshape(-1))) < 1e-10 * np.linalg.norm(u)
