"""FP64 CPU oracle of the McMg online solve.  TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this module; the product path never does.  It is plain numpy in
complex128 / float64, slow and written to be checked against the paper by eye.
It shares no code with the CUDA path.

Arrays: a grid field has the grid shape (Ny, Nx) or (Nz, Ny, Nx), x fastest;
a multi-channel field adds a trailing channel axis.  All operators work in the
h^2-scaled system (the whole equation multiplied by h^2, h = 1/N on the unit
domain), which leaves relative residuals unchanged.

Functions and the passage each one follows:

* ``sponge_gamma``       -- sponge damping profile (Section 2.1, sponge equation)
* ``wavenumber_coef``    -- q = (k h)^2 (1 - i gamma), k = omega / c (Eq. helm, sponge eq.)
* ``apply_A``            -- the 5-/7-point operator (Eq. FDM_stencil)
* ``gelu``, ``conv3``    -- the setup layers (Eq. phys_feature)
* ``setup``              -- Algorithm 1 (feature hierarchy a_l, s_l)
* ``op_A``, ``op_S``     -- neural PDE operator and smoother (Section 3.2)
* ``restrict``, ``prolong`` -- strided and transposed convolutions (Section 3.2)
* ``vcycle``             -- Algorithm 2
* ``fgmres``             -- flexible GMRES(m), right preconditioned (the paper's
  GMRES+McMg, Section 3.3 and Table 2, in Saad's flexible form)
* ``stationary_solve``   -- the stationary McMg iteration (Eq. mcmg_iteration)
* ``coarse_basis``       -- raw coarse-basis response (Eq. coarse_basis)
* ``born_background``, ``green_symbol``, ``apply_G``, ``born_solve`` -- the
  Born+McMg variant with the discrete Green operator (Appendix, Born-series
  variant; Eq. discrete_symbol)
* ``dense_matrix``       -- brute-force dense assembly for tiny grids

Readings where the paper is silent (each is a parameter or stated here):
the grid size N includes the sponge cells; the sponge profile is quadratic in
the depth into the layer, max over axes, with peak gamma_max; neighbours
outside the grid are zero; the channels and weights are complex; K_x is a
separate pointwise matrix K_A for the PDE operator and K_S for the smoother.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

# --------------------------------------------------------------------------
# problem: sponge, wavenumber, operator
# --------------------------------------------------------------------------


def sponge_gamma(shape, width: int, gamma_max: float) -> np.ndarray:
    """Damping gamma: zero inside, growing quadratically into the sponge layer.

    Section 2.1: gamma vanishes in the domain and increases polynomially with
    the distance into the absorbing layer.  Per axis the depth of cell i is
    max(width - i, i - (N - 1 - width), 0) cells; the cell's depth is the
    largest over axes and gamma = gamma_max * (depth / width)^2.
    """
    depth = np.zeros(shape)
    for ax, n in enumerate(shape):
        i = np.arange(n, dtype=np.float64)
        d1 = np.maximum(np.maximum(width - i, i - (n - 1 - width)), 0.0)
        sh = [1] * len(shape)
        sh[ax] = n
        depth = np.maximum(depth, d1.reshape(sh))
    if width == 0:
        return np.zeros(shape)
    return gamma_max * (depth / width) ** 2


def wavenumber_coef(c: np.ndarray, omega: float, width: int, gamma_max: float) -> np.ndarray:
    """q = (k h)^2 (1 - i gamma) with k = omega / c and h = 1 / N (Eq. helm, sponge eq.)."""
    h = 1.0 / c.shape[0]
    kh2 = (omega * h / c) ** 2
    return kh2 * (1.0 - 1j * sponge_gamma(c.shape, width, gamma_max))


def apply_A(q: np.ndarray, u: np.ndarray) -> np.ndarray:
    """h^2 A u for the 5-point (2D) / 7-point (3D) stencil of Eq. FDM_stencil.

    (h^2 A u)_p = 2d u_p - sum of the 2d neighbours u_q - q_p u_p, where q
    carries the sponge factor (1 - i gamma) and neighbours outside the grid are
    zero.
    """
    d = u.ndim
    out = 2 * d * u - q * u
    for ax in range(d):
        out = out - _shift_grid(u, ax, -1) - _shift_grid(u, ax, +1)
    return out


def _shift_grid(u: np.ndarray, ax: int, s: int) -> np.ndarray:
    """y[p] = u[p + s e_ax], zero where p + s e_ax leaves the grid."""
    y = np.zeros_like(u)
    n = u.shape[ax]
    src = [slice(None)] * u.ndim
    dst = [slice(None)] * u.ndim
    if s > 0:
        src[ax] = slice(s, n)
        dst[ax] = slice(0, n - s)
    else:
        src[ax] = slice(0, n + s)
        dst[ax] = slice(-s, n)
    y[tuple(dst)] = u[tuple(src)]
    return y


# --------------------------------------------------------------------------
# multi-channel building blocks (trailing channel axis)
# --------------------------------------------------------------------------


def stencil_offsets(d: int):
    """Tap order centre, -x, +x, -y, +y[, -z, +z] as grid-axis offset tuples.

    Grid axes are ordered (z,) y, x, so x is the last grid axis.
    """
    offs = [(0,) * d]
    for ax in range(d):  # x, y, z
        g = d - 1 - ax
        for s in (-1, +1):
            o = [0] * d
            o[g] = s
            offs.append(tuple(o))
    return offs


def transfer_offsets(d: int):
    """3^d taps indexed ((oz+1)*3+(oy+1))*3+(ox+1); offsets in grid-axis order."""
    rng = (-1, 0, 1)
    if d == 2:
        return [(oy, ox) for oy in rng for ox in rng]
    return [(oz, oy, ox) for oz in rng for oy in rng for ox in rng]


def shift(x: np.ndarray, off) -> np.ndarray:
    """y[p] = x[p + off] over the grid axes (channel axis last), zero outside."""
    y = x
    for ax, s in enumerate(off):
        if s != 0:
            y = _shift_grid_ch(y, ax, s)
    return y


def _shift_grid_ch(x, ax, s):
    y = np.zeros_like(x)
    n = x.shape[ax]
    src = [slice(None)] * x.ndim
    dst = [slice(None)] * x.ndim
    if s > 0:
        src[ax] = slice(s, n)
        dst[ax] = slice(0, n - s)
    else:
        src[ax] = slice(0, n + s)
        dst[ax] = slice(-s, n)
    y[tuple(dst)] = x[tuple(src)]
    return y


def mix(M: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Pointwise channel mixing: y[..., co] = sum_ci M[co, ci] x[..., ci]."""
    return x @ M.T


def stencil_conv(W: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Multi-channel cross-shaped convolution: sum over taps t of W[t] x[p + o_t]."""
    d = x.ndim - 1
    out = np.zeros(x.shape[:-1] + (W.shape[1],), dtype=np.complex128)
    for t, off in enumerate(stencil_offsets(d)):
        out = out + mix(W[t], shift(x, off))
    return out


def op_A(lv: dict, a: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Neural PDE operator A_l(x) = W_l * x + a_l (.) (K_A x)   (Section 3.2)."""
    return stencil_conv(lv["W"], x) + a * mix(lv["KA"], x)


def op_S(lv: dict, s: np.ndarray, i: int, x: np.ndarray) -> np.ndarray:
    """Neural smoother S^(i)(x) = W^(i) (s_l (.) (K_S x))   (Section 3.2); i is 0-based."""
    return mix(lv["Wsm"][i], s * mix(lv["KS"], x))


def restrict(R: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Strided (stride 2, padding 1) 3^d convolution: y[J] = sum_o R[o] x[2J + o]."""
    d = x.ndim - 1
    coarse = tuple(m // 2 for m in x.shape[:-1])
    y = np.zeros(coarse + (R.shape[1],), dtype=np.complex128)
    for t, off in enumerate(transfer_offsets(d)):
        xs = shift(x, off)
        sl = tuple(slice(0, 2 * m, 2) for m in coarse)
        y = y + mix(R[t], xs[sl])
    return y


def prolong(P: np.ndarray, y: np.ndarray, fine_shape) -> np.ndarray:
    """Transposed strided convolution: x[2J + o] += P[o] y[J] (zero outside the grid)."""
    d = y.ndim - 1
    x = np.zeros(tuple(fine_shape) + (P.shape[1],), dtype=np.complex128)
    for t, off in enumerate(transfer_offsets(d)):
        z = np.zeros_like(x)
        sl = tuple(slice(0, 2 * m, 2) for m in y.shape[:-1])
        z[sl] = mix(P[t], y)
        # z holds the contribution at 2J; move it to 2J + o
        x = x + shift(z, tuple(-o for o in off))
    return x


# --------------------------------------------------------------------------
# setup (Algorithm 1)
# --------------------------------------------------------------------------


def gelu(x: np.ndarray) -> np.ndarray:
    """Exact GELU x * Phi(x) with Phi the standard normal CDF (Eq. phys_feature's sigma)."""
    return x * 0.5 * (1.0 + erf(x / math.sqrt(2.0)))


def conv3(w: np.ndarray, b: np.ndarray, x: np.ndarray, stride: int = 1) -> np.ndarray:
    """Real 3^d convolution with zero padding 1 and bias.

    x: grid + (Cin,), w: (Cout, Cin, 3^d), b: (Cout,).  With stride 2 the
    output node J reads the input around 2J.
    """
    d = x.ndim - 1
    out_grid = tuple(m // stride for m in x.shape[:-1])
    y = np.zeros(out_grid + (w.shape[0],))
    sl = tuple(slice(0, stride * m, stride) for m in out_grid)
    for t, off in enumerate(transfer_offsets(d)):
        y = y + shift(x, off)[sl] @ w[:, :, t].T
    return y + b


def _to_complex(xr: np.ndarray) -> np.ndarray:
    """Pairs of real channels (2c, 2c+1) -> complex channel c."""
    return xr[..., 0::2] + 1j * xr[..., 1::2]


def setup(q: np.ndarray, wts: dict):
    """Algorithm 1: cached features {a_l, s_l} for every level.

    Nonlinear branch (the setup networks): input m = ((kh)^2, (kh)^2 gamma) as
    two real channels; a_1 = f_lift(m); s_l = f_s^l(a_l); a_{l+1} = f_a^l(a_l),
    each one 3^d convolution + bias + GELU (f_a with stride 2), real channels
    paired into complex ones.

    Classical branch, active on channel 0 when feat_sl = 1: the shifted-Laplacian
    coefficients of Appendix A.3, q_1 = q, q_{l+1} = full-weighting restriction
    of q_l, a_l = -(beta1 + i beta2) q_l and s_l = 1 / (2d 4^(1-l) + a_l), the
    inverse diagonal of the level-l shifted operator in fine-grid h^2 units.

    Features: a_l = feat_eps * network output on every channel, except that
    channel 0 holds feat_sl * classical coefficient instead when feat_sl != 0.
    """
    d = q.ndim
    L = wts["levels"]
    beta = complex(*wts["sl_shift"])
    m = np.stack([q.real, -q.imag], axis=-1)
    net_a = gelu(conv3(wts["flift_w"], wts["flift_b"], m))
    fw = np.zeros((3 ** d, 1, 1), dtype=np.complex128)
    w1 = np.array([0.25, 0.5, 0.25])
    fwt = w1
    for _ in range(d - 1):
        fwt = np.multiply.outer(fwt, w1)
    fw[:, 0, 0] = fwt.reshape(-1)
    ql = q[..., None].astype(np.complex128)
    feats = []
    for l in range(L):
        lv = wts["lvl"][l]
        C = wts["channels"][l]
        net_s = gelu(conv3(lv["fs_w"], lv["fs_b"], net_a))
        a = wts["feat_eps"] * _to_complex(net_a)
        s = wts["feat_eps"] * _to_complex(net_s)
        if wts["feat_sl"] != 0.0:
            a_sl = -beta * ql[..., 0]
            s_sl = 1.0 / (2 * d * 4.0 ** (-l) + a_sl)
            a[..., 0] = wts["feat_sl"] * a_sl
            s[..., 0] = wts["feat_sl"] * s_sl
        assert a.shape[-1] == C
        feats.append((a, s))
        if l < L - 1:
            net_a = gelu(conv3(lv["fa_w"], lv["fa_b"], net_a, stride=2))
            ql = restrict(fw, ql)
    return feats


# --------------------------------------------------------------------------
# V-cycle (Algorithm 2)
# --------------------------------------------------------------------------


def vcycle(wts: dict, feats, r: np.ndarray) -> np.ndarray:
    """Algorithm 2: e = MG(r) for one scalar residual r (grid array, complex)."""
    L = wts["levels"]
    lvs = wts["lvl"]
    nu1, nu2 = wts["nu_pre"], wts["nu_post"]
    rs = [None] * L
    es = [None] * L
    rs[0] = r[..., None] * wts["lift"]                      # r_1 = g_lift(r)
    for l in range(L):                                       # down cycle
        a, s = feats[l]
        e = np.zeros_like(rs[l])                             # e_l^(0) = 0
        for i in range(nu1[l]):
            e = e + op_S(lvs[l], s, i, rs[l] - op_A(lvs[l], a, e))
        es[l] = e
        if l < L - 1:
            rs[l + 1] = restrict(lvs[l]["R"], rs[l] - op_A(lvs[l], a, e))
    for l in range(L - 2, -1, -1):                           # up cycle
        a, s = feats[l]
        e = es[l] + prolong(lvs[l]["P"], es[l + 1], es[l].shape[:-1])
        for i in range(nu2[l]):
            e = e + op_S(lvs[l], s, nu1[l] + i, rs[l] - op_A(lvs[l], a, e))
        es[l] = e
    return es[0] @ wts["proj"]                               # e = g_proj(e_1)


# --------------------------------------------------------------------------
# outer iterations
# --------------------------------------------------------------------------


def coarse_basis(wts: dict, level: int, index, channel: int, fine_shape) -> np.ndarray:
    """Raw coarse-basis response of Eq. coarse_basis (Section 3.4): the one-hot
    latent tensor delta_alpha at grid location `index` (slowest axis first)
    and channel `channel` of `level` (0-based, >= 1), carried to the finest
    level by the learned prolongations in turn, then mapped to a scalar field
    by g_proj."""
    lv = wts["lvl"]
    shapes = [tuple(n >> l for n in fine_shape) for l in range(wts["levels"])]
    y = np.zeros(shapes[level] + (wts["channels"][level],), dtype=np.complex128)
    y[tuple(index) + (channel,)] = 1.0
    for l in range(level - 1, -1, -1):
        y = prolong(lv[l]["P"], y, shapes[l])
    return y @ wts["proj"]


def _norm(x):
    return float(np.sqrt(np.vdot(x, x).real))


def fgmres(A, M, f: np.ndarray, x0=None, m: int = 20, tol: float = 1e-6,
           max_iters: int | None = None):
    """Restarted flexible GMRES(m) with right preconditioner M (Saad's FGMRES).

    The paper uses McMg as a GMRES preconditioner (Section 3.3, Table 2); the
    flexible form stores the preconditioned vectors z_j = M(v_j) so that the
    preconditioner may vary between applications.  Modified Gram-Schmidt,
    complex Givens rotations, zero initial guess by default.  A cycle ends when
    the implicit residual |g_{j+1}| / ||f|| <= tol, on happy breakdown, or after
    m steps; convergence is then confirmed by the true residual ||f - A x|| /
    ||f||, and the method restarts from x if it is not met.

    Returns (x, info) with info = dict(iters, restarts, rel_residual, history,
    converged); iters counts preconditioner applications.
    """
    x = np.zeros_like(f) if x0 is None else x0.copy()
    fnorm = _norm(f)
    if max_iters is None:
        max_iters = 20 * f.shape[0]
    iters, restarts = 0, 0
    hist = []
    if fnorm == 0.0:
        return np.zeros_like(f), dict(iters=0, restarts=0, rel_residual=0.0, history=[0.0],
                                      converged=True)
    while True:
        r = f - A(x)
        beta = _norm(r)
        rel = beta / fnorm
        hist.append(rel)
        if rel <= tol or iters >= max_iters:
            return x, dict(iters=iters, restarts=restarts, rel_residual=rel, history=hist,
                           converged=rel <= tol)
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        k = 0
        for j in range(m):
            z = M(V[j])
            Z.append(z)
            w = A(z)
            w0 = _norm(w)
            for i in range(j + 1):                       # modified Gram-Schmidt
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            hn = _norm(w)
            H[j + 1, j] = hn
            for i in range(j):                           # previous rotations
                h0, h1 = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * h0 + sn[i] * h1
                H[i + 1, j] = -np.conj(sn[i]) * h0 + cs[i] * h1
            a, b = H[j, j], H[j + 1, j]
            rho = math.sqrt(abs(a) ** 2 + abs(b) ** 2)
            if abs(a) == 0.0:
                cs[j], sn[j] = 0.0, 1.0
            else:
                cs[j] = abs(a) / rho
                sn[j] = (a / abs(a)) * np.conj(b) / rho
            H[j, j] = cs[j] * a + sn[j] * b
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            iters += 1
            k = j + 1
            hist.append(abs(g[j + 1]) / fnorm)
            if abs(g[j + 1]) / fnorm <= tol or hn <= 1e-14 * w0 or iters >= max_iters:
                break
            V.append(w / hn)
        y = np.zeros(k, dtype=np.complex128)              # back substitution
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
        for i in range(k):
            x = x + y[i] * Z[i]
        restarts += 1


def stationary_solve(A, M, f: np.ndarray, tol: float = 1e-6, max_iters: int = 1000):
    """Stationary McMg iteration r = f - A u, u <- u + MG(r) (Eq. mcmg_iteration)."""
    u = np.zeros_like(f)
    fnorm = _norm(f)
    hist = []
    for it in range(max_iters + 1):
        r = f - A(u)
        rel = _norm(r) / fnorm
        hist.append(rel)
        if rel <= tol or it == max_iters or not np.isfinite(rel):
            return u, dict(iters=it, rel_residual=rel, history=hist, converged=rel <= tol)
        u = u + M(r)


# --------------------------------------------------------------------------
# Born+McMg (Appendix, Born-series variant and discrete Green operator)
# --------------------------------------------------------------------------


def born_background(q: np.ndarray) -> complex:
    """Background q0 = (k0 h)^2 of the Born-series form, V = q - q0.  The
    paper leaves k0 open; reading: Re q0 halfway between the extremes of
    Re q, and Im q0 = -max |q - Re q0| (the convergent-Born-series choice,
    with the sponge's damping sign), so the background symbol never vanishes
    and |V| <= |Im q0|."""
    mid = 0.5 * (float(q.real.max()) + float(q.real.min()))
    eps = float(np.abs(q - mid).max())
    return complex(mid, -eps)


def green_symbol(shape, q0: complex) -> np.ndarray:
    """Fourier multiplier of G = (-Delta_h - k0^2)^{-1} in the h^2-scaled
    system: 1 / (sum_a 4 sin^2(pi m_a / N_a) - q0), the discrete-Laplacian
    symbol of Eq. discrete_symbol at xi_a h = 2 pi m_a / N_a (periodic modes,
    the FFT used as a diagonalisation of the five-/seven-point operator)."""
    mu = np.zeros(shape)
    for ax, n in enumerate(shape):
        sa = 4.0 * np.sin(np.pi * np.arange(n) / n) ** 2
        mu = mu + sa.reshape([-1 if a == ax else 1 for a in range(len(shape))])
    return 1.0 / (mu - q0)


def apply_G(q0: complex, x: np.ndarray) -> np.ndarray:
    """G x through the FFT (discrete Green operator)."""
    return np.fft.ifftn(np.fft.fftn(x) * green_symbol(x.shape, q0))


def born_solve(A, G, M, f: np.ndarray, tol: float = 1e-6, max_iters: int = 1000):
    """Born+McMg: u <- u + MG(G(V u + f) - u), the Born-series residual taken
    in the paper's equivalent form G(f - A u) with the solver's own A (zero
    Dirichlet closure; G is the periodic background inverse, so the iteration
    is the Helmholtz residual left-preconditioned by G and corrected by MG).
    Stops on the Helmholtz residual ||f - A u|| / ||f||."""
    u = np.zeros_like(f)
    fnorm = _norm(f)
    hist = []
    for it in range(max_iters + 1):
        r = f - A(u)
        rel = _norm(r) / fnorm
        hist.append(rel)
        if rel <= tol or it == max_iters or not np.isfinite(rel):
            return u, dict(iters=it, rel_residual=rel, history=hist, converged=rel <= tol)
        u = u + M(G(r))


def dense_matrix(op, shape) -> np.ndarray:
    """Dense matrix of a linear map on grid fields, built column by column."""
    n = int(np.prod(shape))
    Mx = np.zeros((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1.0
        Mx[:, j] = op(e.reshape(shape)).reshape(-1)
    return Mx


def problem(c: np.ndarray, omega: float, width: int, gamma_max: float):
    """Convenience: q and the closure u -> h^2 A u."""
    q = wavenumber_coef(c, omega, width, gamma_max)
    return q, (lambda u: apply_A(q, u))
