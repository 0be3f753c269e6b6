"""Seeded synthetic inputs for the McMg online solve.

This module draws the media, right-hand sides, residuals and network weights
that both the FP64 oracle and the CUDA path consume.  It holds none of the
method's arithmetic (no operator, smoother, transfer, setup network or Krylov
step): only random draws, the workload parameters, and the constant values the
structured weight initialisation starts from.

Workloads (named by what they are; sizes follow the McMg experiments of
Section 4.1 where the paper fixes them):

* ``helm2d_n64_homogeneous``  -- 64^2, c = 1, 10 points per wavelength, 8-cell
  sponge, 3 levels with 1/4/8 channels, FP32, FGMRES(20).
* ``helm2d_n64_slmg``         -- the same grid with the one-channel degenerate
  weights: classical shifted-Laplacian multigrid (Appendix A.3, Eq. csl_shift).
* ``helm2d_n256_grf``         -- 256^2 Gaussian random field c in [1, 3],
  correlation length 16 cells, 8 ppw at c = 1, 16-cell sponge, 4 levels with
  8/16/32/64 channels, FP32, FGMRES(20).
* ``helm2d_n1024_layers``     -- 1024^2, six layers c in [1, 4] plus twenty
  discs of 10x contrast, 6 ppw, 6 levels with 8/16/32/64/64/64 channels, BF16
  channel mixing, FGMRES(30).
* ``helm3d_n256_grf``         -- 256^3 Gaussian random field c in [1, 3] plus
  three spheres of 5x contrast, 8 ppw, 10-cell sponge, 5 levels with
  8/16/32/64/64 channels, BF16 channel mixing, FGMRES(30).
* ``helm2d_n256_layers``      -- the 1024^2 recipe (layers + discs, 6 ppw,
  6 levels) on a 256^2 grid, small enough for the FP64 oracle's solve.
* ``helm3d_n64_grf``          -- the 256^3 recipe (random field + spheres,
  8 ppw, 10-cell sponge, 5 levels) on a 64^3 grid.
* ``serving_stream``          -- 256 requests, grids from {128, 256, 512,
  1024}^2, one random-field medium per request, 1-8 point sources each.

Weight tensors (all complex unless marked real) use these layouts:

* stencil taps, ``2d + 1`` of them, in the order
  centre, -x, +x, -y, +y[, -z, +z]; grids are stored x fastest;
* ``3^d`` transfer taps indexed ``((oz+1)*3 + (oy+1))*3 + (ox+1)`` with
  offsets in {-1, 0, 1};
* a channel-mixing matrix ``M[co][ci]`` maps input channel ci to output co.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "WORKLOADS", "workload", "nu_schedule", "grf", "layered_with_inclusions",
    "grf_with_spheres", "medium_for", "omega_for_ppw", "point_source",
    "random_point_sources", "complex_normal", "make_weights", "serving_requests",
]

GAMMA_MAX = 1.0          # peak sponge damping (the paper leaves it open)
EPS_STRUCTURED = 0.05    # size of the seeded perturbation in structured weights
SIGMA_RANDOM = 0.5       # scale of the purely random weights
JACOBI_OMEGA = 0.66      # weighted-Jacobi relaxation of the classical baseline


def nu_schedule(levels: int, degenerate: bool = False):
    """Pre/post smoothing counts per level.

    The paper's level lists such as [1,2,4,8,8] give the smoothing steps per
    level (Section 4.1, Appendix A.6).  Read as nu1 = nu2 = min(2^(l-1), 8) on
    levels l < L and nu1 = min(2^(L-1), 8), nu2 = 0 on the coarsest level, which
    Algorithm 2 only pre-smooths.  The degenerate shifted-Laplacian instance uses
    (2, 2) and 2 coarse steps (Appendix A.3).
    """
    if degenerate:
        pre = [2] * levels
        post = [2] * (levels - 1) + [0]
        return pre, post
    pre = [min(2 ** l, 8) for l in range(levels)]
    post = [min(2 ** l, 8) for l in range(levels - 1)] + [0]
    return pre, post


def _wl(name, dim, n, medium, ppw, sponge, levels, channels, precision, restart,
        mode="structured", seed=0, tol=1e-6, nrhs=1):
    pre, post = nu_schedule(levels, degenerate=(mode == "degenerate"))
    return dict(name=name, dim=dim, n=n, medium=medium, ppw=ppw, sponge=sponge,
                gamma_max=GAMMA_MAX, levels=levels, channels=list(channels),
                nu_pre=pre, nu_post=post, precision=precision, restart=restart,
                mode=mode, seed=seed, tol=tol, nrhs=nrhs)


WORKLOADS = {
    "helm2d_n64_homogeneous": _wl("helm2d_n64_homogeneous", 2, 64, "homogeneous", 10, 8,
                                  3, [1, 4, 8], "fp32", 20, seed=0),
    "helm2d_n64_slmg": _wl("helm2d_n64_slmg", 2, 64, "homogeneous", 10, 8,
                           3, [1, 1, 1], "fp32", 20, mode="degenerate", seed=0),
    "helm2d_n256_grf": _wl("helm2d_n256_grf", 2, 256, "grf", 8, 16,
                           4, [8, 16, 32, 64], "fp32", 20, seed=1),
    "helm2d_n1024_layers": _wl("helm2d_n1024_layers", 2, 1024, "layers", 6, 16,
                               6, [8, 16, 32, 64, 64, 64], "bf16", 30, seed=2),
    "helm3d_n256_grf": _wl("helm3d_n256_grf", 3, 256, "grf_spheres", 8, 10,
                           5, [8, 16, 32, 64, 64], "bf16", 30, seed=4),
    # the two large recipes at the largest sizes the FP64 oracle solves in
    # minutes: the same medium kind, ppw, sponge, levels, channels and Krylov
    "helm2d_n256_layers": _wl("helm2d_n256_layers", 2, 256, "layers", 6, 16,
                              6, [8, 16, 32, 64, 64, 64], "bf16", 30, seed=2),
    "helm3d_n64_grf": _wl("helm3d_n64_grf", 3, 64, "grf_spheres", 8, 10,
                          5, [8, 16, 32, 64, 64], "bf16", 30, seed=4),
}


def workload(name: str, **override) -> dict:
    """A copy of a named workload, with optional field overrides."""
    wl = dict(WORKLOADS[name])
    wl.update(override)
    if "levels" in override and "nu_pre" not in override:
        wl["nu_pre"], wl["nu_post"] = nu_schedule(wl["levels"], wl["mode"] == "degenerate")
    return wl


# --------------------------------------------------------------------------
# media
# --------------------------------------------------------------------------

def grf(shape, corr_len: float, c_min: float, c_max: float, rng) -> np.ndarray:
    """Gaussian random field: seeded white noise filtered by exp(-|xi|^2 l^2 / 2).

    xi is in radians per cell, the filter is applied with a periodic FFT, and
    the result is mapped linearly onto [c_min, c_max].
    """
    noise = rng.standard_normal(shape)
    spec = np.fft.fftn(noise)
    k2 = np.zeros(shape)
    for ax, m in enumerate(shape):
        xi = 2.0 * np.pi * np.fft.fftfreq(m)
        sh = [1] * len(shape)
        sh[ax] = m
        k2 = k2 + (xi ** 2).reshape(sh)
    field = np.real(np.fft.ifftn(spec * np.exp(-0.5 * k2 * corr_len ** 2)))
    lo, hi = field.min(), field.max()
    return c_min + (c_max - c_min) * (field - lo) / (hi - lo)


def layered_with_inclusions(n: int, rng, n_layers=6, n_discs=20, c_lo=1.0, c_hi=4.0,
                            contrast=10.0) -> np.ndarray:
    """Horizontal layers with uniform speeds plus fast circular inclusions (2D)."""
    cuts = np.sort(rng.integers(1, n, size=n_layers - 1))
    speeds = rng.uniform(c_lo, c_hi, size=n_layers)
    rows = np.searchsorted(cuts, np.arange(n), side="right")
    c = np.repeat(speeds[rows][:, None], n, axis=1)
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    bg = c.copy()
    for _ in range(n_discs):
        cy, cx = rng.uniform(0, n, size=2)
        rad = rng.uniform(n / 64, n / 16)
        inside = (yy - cy) ** 2 + (xx - cx) ** 2 <= rad ** 2
        c[inside] = contrast * bg[inside]
    return c


def grf_with_spheres(n: int, rng, n_spheres=3, contrast=5.0, corr_len=16.0) -> np.ndarray:
    """3D Gaussian random field in [1, 3] with fast spherical inclusions."""
    c = grf((n, n, n), corr_len, 1.0, 3.0, rng)
    bg = c.copy()
    zz, yy, xx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    for _ in range(n_spheres):
        cz, cy, cx = rng.uniform(0, n, size=3)
        rad = rng.uniform(n / 16, n / 8)
        inside = (zz - cz) ** 2 + (yy - cy) ** 2 + (xx - cx) ** 2 <= rad ** 2
        c[inside] = contrast * bg[inside]
    return c


def medium_for(wl: dict) -> np.ndarray:
    """Wave speed c on the workload's grid (float64, x fastest)."""
    shape = (wl["n"],) * wl["dim"]
    rng = np.random.Generator(np.random.PCG64(1000 + wl["seed"]))
    kind = wl["medium"]
    if kind == "homogeneous":
        return np.ones(shape)
    if kind == "grf":
        return grf(shape, 16.0, 1.0, 3.0, rng)
    if kind == "layers":
        return layered_with_inclusions(wl["n"], rng)
    if kind == "grf_spheres":
        return grf_with_spheres(wl["n"], rng)
    raise ValueError(kind)


def omega_for_ppw(c_min: float, ppw: float, n: int) -> float:
    """Angular frequency giving `ppw` points per wavelength at speed c_min.

    On the unit domain h = 1/n, and ppw = 2 pi / (k h) with k = omega / c
    (Section 4.1), so omega = 2 pi c_min n / ppw.
    """
    return 2.0 * math.pi * c_min * n / ppw


# --------------------------------------------------------------------------
# right-hand sides and residuals
# --------------------------------------------------------------------------

def point_source(shape, pos=None) -> np.ndarray:
    """Unit point source (complex128) at `pos`, default the grid centre."""
    f = np.zeros(shape, dtype=np.complex128)
    if pos is None:
        pos = tuple(m // 2 for m in shape)
    f[tuple(pos)] = 1.0
    return f


def random_point_sources(shape, sponge: int, count: int, rng) -> np.ndarray:
    """`count` unit point sources at seeded cells inside the non-sponge region.

    Returns an array of shape (count,) + shape: one right-hand side per source.
    """
    out = np.zeros((count,) + tuple(shape), dtype=np.complex128)
    for k in range(count):
        pos = tuple(int(rng.integers(sponge, m - sponge)) for m in shape)
        out[(k,) + pos] = 1.0
    return out


def complex_normal(shape, rng, scale=1.0) -> np.ndarray:
    """Complex Gaussian with unit variance per entry."""
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2.0)


# --------------------------------------------------------------------------
# weights
# --------------------------------------------------------------------------

def _fw_weights(dim: int) -> np.ndarray:
    """Full-weighting taps (1,2,1)/4 per axis over the 3^d transfer taps."""
    w1 = np.array([0.25, 0.5, 0.25])
    w = w1
    for _ in range(dim - 1):
        w = np.multiply.outer(w, w1)
    return w.reshape(-1)  # tap index ((oz+1)*3+(oy+1))*3+(ox+1)


def make_weights(dim: int, channels, nu_pre, nu_post, mode: str = "structured",
                 seed: int = 0) -> dict:
    """Seeded weights for a McMg model.

    mode:
      * ``"structured"`` -- the classical shifted-Laplacian multigrid values on
        channel (0, 0) (Laplacian cross scaled by 4^(1-l), weighted Jacobi 0.66,
        full weighting, bilinear prolongation, identity lift/projection) plus a
        complex Gaussian perturbation of size 0.05/sqrt(fan_in) on every entry
        except channel (0, 0), which keeps the classical value exactly.  The
        setup features are the classical coefficients on channel 0 and 0.05
        times the setup networks' output on the other channels (``feat_sl = 1``,
        ``feat_eps = 0.05``).
      * ``"degenerate"`` -- the classical values only, no perturbation and
        ``feat_eps = 0``: with one channel this is shifted-Laplacian multigrid.
      * ``"random"`` -- purely random complex weights of size 0.5/sqrt(fan_in)
        and features from the setup networks alone (``feat_sl = 0``,
        ``feat_eps = 1``).

    Draw order (one PCG64 stream): f_lift (weight, bias); then per level:
    stencil W, K_A, K_S, smoother W^(i), f_s (weight, bias), and for l < L:
    R, P, f_a (weight, bias); then g_lift and g_proj.
    """
    if mode not in ("structured", "degenerate", "random"):
        raise ValueError(mode)
    rng = np.random.Generator(np.random.PCG64(seed))
    L = len(channels)
    T = 2 * dim + 1
    T3 = 3 ** dim
    eps = {"structured": EPS_STRUCTURED, "degenerate": 0.0, "random": SIGMA_RANDOM}[mode]
    base_on = mode != "random"

    def cmat(shape, fan_in):
        z = complex_normal(shape, rng) * (eps / math.sqrt(fan_in))
        if base_on:
            z[..., 0, 0] = 0.0      # channel (0, 0) keeps the exact classical value
        return z

    def rconv(cout, cin):
        w = rng.standard_normal((cout, cin, T3)) / math.sqrt(cin * T3)
        b = 0.1 * rng.standard_normal(cout)
        return w, b

    fw = _fw_weights(dim)
    wts = dict(dim=dim, levels=L, channels=list(channels), nu_pre=list(nu_pre),
               nu_post=list(nu_post), feat_sl=1.0 if base_on else 0.0,
               feat_eps={"structured": EPS_STRUCTURED, "degenerate": 0.0, "random": 1.0}[mode],
               sl_shift=(1.0, -1.0))
    wts["flift_w"], wts["flift_b"] = rconv(2 * channels[0], 2)
    lv = []
    for l in range(L):
        C = channels[l]
        d = {}
        W = cmat((T, C, C), C * T)
        KA = cmat((C, C), C)
        KS = cmat((C, C), C)
        nsteps = nu_pre[l] + nu_post[l]
        Wsm = cmat((max(nsteps, 1), C, C), C)[:nsteps]
        if base_on:
            s = 4.0 ** (-l)
            W[0, 0, 0] += 2 * dim * s
            W[1:, 0, 0] += -s
            KA[0, 0] += 1.0
            KS[0, 0] += 1.0
            Wsm[:, 0, 0] += JACOBI_OMEGA
        d["W"], d["KA"], d["KS"], d["Wsm"] = W, KA, KS, Wsm
        d["fs_w"], d["fs_b"] = rconv(2 * C, 2 * C)
        if l < L - 1:
            Cn = channels[l + 1]
            R = cmat((T3, Cn, C), C * T3)
            P = cmat((T3, C, Cn), Cn * T3)
            if base_on:
                R[:, 0, 0] += fw
                P[:, 0, 0] += (2 ** dim) * fw
            d["R"], d["P"] = R, P
            d["fa_w"], d["fa_b"] = rconv(2 * Cn, 2 * C)
        lv.append(d)
    wts["lvl"] = lv
    lift = complex_normal((channels[0],), rng) * eps
    proj = complex_normal((channels[0],), rng) * (eps / math.sqrt(channels[0]))
    if base_on:
        lift[0] = 0.0
        proj[0] = 0.0
    if base_on:
        lift[0] += 1.0
        proj[0] += 1.0
    wts["lift"], wts["proj"] = lift, proj
    return wts


def weights_for(wl: dict) -> dict:
    return make_weights(wl["dim"], wl["channels"], wl["nu_pre"], wl["nu_post"],
                        wl["mode"], wl["seed"])


# --------------------------------------------------------------------------
# serving stream
# --------------------------------------------------------------------------

SERVING_CHANNELS = [8, 16, 32, 64, 64, 64]


def serving_levels(n: int) -> int:
    """Levels a request of grid n uses: a prefix of the shared 6-level model
    with the coarsest grid no smaller than 16 (128 -> 4, 256 -> 5, >= 512 -> 6)."""
    return min(6, int(round(math.log2(n / 16))) + 1)


def prefix_weights(w: dict, L: int) -> dict:
    """The first L levels of a model: level L-1 becomes the coarsest (its
    transfers are dropped and it keeps only its pre-smoothing steps)."""
    lv = [dict(x) for x in w["lvl"][:L]]
    last = lv[-1]
    for k in ("R", "P", "fa_w", "fa_b"):
        last.pop(k, None)
    last["Wsm"] = last["Wsm"][: w["nu_pre"][L - 1]]
    out = dict(w)
    out.update(levels=L, channels=list(w["channels"][:L]), nu_pre=list(w["nu_pre"][:L]),
               nu_post=list(w["nu_post"][: L - 1]) + [0], lvl=lv)
    return out


def serving_request_inputs(req: dict, base_weights: dict):
    """Medium, omega, weights and right-hand sides of one serving request:
    a Gaussian random field (correlation 16 cells, c in [1, 3]), 8 points per
    wavelength at c = 1, a 16-cell sponge and `nrhs` point sources."""
    n = req["n"]
    rng = np.random.Generator(np.random.PCG64(req["medium_seed"]))
    c = grf((n, n), 16.0, 1.0, 3.0, rng)
    omega = omega_for_ppw(1.0, 8.0, n)
    f = random_point_sources((n, n), 16, req["nrhs"], rng)
    return c, omega, prefix_weights(base_weights, req["levels"]), f


def serving_weights(seed: int = 3) -> dict:
    """The shared 6-level model (8/16/32/64/64/64 channels) requests take prefixes of."""
    pre, post = nu_schedule(6)
    return make_weights(2, SERVING_CHANNELS, pre, post, mode="structured", seed=seed)


def serving_requests(count=256, sizes=(128, 256, 512, 1024), rate_hz=100.0, seed=3):
    """Seeded request stream: grid size, medium seed, source count and arrival time.

    Arrivals are a Poisson process (exponential gaps) of rate `rate_hz`.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    reqs = []
    for i in range(count):
        t += rng.exponential(1.0 / rate_hz)
        n = int(sizes[rng.integers(0, len(sizes))])
        reqs.append(dict(id=i, n=n, nrhs=int(rng.integers(1, 9)), arrival_s=t,
                         medium_seed=10_000 + i, levels=serving_levels(n)))
    return reqs
