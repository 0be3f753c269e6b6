"""Shared helpers for the tests: build the same model for the oracle and for
the CUDA path from the seeded input generators."""
from __future__ import annotations

import numpy as np

from oracle import mcmg_oracle as O
from paper_2606_30495_b300 import inputs as I


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def model(shape, channels, mode="structured", seed=0, ppw=8.0, sponge=4, medium="grf",
          nu=None, gamma_max=1.0):
    """Medium, omega, oracle q and features, and weights for a small case."""
    d = len(shape)
    L = len(channels)
    pre, post = nu if nu is not None else I.nu_schedule(L, degenerate=(mode == "degenerate"))
    w = I.make_weights(d, list(channels), pre, post, mode=mode, seed=seed)
    if medium == "grf":
        c = I.grf(shape, 4.0, 1.0, 3.0, rng(100 + seed))
    else:
        c = np.ones(shape)
    omega = I.omega_for_ppw(c.min(), ppw, shape[0])
    q = O.wavenumber_coef(c, omega, sponge, gamma_max)
    feats = O.setup(q, w)
    return dict(c=c, omega=omega, q=q, w=w, feats=feats, sponge=sponge, gamma_max=gamma_max,
                shape=tuple(shape))


def workload_model(name, **over):
    wl = I.workload(name, **over)
    c = I.medium_for(wl)
    omega = I.omega_for_ppw(c.min(), wl["ppw"], wl["n"])
    q = O.wavenumber_coef(c, omega, wl["sponge"], wl["gamma_max"])
    w = I.weights_for(wl)
    return dict(c=c, omega=omega, q=q, w=w, feats=None, sponge=wl["sponge"],
                gamma_max=wl["gamma_max"], shape=c.shape, wl=wl)


def relerr(a, b):
    """The larger of the relative L2 error ||a - b|| / ||b|| and the
    element-wise error max|a - b| / max|b|, so one bound checks both the
    field as a whole and every element (an error confined to the sponge or
    the boundary cells cannot hide under the interior's L2 norm)."""
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    d = a - b
    l2 = float(np.linalg.norm(d) / max(np.linalg.norm(b), 1e-300))
    if d.size == 0:
        return l2
    mx = float(np.max(np.abs(d)) / max(np.max(np.abs(b)), 1e-300))
    return max(l2, mx)
