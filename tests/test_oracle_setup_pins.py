"""Pins of the oracle's setup networks (Algorithm 1, Eq. phys_feature) and of
the multi-channel lift / projection of Algorithm 2, recomputed by hand.

Every expected value here is built at the test site from library routines
(scipy.ndimage.correlate for each real convolution, scipy.special.erf for the
GELU of Eq. phys_feature) in the order Algorithm 1 states, not from the
oracle's own helpers:

  m    = ((kh)^2, (kh)^2 gamma)            two real input channels
  a_1  = f_lift(m)                         3^d convolution + bias + GELU
  s_l  = f_s^l(a_l)                        same level's a_l
  a_l+1 = f_a^l(a_l)                       3^d convolution, stride 2, + GELU

and real channel pairs (2c, 2c+1) become complex channel c, scaled by the
feature scale; channel 0 takes the classical coefficient when that branch is on.
A mistake such as feeding f_s the next level's a, pairing (c, c + C), dropping
the bias, applying GELU before the bias or skipping the feature scale fails
one of these tests.
"""
import math

import numpy as np
import pytest
import scipy.ndimage
from scipy.special import erf

from oracle import mcmg_oracle as O
from paper_2606_30495_b300 import inputs as I


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _gelu(x):
    # x * Phi(x), Phi the standard normal CDF, written from erf
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def _conv_layer(x, w, b, stride=1):
    """sum_ci correlate(x[..., ci], kernel(co, ci)) + b[co], zero padding,
    then the stride-2 subsample y[J] = full[2J]."""
    d = x.ndim - 1
    cout, cin = w.shape[0], w.shape[1]
    grid = x.shape[:-1]
    out = np.zeros(grid + (cout,))
    for co in range(cout):
        acc = np.zeros(grid)
        for ci in range(cin):
            k = w[co, ci].reshape((3,) * d)      # k[oy+1, ox+1] (C order, x fastest)
            acc += scipy.ndimage.correlate(x[..., ci], k, mode="constant", cval=0.0)
        out[..., co] = acc + b[co]
    if stride == 2:
        out = out[tuple(slice(0, 2 * (m // 2), 2) for m in grid)]
    return out


def _pair(xr):
    C = xr.shape[-1] // 2
    z = np.zeros(xr.shape[:-1] + (C,), dtype=np.complex128)
    for c in range(C):
        z[..., c] = xr[..., 2 * c] + 1j * xr[..., 2 * c + 1]
    return z


def _setup_by_hand(q, w):
    d = q.ndim
    beta = complex(*w["sl_shift"])
    kh2 = q.real
    kh2gamma = -q.imag                  # q = (kh)^2 (1 - i gamma)
    m = np.stack([kh2, kh2gamma], axis=-1)
    net_a = _gelu(_conv_layer(m, w["flift_w"], w["flift_b"]))
    # classical coefficients, level by level: q_1 = q, q_l+1 = full weighting of q_l
    fw1 = np.array([0.25, 0.5, 0.25])
    fwk = fw1
    for _ in range(d - 1):
        fwk = np.multiply.outer(fwk, fw1)
    ql = q.copy()
    out = []
    for l in range(w["levels"]):
        lv = w["lvl"][l]
        net_s = _gelu(_conv_layer(net_a, lv["fs_w"], lv["fs_b"]))
        a = w["feat_eps"] * _pair(net_a)
        s = w["feat_eps"] * _pair(net_s)
        if w["feat_sl"] != 0.0:
            a_sl = -beta * ql
            a[..., 0] = w["feat_sl"] * a_sl
            s[..., 0] = w["feat_sl"] / (2 * d * 4.0 ** (-l) + a_sl)
        out.append((a, s))
        if l < w["levels"] - 1:
            net_a = _gelu(_conv_layer(net_a, lv["fa_w"], lv["fa_b"], stride=2))
            full = (scipy.ndimage.correlate(ql.real, fwk, mode="constant")
                    + 1j * scipy.ndimage.correlate(ql.imag, fwk, mode="constant"))
            ql = full[tuple(slice(0, 2 * (mm // 2), 2) for mm in ql.shape)]
    return out


@pytest.mark.parametrize("shape,channels,mode", [
    ((12, 10), (2, 3), "random"),
    ((8, 8, 6), (2, 2), "random"),
    ((16, 12), (3, 2, 2), "structured"),
    ((8, 6, 8), (2, 3), "structured"),
])
def test_setup_networks_follow_algorithm_1(shape, channels, mode):
    L = len(channels)
    pre, post = I.nu_schedule(L)
    w = I.make_weights(len(shape), list(channels), pre, post, mode=mode, seed=3)
    c = I.grf(shape, 3.0, 1.0, 3.0, _rng(21))
    q = O.wavenumber_coef(c, 1.7 * shape[0], 2, 1.0)
    got = O.setup(q, w)
    want = _setup_by_hand(q, w)
    assert len(got) == L
    for l in range(L):
        for k in range(2):
            g, h = got[l][k], want[l][k]
            assert g.shape == h.shape == tuple(n >> l for n in shape) + (channels[l],)
            assert np.max(np.abs(g - h)) <= 1e-13 * max(np.max(np.abs(h)), 1.0), (l, k)
    # the network channels are live (not all zero) on every level
    for l in range(L):
        assert np.max(np.abs(got[l][0][..., 1:])) > 1e-4 * w["feat_eps"]


def test_setup_rejects_misreadings():
    """The by-hand setup separates the readings that a slip would produce."""
    shape, channels = (12, 12), (2, 2)
    pre, post = I.nu_schedule(2)
    w = I.make_weights(2, list(channels), pre, post, mode="random", seed=5)
    c = I.grf(shape, 3.0, 1.0, 3.0, _rng(22))
    q = O.wavenumber_coef(c, 20.0, 2, 1.0)
    got = O.setup(q, w)
    m = np.stack([q.real, -q.imag], axis=-1)
    net_a = _gelu(_conv_layer(m, w["flift_w"], w["flift_b"]))
    # pairing (c, c + C) instead of (2c, 2c + 1)
    C = channels[0]
    wrong_pair = net_a[..., :C] + 1j * net_a[..., C:]
    assert np.max(np.abs(got[0][0] - wrong_pair)) > 1e-3
    # f_s fed the next level's a: s_2 from net_a of level 1 (no stride) differs
    lv0, lv1 = w["lvl"]
    net_a2 = _gelu(_conv_layer(net_a, lv0["fa_w"], lv0["fa_b"], stride=2))
    s2_right = _pair(_gelu(_conv_layer(net_a2, lv1["fs_w"], lv1["fs_b"])))
    s2_wrong = _pair(_gelu(_conv_layer(net_a, lv1["fs_w"], lv1["fs_b"])))[::2, ::2]
    assert np.max(np.abs(got[1][1] - s2_right)) < 1e-13
    assert np.max(np.abs(got[1][1] - s2_wrong)) > 1e-3
    # the input's second channel is (kh)^2 gamma >= 0, not Im q
    m_wrong = np.stack([q.real, q.imag], axis=-1)
    a_wrong = _pair(_gelu(_conv_layer(m_wrong, w["flift_w"], w["flift_b"])))
    assert np.max(np.abs(got[0][0] - a_wrong)) > 1e-6


def test_feature_scale_and_classical_channel():
    """Structured weights: channels >= 1 are feat_eps times the network output;
    channel 0 is the classical coefficient; halving feat_eps halves the rest."""
    shape, channels = (8, 8), (3, 2)
    pre, post = I.nu_schedule(2)
    w = I.make_weights(2, list(channels), pre, post, mode="structured", seed=7)
    q = O.wavenumber_coef(np.ones(shape), 12.0, 2, 1.0)
    f1 = O.setup(q, w)
    w2 = dict(w, feat_eps=0.5 * w["feat_eps"])
    f2 = O.setup(q, w2)
    for l in range(2):
        for k in range(2):
            np.testing.assert_allclose(f2[l][k][..., 1:], 0.5 * f1[l][k][..., 1:], rtol=1e-14,
                                       atol=0)
            np.testing.assert_array_equal(f2[l][k][..., 0], f1[l][k][..., 0])
    beta = complex(*w["sl_shift"])
    np.testing.assert_allclose(f1[0][0][..., 0], -beta * q, rtol=1e-15)


@pytest.mark.parametrize("shape,C", [((6, 5), 4), ((3, 4, 5), 3)])
def test_single_level_single_step_vcycle_is_proj_W_s_KS_lift(shape, C):
    """One level, one pre-smoothing step from e = 0: Algorithm 2 reduces to
    e(p) = g_proj . W^(1) (s_p (.) (K_S (g_lift r(p)))) at every node, a closed
    form that pins the lift (a column applied to r), the projection (a row
    contracted with e_1, no conjugation) and the order W^(1) o diag(s) o K_S."""
    g = _rng(31)
    d = len(shape)
    w = I.make_weights(d, [C], [1], [0], mode="random", seed=9)
    s = I.complex_normal(shape + (C,), g)
    a = I.complex_normal(shape + (C,), g)
    r = I.complex_normal(shape, g)
    got = O.vcycle(w, [(a, s)], r)
    lift, proj = w["lift"], w["proj"]
    KS, W1 = w["lvl"][0]["KS"], w["lvl"][0]["Wsm"][0]
    want = np.zeros(shape, dtype=np.complex128)
    for p in np.ndindex(*shape):
        r1 = lift * r[p]                       # C-vector
        z = s[p] * (KS @ r1)
        e1 = W1 @ z
        want[p] = np.sum(proj * e1)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))
    # the swapped roles (proj as lift) give a different field
    swapped = np.zeros(shape, dtype=np.complex128)
    for p in np.ndindex(*shape):
        swapped[p] = np.sum(lift * (W1 @ (s[p] * (KS @ (proj * r[p])))))
    assert np.max(np.abs(swapped - want)) > 1e-3 * np.max(np.abs(want))
