"""Parity of the tensor-core smoothing step and residual whose A operands
live in tensor memory (persistent CTAs), in both operand precisions, with the
FP64 oracle.

* FP32-accurate mixing (three TF32 products per FP32 product): held to the
  FP32 bound, 1e-5 relative (L2 and element-wise), per step, per residual
  and per V-cycle, and the full-size 256^2 solve to the stored oracle
  iteration count within 10%.
* BF16 mixing: 1e-2 per step, 2e-2 per V-cycle (the BF16 bound).

The large cases have more 128-node tiles than the grid has CTAs, so every
CTA walks several tiles, and node counts that are not a multiple of 128; the
C = 32 / 64 cases run the variant that streams its weights through shared
memory (one CTA per SM).
The tensor-core restriction and prolongation (the last transfer shape, on
levels whose transfer input has 16 or more channels) are held to the same
bounds, alone, with many items per CTA, and inside V-cycles.
Every bounded wait inside the kernels must have finished (error word 0).
"""
import numpy as np
import pytest

from oracle import mcmg_oracle as O
from paper_2606_30495_b300 import inputs as I
from tests._models import model, relerr, rng, workload_model

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL_BF16_STEP = 1e-2
TOL_BF16_VCYCLE = 2e-2


@pytest.fixture(scope="module")
def ctx():
    from paper_2606_30495_b300 import mcmg
    c = mcmg.Context(0)
    yield c
    c.close()


def dev(a, dtype=torch.complex64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


def handle(ctx, m, precision):
    from paper_2606_30495_b300 import mcmg
    return mcmg.Handle(ctx, m["c"], m["omega"], m["sponge"], m["gamma_max"], m["w"],
                       precision=precision)


def _prec(name):
    from paper_2606_30495_b300 import mcmg
    return {"fp32tc": mcmg.FP32_TC, "bf16": mcmg.BF16}[name]


def _tols(name):
    return (TOL32, TOL32) if name == "fp32tc" else (TOL_BF16_STEP, TOL_BF16_VCYCLE)


CASES = [
    ("fp32tc", (34, 30), [8, 16], "random"),
    ("fp32tc", (20, 36), [16, 32], "random"),
    ("fp32tc", (34, 30), [8, 16], "structured"),
    ("fp32tc", (6, 8, 10), [8, 16], "random"),
    ("fp32tc", (10, 6, 14), [16, 16], "random"),
    ("fp32tc", (16, 12), [32, 64], "random"),
    ("fp32tc", (4, 6, 8), [64, 64], "random"),
    ("fp32tc", (8, 6, 10), [32, 32], "structured"),
    ("bf16", (22, 18), [8, 32], "random"),
    ("bf16", (6, 10, 14), [32, 32], "random"),
    ("bf16", (16, 12), [64, 64], "random"),
    ("bf16", (4, 6, 8), [64, 64], "random"),
    ("fp32tc", (6, 8, 64), [8, 16], "random"),     # coarse x extent 32: line-staged restriction
    ("bf16", (20, 64), [8, 8], "random"),
]
IDS = [f"{p}-{'x'.join(map(str, s))}-C{'-'.join(map(str, c))}-{m}" for p, s, c, m in CASES]


@pytest.fixture(scope="module", params=CASES, ids=IDS)
def case(request, ctx):
    prec, shape, channels, mode = request.param
    m = model(shape, channels, mode=mode, seed=6)
    h = handle(ctx, m, _prec(prec))
    yield prec, m, h
    assert h.device_error() == 0
    h.close()


def _check_step(prec, m, h, l, first, nrhs=2, seed=10):
    w = m["w"]
    C = w["channels"][l]
    shp = tuple(n >> l for n in m["shape"]) + (C,)
    a, s = m["feats"][l]
    nsteps = w["nu_pre"][l] + w["nu_post"][l]
    tol = _tols(prec)[0]
    for step in sorted({0, nsteps - 1}):
        r = I.complex_normal((nrhs,) + shp, rng(seed + step))
        e_in = None if first else I.complex_normal((nrhs,) + shp, rng(seed + 10 + step))
        out = torch.zeros(r.shape, dtype=torch.complex64, device="cuda")
        h.smooth(l, step, dev(r), None if first else dev(e_in), out, nrhs=nrhs)
        want = []
        for k in range(nrhs):
            e0 = np.zeros(shp, complex) if first else e_in[k]
            want.append(e0 + O.op_S(w["lvl"][l], s, step, r[k] - O.op_A(w["lvl"][l], a, e0)))
        err = relerr(host(out), np.stack(want))
        assert err < tol, (l, step, err)


@pytest.mark.parametrize("first", [True, False])
def test_step(case, first):
    prec, m, h = case
    for l in range(m["w"]["levels"]):
        _check_step(prec, m, h, l, first)


def test_residual_restrict(case):
    """r - A_l(e) (the tensor-core residual on C_l in {8, 16[, 32]}), then R."""
    prec, m, h = case
    w = m["w"]
    tol = _tols(prec)[0]
    for l in range(w["levels"] - 1):
        C, Cn = w["channels"][l], w["channels"][l + 1]
        shp = tuple(n >> l for n in m["shape"])
        cshp = tuple(n >> (l + 1) for n in m["shape"])
        a, _ = m["feats"][l]
        lv = w["lvl"][l]
        r = I.complex_normal((2,) + shp + (C,), rng(30))
        e = I.complex_normal((2,) + shp + (C,), rng(31))
        rc = torch.zeros((2,) + cshp + (Cn,), dtype=torch.complex64, device="cuda")
        h.residual_restrict(l, dev(r), dev(e), rc, nrhs=2)
        want = np.stack([O.restrict(lv["R"], r[k] - O.op_A(lv, a, e[k])) for k in range(2)])
        assert relerr(host(rc), want) < tol, l


def _xts_supported(C, Cn, restrict_):
    """Channel pairs of the tensor-core transfer: input side >= 16 channels
    (restriction: >= 8), output equal to or half / twice the input (the
    library's model family)."""
    ci, co = (C, Cn) if restrict_ else (Cn, C)
    if restrict_:       # from 8 channels: two taps per 32-wide stage
        return (ci, co) in {(8, 16), (8, 8), (16, 32), (16, 16), (32, 64), (32, 32), (64, 64)}
    return (ci, co) in {(16, 8), (16, 16), (32, 16), (32, 32), (64, 32), (64, 64)}


def _block_supported(d, C, Cn):
    """Block prolongation: C_n in {16, 32, 64}, C = C_n or C_n / 2, all 2^d
    parity classes within one 256-column MMA."""
    return Cn in (16, 32, 64) and C in (Cn, Cn // 2) and (2 ** d) * 2 * C <= 256


def _line_supported(C, Cn, cx):
    """Line-staged restriction: from 8 channels to 8 or 16, coarse x extent a
    multiple of 32 (each warp's 32 coarse nodes on one line)."""
    return C == 8 and Cn in (8, 16) and cx >= 32 and cx % 32 == 0


def test_transfer_every_shape(case):
    """Restriction R_l and prolongation P_l in every kernel shape, the
    tensor-core ones (the last three shapes: per parity class, the block
    form of the prolongation, the line-staged restriction from 8 channels)
    included where the level allows them, against the oracle; then V-cycles
    with the tensor-core transfers forced on every level that has them."""
    from paper_2606_30495_b300 import mcmg
    prec, m, h = case
    w = m["w"]
    L = w["levels"]
    tol = _tols(prec)[0]
    # the last three shapes: the tensor-core transfer, then (prolongation
    # only) its block form over all parity classes, then (restriction only)
    # the line-staged form
    xts = mcmg.kernel_shape_count(mcmg.OP_RESTRICT) - 3
    blk = xts + 1
    line = xts + 2
    assert line == mcmg.kernel_shape_count(mcmg.OP_PROLONG) - 1
    d = len(m["shape"])
    ran_xts = 0
    ran_blk = 0
    ran_line = 0
    try:
        for l in range(L - 1):
            C, Cn = w["channels"][l], w["channels"][l + 1]
            shp = tuple(n >> l for n in m["shape"])
            cshp = tuple(n >> (l + 1) for n in m["shape"])
            lv = w["lvl"][l]
            r = I.complex_normal((2,) + shp + (C,), rng(70))
            zero = torch.zeros(r.shape, dtype=torch.complex64, device="cuda")
            want_r = np.stack([O.restrict(lv["R"], r[k]) for k in range(2)])
            ec = I.complex_normal((2,) + cshp + (Cn,), rng(71))
            e = I.complex_normal((2,) + shp + (C,), rng(72))
            want_p = np.stack([e[k] + O.prolong(lv["P"], ec[k], shp) for k in range(2)])
            for op, want in ((mcmg.OP_RESTRICT, want_r), (mcmg.OP_PROLONG, want_p)):
                ok_xts = _xts_supported(C, Cn, op == mcmg.OP_RESTRICT)
                for sh in range(mcmg.kernel_shape_count(op)):
                    ran = h.set_kernel_shape(l, op, sh)
                    if sh == xts:
                        assert ran == ok_xts, (l, op, C, Cn)
                    if sh == blk:
                        assert ran == (op == mcmg.OP_PROLONG and _block_supported(d, C, Cn)
                                       and prec in ("fp32tc", "bf16")), (l, op, C, Cn)
                    if sh == line:
                        assert ran == (op == mcmg.OP_RESTRICT and _line_supported(C, Cn, cshp[-1])
                                       and prec in ("fp32tc", "bf16")), (l, op, C, Cn)
                    if not ran:
                        continue
                    if op == mcmg.OP_RESTRICT:
                        rc = torch.zeros((2,) + cshp + (Cn,), dtype=torch.complex64, device="cuda")
                        h.residual_restrict(l, dev(r), zero, rc, nrhs=2)
                        got = host(rc)
                    else:
                        ef = dev(e)
                        h.prolong_add(l, dev(ec), ef, nrhs=2)
                        got = host(ef)
                    assert relerr(got, want) < tol, (l, op, sh)
                    ran_xts += sh == xts
                    ran_blk += sh == blk
                    ran_line += sh == line
                h.set_kernel_shape(l, op, -1)
        if any(_xts_supported(w["channels"][l], w["channels"][l + 1], rr)
               for l in range(L - 1) for rr in (True, False)):
            assert ran_xts > 0
            if any(_block_supported(d, w["channels"][l], w["channels"][l + 1])
                   for l in range(L - 1)):
                assert ran_blk > 0
            if any(_line_supported(w["channels"][l], w["channels"][l + 1],
                                   m["shape"][-1] >> (l + 1)) for l in range(L - 1)):
                assert ran_line > 0
            for l in range(L - 1):
                if not h.set_kernel_shape(l, mcmg.OP_RESTRICT, line):
                    h.set_kernel_shape(l, mcmg.OP_RESTRICT, xts)   # False where not available
                if not h.set_kernel_shape(l, mcmg.OP_PROLONG, blk):
                    h.set_kernel_shape(l, mcmg.OP_PROLONG, xts)
            rv = I.complex_normal((2,) + m["shape"], rng(73))
            want_v = np.stack([O.vcycle(w, m["feats"], ri) for ri in rv])
            ev = torch.zeros(rv.shape, dtype=torch.complex64, device="cuda")
            h.vcycle(dev(rv), ev, nrhs=2)
            assert relerr(host(ev), want_v) < _tols(prec)[1]
        assert h.device_error() == 0
    finally:
        for l in range(L - 1):
            for op in (mcmg.OP_RESTRICT, mcmg.OP_PROLONG):
                h.set_kernel_shape(l, op, -1)


@pytest.mark.parametrize("prec,shape,channels", [
    ("fp32tc", (94, 80, 70), [16, 32]),     # restriction 514.1 tiles, prolongation 8 classes
    ("fp32tc", (94, 80, 70), [8, 16]),      # restriction with two taps per stage
    ("bf16", (500, 330), [8, 16]),
    ("bf16", (94, 80, 70), [32, 32]),
    ("fp32tc", (62, 48, 40), [64, 64]),     # four K parts per tap (TF32)
    ("fp32tc", (500, 330), [16, 32]),       # 2D: 322.3 tiles, 4 classes
    ("bf16", (500, 330), [16, 16]),
    ("fp32tc", (70, 78, 64), [8, 16]),      # line-staged: 341.25 tiles, cx = 32
    ("fp32tc", (42, 40, 192), [8, 8]),      # line-staged: 315 tiles, three warps' lines per tile
    ("bf16", (702, 128), [8, 16]),          # line-staged 2D: 175.5 tiles
    ("fp32tc", (700, 256), [8, 16]),        # line-staged 2D: 350 tiles, a tile per coarse line
])
def test_transfer_ts_many_items(ctx, prec, shape, channels):
    """The tensor-core transfers with more items than CTAs (each persistent
    CTA walks several tiles and parity classes) and a ragged last tile,
    nrhs = 2, against the oracle, the prolongation also in its block form.
    Setup features are not needed: the restriction is taken through the
    residual with e = 0."""
    from paper_2606_30495_b300 import mcmg
    d = len(shape)
    pre, post = I.nu_schedule(2)
    w = I.make_weights(d, list(channels), pre, post, mode="random", seed=9)
    c = I.grf(shape, 4.0, 1.0, 3.0, rng(109))
    omega = I.omega_for_ppw(c.min(), 8.0, shape[0])
    h = mcmg.Handle(ctx, c, omega, 4, 1.0, w, precision=_prec(prec))
    xts = mcmg.kernel_shape_count(mcmg.OP_RESTRICT) - 3
    try:
        C, Cn = channels
        lv = w["lvl"][0]
        cshp = tuple(n >> 1 for n in shape)
        tol = _tols(prec)[0]
        rshapes = ([xts] if _xts_supported(C, Cn, True) else []) + \
            ([xts + 2] if _line_supported(C, Cn, cshp[-1]) else [])
        if rshapes:
            r = I.complex_normal((2,) + shape + (C,), rng(80))
            want = np.stack([O.restrict(lv["R"], r[k]) for k in range(2)])
        for sh in rshapes:
            assert h.set_kernel_shape(0, mcmg.OP_RESTRICT, sh)
            rc = torch.full((2,) + cshp + (Cn,), float("nan"), dtype=torch.complex64,
                            device="cuda")
            h.residual_restrict(0, dev(r), torch.zeros(r.shape, dtype=torch.complex64,
                                                       device="cuda"), rc, nrhs=2)
            assert relerr(host(rc), want) < tol, sh
        ec = I.complex_normal((2,) + cshp + (Cn,), rng(81))
        e = I.complex_normal((2,) + shape + (C,), rng(82))
        want = np.stack([e[k] + O.prolong(lv["P"], ec[k], shape) for k in range(2)])
        shapes = ([xts] if _xts_supported(C, Cn, False) else []) + \
            ([xts + 1] if _block_supported(d, C, Cn) else [])
        for sh in shapes:
            assert h.set_kernel_shape(0, mcmg.OP_PROLONG, sh)
            ef = dev(e)
            h.prolong_add(0, dev(ec), ef, nrhs=2)
            assert relerr(host(ef), want) < tol, sh
        assert h.device_error() == 0
    finally:
        h.close()


def test_vcycle_one_field(case):
    """One-field V-cycles: where level 0 runs the small-channel tensor-core
    step (C_0 = 8, or 16 with FP32-accurate mixing) the lift and the
    projection are folded into its steps (input and output addresses through
    device cells of the captured graph); two calls with different buffers
    check that the graph follows them."""
    prec, m, h = case
    for seed in (44, 45):
        r = I.complex_normal(m["shape"], rng(seed))
        want = O.vcycle(m["w"], m["feats"], r)
        e = torch.zeros(r.shape, dtype=torch.complex64, device="cuda")
        h.vcycle(dev(r), e)
        assert relerr(host(e), want) < _tols(prec)[1], seed


def test_vcycle(case):
    prec, m, h = case
    r = I.complex_normal((2,) + m["shape"], rng(40))
    want = np.stack([O.vcycle(m["w"], m["feats"], ri) for ri in r])
    e = torch.zeros(r.shape, dtype=torch.complex64, device="cuda")
    h.vcycle(dev(r), e, nrhs=2)
    assert relerr(host(e), want) < _tols(prec)[1]


@pytest.mark.parametrize("prec,shape,channels", [
    ("fp32tc", (254, 162), [16, 16]),       # 322 tiles over 2 CTAs per SM
    ("fp32tc", (60, 66, 42), [8, 8]),       # 1300 tiles over 4 CTAs per SM, ragged
    ("bf16", (60, 66, 42), [8, 8]),         # 1300 tiles over 8 CTAs per SM, ragged
    ("fp32tc", (160, 130), [64, 64]),       # 163 tiles over one CTA per SM, ragged
    ("fp32tc", (34, 32, 30), [32, 32]),     # 255 tiles over one CTA per SM, ragged
    ("bf16", (160, 130), [64, 64]),
])
def test_persistent_multi_tile(ctx, prec, shape, channels):
    """More tiles than CTAs: each persistent CTA walks several tiles."""
    m = model(shape, channels, mode="random", seed=8)
    h = handle(ctx, m, _prec(prec))
    try:
        for first in (True, False):
            _check_step(prec, m, h, 0, first, nrhs=1, seed=50)
        w = m["w"]
        a, _ = m["feats"][0]
        lv = w["lvl"][0]
        C, Cn = w["channels"][0], w["channels"][1]
        r = I.complex_normal(shape + (C,), rng(60))
        e = I.complex_normal(shape + (C,), rng(61))
        rc = torch.zeros(tuple(n >> 1 for n in shape) + (Cn,), dtype=torch.complex64, device="cuda")
        h.residual_restrict(0, dev(r), dev(e), rc, nrhs=1)
        want = O.restrict(lv["R"], r - O.op_A(lv, a, e))
        assert relerr(host(rc), want) < _tols(prec)[0]
        assert h.device_error() == 0
    finally:
        h.close()


def test_fp32tc_full_size_256_vcycle_and_solve(ctx):
    """The 256^2 workload with FP32-accurate tensor-core mixing: V-cycle within
    1e-5 of the oracle, and the solve within 10% of the stored oracle
    iteration count with the true FP64 residual at 1e-6."""
    import json
    import os
    from paper_2606_30495_b300 import mcmg
    m = workload_model("helm2d_n256_grf")
    feats = O.setup(m["q"], m["w"])
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                    "oracle_solves.json")))["helm2d_n256_grf"]
    h = handle(ctx, m, mcmg.FP32_TC)
    try:
        for r in (I.point_source(m["shape"]), I.complex_normal(m["shape"], rng(6))):
            want = O.vcycle(m["w"], feats, r)
            e = torch.zeros(m["shape"], dtype=torch.complex64, device="cuda")
            h.vcycle(dev(r), e)
            assert relerr(host(e), want) < TOL32
        f = I.point_source(m["shape"])
        u = torch.zeros(m["shape"], dtype=torch.complex128, device="cuda")
        st, info = h.solve(dev(f, torch.complex128), u, tol=1e-6, restart_m=g["restart"],
                           max_iters=4000)
        assert st == 0 and info["converged"], info
        res = np.linalg.norm(f - O.apply_A(m["q"], host(u))) / np.linalg.norm(f)
        assert res <= 1e-6, res
        assert abs(info["iters"] - g["iters"]) <= 0.1 * g["iters"], (info, g)
        assert h.device_error() == 0
    finally:
        h.close()
