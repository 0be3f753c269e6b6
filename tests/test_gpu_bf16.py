"""Parity of the tensor-core (tcgen05, BF16 operands, FP32 accumulation)
smoothing step and V-cycle with the FP64 oracle.

Bound: 2e-2 relative L2 for a BF16 V-cycle application (the north-star
tolerance for BF16 channel mixing); a single smoothing step is held to 1e-2.
Every bounded wait inside the kernel must have finished (error word 0).
"""
import numpy as np
import pytest

from oracle import mcmg_oracle as O
from paper_2606_30495_b300 import inputs as I
from tests._models import model, relerr, rng, workload_model

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_STEP = 1e-2
TOL_VCYCLE = 2e-2


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


def handle_bf16(ctx, m):
    from paper_2606_30495_b300 import mcmg
    return mcmg.Handle(ctx, m["c"], m["omega"], m["sponge"], m["gamma_max"], m["w"],
                       precision=mcmg.BF16)


CASES = [
    ((34, 30), [8, 16], "random"),
    ((20, 36), [16, 32], "random"),
    ((18, 14), [32, 64], "random"),
    ((16, 12), [64, 64], "random"),
    ((34, 30), [8, 16], "structured"),
    ((6, 8, 10), [8, 16], "random"),
    ((4, 6, 8), [32, 64], "random"),
]
IDS = [f"{'x'.join(map(str, s))}-C{'-'.join(map(str, c))}-{m}" for s, c, m in CASES]


@pytest.fixture(scope="module", params=CASES, ids=IDS)
def case(request, ctx):
    shape, channels, mode = request.param
    m = model(shape, channels, mode=mode, seed=5)
    h = handle_bf16(ctx, m)
    yield m, h
    assert h.device_error() == 0
    h.close()


@pytest.mark.parametrize("first", [True, False])
def test_tc_smooth_step(case, first):
    m, h = case
    w = m["w"]
    for l in range(w["levels"]):
        C = w["channels"][l]
        shp = tuple(n >> l for n in m["shape"]) + (C,)
        a, s = m["feats"][l]
        nsteps = w["nu_pre"][l] + w["nu_post"][l]
        for step in sorted({0, nsteps - 1}):
            r = I.complex_normal((2,) + shp, rng(10 + step))
            e_in = None if first else I.complex_normal((2,) + shp, rng(20 + step))
            out = torch.zeros(r.shape, dtype=torch.complex64, device="cuda")
            h.smooth(l, step, dev(r), None if first else dev(e_in), out, nrhs=2)
            want = []
            for k in range(2):
                e0 = np.zeros(shp, complex) if first else e_in[k]
                want.append(e0 + O.op_S(w["lvl"][l], s, step, r[k] - O.op_A(w["lvl"][l], a, e0)))
            err = relerr(host(out), np.stack(want))
            assert err < TOL_STEP, (l, step, err)
            assert err > 1e-7 or C < 8, "BF16 path expected to differ from FP64 at BF16 level"


def test_tc_vcycle(case):
    m, h = case
    r = I.complex_normal((2,) + m["shape"], rng(40))
    want = np.stack([O.vcycle(m["w"], m["feats"], ri) for ri in r])
    e = torch.zeros(r.shape, dtype=torch.complex64, device="cuda")
    h.vcycle(dev(r), e, nrhs=2)
    assert relerr(host(e), want) < TOL_VCYCLE


def test_tc_workload_vcycle_256(ctx):
    """The 256^2 workload's weights with BF16 channel mixing."""
    m = workload_model("helm2d_n256_grf")
    feats = O.setup(m["q"], m["w"])
    h = handle_bf16(ctx, m)
    try:
        for r in (I.point_source(m["shape"]), I.complex_normal(m["shape"], rng(6))):
            want = O.vcycle(m["w"], feats, r)
            e = torch.zeros(m["shape"], dtype=torch.complex64, device="cuda")
            h.vcycle(dev(r), e)
            assert relerr(host(e), want) < TOL_VCYCLE
        assert h.device_error() == 0
    finally:
        h.close()


def test_tc_residual_restrict(case):
    """Residual r - A_l(e) and restriction on a BF16 handle (the residual runs
    on the tensor cores for C_l <= 32, on the CUDA cores in FP32 above)."""
    m, h = case
    w = m["w"]
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
        assert relerr(host(rc), want) < TOL_STEP
