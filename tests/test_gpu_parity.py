"""Parity of the CUDA path with the FP64 oracle, step by step and end to end.

Every call goes through the C ABI (the ctypes binding).  Tolerances: the FP32
path within 1e-5 relative L2 of the oracle per application (the FP32 V-cycle
bound), FP64 kernels within 1e-13; solves reach the true FP64 relative
residual 1e-6 with iteration counts within 10% of the oracle's.
Sizes span several thread blocks with ragged tails and every supported
channel count.
"""
import numpy as np
import pytest

from oracle import mcmg_oracle as O
from paper_2606_30495_b300 import inputs as I
from tests._models import model, relerr, rng, workload_model

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.fixture(scope="module")
def ctx():
    from paper_2606_30495_b300 import mcmg
    c = mcmg.Context(0)
    yield c
    c.close()


def dev(a, dtype=None):
    a = np.ascontiguousarray(a)
    if dtype is None:
        dtype = torch.complex64
    return torch.from_numpy(a).to(device="cuda", dtype=dtype).contiguous()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.complex128)


def handle(ctx, m):
    from paper_2606_30495_b300 import mcmg
    return mcmg.Handle(ctx, m["c"], m["omega"], m["sponge"], m["gamma_max"], m["w"])


CASES = [
    ((36, 20), [1, 2], "random"),
    ((24, 40), [4, 8], "random"),
    ((34, 30), [8, 16], "random"),
    ((18, 34), [16, 32], "random"),
    ((12, 20), [32, 64], "random"),
    ((10, 6), [64, 64], "random"),
    ((34, 30), [8, 16], "structured"),
    ((8, 6, 10), [2, 4], "random"),
    ((6, 8, 4), [8, 16], "random"),
    ((4, 6, 4), [32, 64], "random"),
]
IDS = [f"{'x'.join(map(str, s))}-C{'-'.join(map(str, c))}-{m}" for s, c, m in CASES]


@pytest.fixture(scope="module", params=CASES, ids=IDS)
def case(request, ctx):
    shape, channels, mode = request.param
    m = model(shape, channels, mode=mode, seed=3)
    h = handle(ctx, m)
    yield m, h
    h.close()


def test_apply_A(case):
    m, h = case
    x = I.complex_normal((2,) + m["shape"], rng(1))
    want = np.stack([O.apply_A(m["q"], xi) for xi in x])
    y32 = torch.zeros(x.shape, dtype=torch.complex64, device="cuda")
    h.apply_A(dev(x), y32, fp64=False, nrhs=2)
    assert relerr(host(y32), want) < 1e-6
    y64 = torch.zeros(x.shape, dtype=torch.complex128, device="cuda")
    h.apply_A(dev(x, torch.complex128), y64, fp64=True, nrhs=2)
    assert relerr(host(y64), want) < 1e-13


def test_setup_features(case):
    m, h = case
    for l, (a, s) in enumerate(m["feats"]):
        for which, ref in ((0, a), (1, s)):
            out = torch.zeros(ref.shape, dtype=torch.complex64, device="cuda")
            h.get_feature(l, which, out)
            assert relerr(host(out), ref) < TOL32, (l, which)


def test_lift_project(case):
    m, h = case
    w = m["w"]
    r = I.complex_normal((3,) + m["shape"], rng(2))
    r1 = torch.zeros((3,) + m["shape"] + (w["channels"][0],), dtype=torch.complex64, device="cuda")
    h.lift(dev(r), r1, nrhs=3)
    want = np.stack([ri[..., None] * w["lift"] for ri in r])
    assert relerr(host(r1), want) < 1e-6
    e1 = I.complex_normal(want.shape, rng(3))
    e = torch.zeros(r.shape, dtype=torch.complex64, device="cuda")
    h.project(dev(e1), e, nrhs=3)
    assert relerr(host(e), e1 @ w["proj"]) < 1e-6


@pytest.mark.parametrize("first", [True, False])
def test_smooth_step(case, first):
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
            assert relerr(host(out), np.stack(want)) < TOL32, (l, step)


def test_residual_restrict_and_prolong(case):
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
        assert relerr(host(rc), want) < TOL32
        ec = I.complex_normal((2,) + cshp + (Cn,), rng(32))
        ef = dev(e)
        h.prolong_add(l, dev(ec), ef, nrhs=2)
        want = np.stack([e[k] + O.prolong(lv["P"], ec[k], shp) for k in range(2)])
        assert relerr(host(ef), want) < TOL32


def test_every_kernel_shape(case):
    """Every CUDA-core kernel and thread shape of the four V-cycle operations
    against the oracle: the smoothing step (with e and with e = 0), the
    residual, the restriction and the prolongation.  Setup's autotuner picks
    among them by timing, so each must be exact on its own; grids here leave
    ragged last blocks for every shape."""
    from paper_2606_30495_b300 import mcmg
    m, h = case
    w = m["w"]
    L = w["levels"]
    ran = {op: set() for op in range(4)}
    try:
        for l in range(L):
            C = w["channels"][l]
            shp = tuple(n >> l for n in m["shape"]) + (C,)
            a, s = m["feats"][l]
            lv = w["lvl"][l]
            step = w["nu_pre"][l] + w["nu_post"][l] - 1
            r = I.complex_normal((2,) + shp, rng(50))
            e_in = I.complex_normal((2,) + shp, rng(51))
            want = np.stack([e_in[k] + O.op_S(lv, s, step, r[k] - O.op_A(lv, a, e_in[k]))
                             for k in range(2)])
            want0 = np.stack([O.op_S(lv, s, 0, r[k]) for k in range(2)])
            for sh in range(mcmg.kernel_shape_count(mcmg.OP_SMOOTH)):
                if not h.set_kernel_shape(l, mcmg.OP_SMOOTH, sh):
                    continue
                ran[0].add(sh)
                out = torch.zeros(r.shape, dtype=torch.complex64, device="cuda")
                h.smooth(l, step, dev(r), dev(e_in), out, nrhs=2)
                assert relerr(host(out), want) < TOL32, (l, sh)
                out.zero_()
                h.smooth(l, 0, dev(r), None, out, nrhs=2)
                assert relerr(host(out), want0) < TOL32, (l, sh, "e = 0")
            h.set_kernel_shape(l, mcmg.OP_SMOOTH, -1)
            if l == L - 1:
                continue
            cshp = tuple(n >> (l + 1) for n in m["shape"]) + (w["channels"][l + 1],)
            want_rc = np.stack([O.restrict(lv["R"], r[k] - O.op_A(lv, a, e_in[k])) for k in range(2)])
            for op in (mcmg.OP_RESIDUAL, mcmg.OP_RESTRICT):
                for sh in range(mcmg.kernel_shape_count(op)):
                    if not h.set_kernel_shape(l, op, sh):
                        continue
                    ran[op].add(sh)
                    rc = torch.zeros((2,) + cshp, dtype=torch.complex64, device="cuda")
                    h.residual_restrict(l, dev(r), dev(e_in), rc, nrhs=2)
                    assert relerr(host(rc), want_rc) < TOL32, (l, op, sh)
                h.set_kernel_shape(l, op, -1)
            ec = I.complex_normal((2,) + cshp, rng(53))
            want_p = np.stack([e_in[k] + O.prolong(lv["P"], ec[k], shp[:-1]) for k in range(2)])
            for sh in range(mcmg.kernel_shape_count(mcmg.OP_PROLONG)):
                if not h.set_kernel_shape(l, mcmg.OP_PROLONG, sh):
                    continue
                ran[3].add(sh)
                ef = dev(e_in)
                h.prolong_add(l, dev(ec), ef, nrhs=2)
                assert relerr(host(ef), want_p) < TOL32, (l, "prolong", sh)
            h.set_kernel_shape(l, mcmg.OP_PROLONG, -1)
        assert len(ran[0]) >= 3 and len(ran[1]) >= 3 and 0 in ran[2] and 0 in ran[3]
        if max(w["channels"]) >= 4:
            assert ran[0] & set(range(6, mcmg.kernel_shape_count(0))), "no register-tiled smoothing"
        pairs = [(w["channels"][l], w["channels"][l + 1]) for l in range(L - 1)]
        if any(cf >= 4 and cc in (cf, 2 * cf) for cf, cc in pairs):
            assert len(ran[2]) > 1 and len(ran[3]) > 1, "no register-tiled transfer"
        # V-cycles with the register-tiled shapes forced on every level and
        # operation (the captured graph must follow each change)
        rv = I.complex_normal((2,) + m["shape"], rng(52))
        want_v = np.stack([O.vcycle(w, m["feats"], ri) for ri in rv])
        for k in range(1, 13):
            for l in range(L):
                for op in range(4 if l < L - 1 else 2):
                    n_op = mcmg.kernel_shape_count(op)
                    sh = (5 + k) % n_op if op < 2 else k % n_op
                    h.set_kernel_shape(l, op, sh)
            ev = torch.zeros(rv.shape, dtype=torch.complex64, device="cuda")
            h.vcycle(dev(rv), ev, nrhs=2)
            assert relerr(host(ev), want_v) < TOL32, k
    finally:
        for l in range(L):
            for op in range(4 if l < L - 1 else 2):
                h.set_kernel_shape(l, op, -1)


def test_coarse_basis(case):
    """Raw coarse-basis response (Eq. coarse_basis) through the C ABI against
    the oracle, for random (level, node, channel) on every case; out-of-range
    arguments are refused."""
    from paper_2606_30495_b300 import mcmg
    m, h = case
    w = m["w"]
    g = rng(60)
    out = torch.zeros(m["shape"], dtype=torch.complex64, device="cuda")
    for level in range(1, w["levels"]):
        cshape = tuple(n >> level for n in m["shape"])
        for _ in range(2):
            idx = tuple(int(g.integers(0, n)) for n in cshape)
            ch = int(g.integers(0, w["channels"][level]))
            h.coarse_basis(level, int(np.ravel_multi_index(idx, cshape)), ch, out)
            want = O.coarse_basis(w, level, idx, ch, m["shape"])
            assert relerr(host(out), want) < TOL32, (level, idx, ch)
    for bad in ((0, 0, 0), (w["levels"], 0, 0), (1, -1, 0), (1, 0, w["channels"][1])):
        with pytest.raises(mcmg.McmgError):
            h.coarse_basis(*bad, out)


def test_vcycle_and_batch(case):
    m, h = case
    r = I.complex_normal((3,) + m["shape"], rng(40))
    want = np.stack([O.vcycle(m["w"], m["feats"], ri) for ri in r])
    e = torch.zeros(r.shape, dtype=torch.complex64, device="cuda")
    h.vcycle(dev(r), e, nrhs=3)
    got = host(e)
    assert relerr(got, want) < TOL32
    e1 = torch.zeros(m["shape"], dtype=torch.complex64, device="cuda")
    h.vcycle(dev(r[1]), e1, nrhs=1)
    assert relerr(host(e1), want[1]) < TOL32
    # batched and single application agree to rounding (same kernels, same order)
    assert np.max(np.abs(host(e1) - got[1])) <= 1e-6 * np.max(np.abs(got[1]))


def test_vcycle_linearity_on_gpu(case):
    m, h = case
    g = rng(41)
    r1, r2 = I.complex_normal(m["shape"], g), I.complex_normal(m["shape"], g)
    al, be = 0.3 - 1.2j, -0.7 + 0.4j
    outs = []
    for r in (al * r1 + be * r2, r1, r2):
        e = torch.zeros(m["shape"], dtype=torch.complex64, device="cuda")
        h.vcycle(dev(r), e)
        outs.append(host(e))
    assert relerr(outs[0], al * outs[1] + be * outs[2]) < 3 * TOL32


@pytest.mark.parametrize("name", ["helm2d_n64_homogeneous", "helm2d_n64_slmg"])
def test_vcycle_workloads_64(ctx, name):
    m = workload_model(name)
    feats = O.setup(m["q"], m["w"])
    h = handle(ctx, m)
    try:
        for r in (I.point_source(m["shape"]), I.complex_normal(m["shape"], rng(5))):
            want = O.vcycle(m["w"], feats, r)
            e = torch.zeros(m["shape"], dtype=torch.complex64, device="cuda")
            h.vcycle(dev(r), e)
            assert relerr(host(e), want) < TOL32
    finally:
        h.close()


def test_cgs2_against_projection(case):
    m, h = case
    n = int(np.prod(m["shape"]))
    k = 13
    Q, _ = np.linalg.qr(I.complex_normal((n, k), rng(50)))
    V = np.ascontiguousarray(Q.T)
    w = I.complex_normal(n, rng(51))
    Vd, wd = dev(V), dev(w)
    hh, nrm = h.cgs2(Vd, wd)
    V32 = V.astype(np.complex64).astype(np.complex128)
    w32 = w.astype(np.complex64).astype(np.complex128)
    h_exact = V32.conj() @ w32
    resid = w32 - V32.T @ h_exact
    assert relerr(hh, h_exact) < 1e-6
    assert abs(nrm - np.linalg.norm(resid)) < 1e-5 * np.linalg.norm(resid)
    assert relerr(host(wd), resid) < 1e-5


def _oracle_solve(m, restart):
    A = lambda u: O.apply_A(m["q"], u)
    feats = O.setup(m["q"], m["w"])
    f = I.point_source(m["shape"])
    return O.fgmres(A, lambda v: O.vcycle(m["w"], feats, v), f, m=restart, tol=1e-6,
                    max_iters=2000)


def _gpu_solve_check(ctx, m, restart, oracle_iters, max_iters=4000):
    h = handle(ctx, m)
    try:
        f = I.point_source(m["shape"])
        u = torch.zeros(m["shape"], dtype=torch.complex128, device="cuda")
        st, info = h.solve(dev(f, torch.complex128), u, tol=1e-6, restart_m=restart,
                           max_iters=max_iters)
        assert st == 0 and info["converged"], info
        un = host(u)
        res = np.linalg.norm(f - O.apply_A(m["q"], un)) / np.linalg.norm(f)
        assert res <= 1e-6, res                             # against the FP64 operator
        assert abs(info["rel_residual"] - res) <= 1e-3 * res
        assert abs(info["iters"] - oracle_iters) <= 0.1 * oracle_iters, (info, oracle_iters)
        return info
    finally:
        h.close()


@pytest.mark.parametrize("name", ["helm2d_n64_slmg", "helm2d_n64_homogeneous"])
def test_solve_matches_oracle_iterations_and_residual(ctx, name):
    m = workload_model(name)
    restart = m["wl"]["restart"]
    _, oinfo = _oracle_solve(m, restart)
    assert oinfo["converged"]
    _gpu_solve_check(ctx, m, restart, oinfo["iters"])


def _golden(name):
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_solves.json")
    d = json.load(open(path))
    return d[name]


def test_full_size_256_solve_against_stored_oracle_count(ctx):
    """The 256^2 workload at full size: iteration count against the stored
    oracle solve (tests/golden/make_oracle_solves.py), residual against the
    oracle's FP64 operator."""
    m = workload_model("helm2d_n256_grf")
    g = _golden("helm2d_n256_grf")
    assert g["converged"] and g["restart"] == m["wl"]["restart"]
    _gpu_solve_check(ctx, m, g["restart"], g["iters"])


def test_full_size_256_vcycle(ctx):
    m = workload_model("helm2d_n256_grf")
    feats = O.setup(m["q"], m["w"])
    h = handle(ctx, m)
    try:
        for r in (I.point_source(m["shape"]), I.complex_normal(m["shape"], rng(6))):
            want = O.vcycle(m["w"], feats, r)
            e = torch.zeros(m["shape"], dtype=torch.complex64, device="cuda")
            h.vcycle(dev(r), e)
            assert relerr(host(e), want) < TOL32
    finally:
        h.close()


def test_solve_restarted_small_problem(ctx):
    m = model((24, 24), [2, 4], mode="structured", seed=1, ppw=12.0, sponge=4)
    A = lambda u: O.apply_A(m["q"], u)
    f = I.point_source(m["shape"])
    _, oinfo = O.fgmres(A, lambda v: O.vcycle(m["w"], m["feats"], v), f, m=10, tol=1e-6,
                        max_iters=3000)
    h = handle(ctx, m)
    try:
        u = torch.zeros(m["shape"], dtype=torch.complex128, device="cuda")
        st, info = h.solve(dev(f, torch.complex128), u, tol=1e-6, restart_m=10, max_iters=3000)
        res = np.linalg.norm(f - O.apply_A(m["q"], host(u))) / np.linalg.norm(f)
        assert oinfo["converged"] == bool(info["converged"])
        if oinfo["converged"]:
            assert res <= 1e-6
            assert abs(info["iters"] - oinfo["iters"]) <= max(0.1 * oinfo["iters"], 2)
    finally:
        h.close()


def test_solve_host_buffers_match_device(ctx):
    m = workload_model("helm2d_n64_slmg")
    h = handle(ctx, m)
    try:
        f = I.point_source(m["shape"])
        u = torch.zeros(m["shape"], dtype=torch.complex128, device="cuda")
        st, info = h.solve(dev(f, torch.complex128), u, tol=1e-6, restart_m=20)
        uh = np.zeros(m["shape"], dtype=np.complex128)
        st2, info2 = h.solve_host(np.ascontiguousarray(f), uh, tol=1e-6, restart_m=20)
        assert st == st2 == 0 and info["iters"] == info2["iters"]
        assert np.max(np.abs(uh - host(u))) <= 1e-12 * np.max(np.abs(uh))
    finally:
        h.close()


def test_errors_are_reported(ctx):
    from paper_2606_30495_b300 import mcmg
    m = model((12, 12), [2, 4], mode="random", seed=0)
    with pytest.raises(mcmg.McmgError) as ei:          # 3 levels need divisibility by 4
        bad = dict(m["w"])
        w3 = I.make_weights(2, [2, 2, 2], *I.nu_schedule(3), mode="random")
        mcmg.Handle(ctx, np.ones((10, 12)), 10.0, 2, 1.0, w3)
    assert ei.value.status == -2
    w5 = I.make_weights(2, [2, 3], *I.nu_schedule(2), mode="random")   # 3 channels unsupported
    with pytest.raises(mcmg.McmgError) as ei:
        mcmg.Handle(ctx, np.ones((12, 12)), 10.0, 2, 1.0, w5)
    assert ei.value.status == -2
    h = handle(ctx, m)
    try:
        x = torch.zeros((12, 12), dtype=torch.complex64, device="cuda")
        with pytest.raises(mcmg.McmgError) as ei:
            h.vcycle(x, x.clone(), nrhs=0)
        assert ei.value.status == -1
        with pytest.raises(mcmg.McmgError):
            h.smooth(5, 0, x, None, x.clone())
    finally:
        h.close()


@pytest.mark.parametrize("name", ["helm2d_n64_homogeneous", "helm2d_n64_slmg"])
def test_stationary_iteration_matches_oracle(ctx, name):
    """The stationary McMg iteration (Eq. mcmg_iteration): the iterate u and
    its true residual after k = 1..6 V-cycles match the oracle's, u element
    by element."""
    m = workload_model(name)
    feats = O.setup(m["q"], m["w"])
    f = I.point_source(m["shape"])
    _, oinfo = O.stationary_solve(lambda u: O.apply_A(m["q"], u),
                                  lambda v: O.vcycle(m["w"], feats, v), f, tol=1e-30, max_iters=6)
    h = handle(ctx, m)
    try:
        from paper_2606_30495_b300 import mcmg
        for k in range(1, 7):
            u = torch.zeros(m["shape"], dtype=torch.complex128, device="cuda")
            st, info = h.solve(dev(f, torch.complex128), u, tol=1e-30, restart_m=1, max_iters=k,
                               flags=mcmg.SOLVE_STATIONARY)
            assert st == -5 and info["iters"] == k
            want = oinfo["history"][k]
            assert abs(info["rel_residual"] - want) <= 1e-4 * want, (k, info, want)
            res = np.linalg.norm(f - O.apply_A(m["q"], host(u))) / np.linalg.norm(f)
            assert abs(res - want) <= 1e-4 * want
            uk, _ = O.stationary_solve(lambda v: O.apply_A(m["q"], v),
                                       lambda v: O.vcycle(m["w"], feats, v), f, tol=1e-30,
                                       max_iters=k)
            assert relerr(host(u), uk) < 1e-4, k
    finally:
        h.close()


def test_multi_rhs_block_solve_equals_single_solves(ctx):
    """Several right-hand sides solved together (V-cycles batched into one
    launch per level) give the same iterates as solving them one by one."""
    m = workload_model("helm2d_n64_homogeneous")
    g = rng(77)
    f = I.random_point_sources(m["shape"], 8, 3, g)
    h = handle(ctx, m)
    try:
        ub = torch.zeros(f.shape, dtype=torch.complex128, device="cuda")
        st, info = h.solve(dev(f, torch.complex128), ub, tol=1e-6, restart_m=20, nrhs=3)
        assert st == 0 and info["converged"]
        blk = host(ub)
        iters = []
        for k in range(3):
            u = torch.zeros(m["shape"], dtype=torch.complex128, device="cuda")
            st1, i1 = h.solve(dev(f[k], torch.complex128), u, tol=1e-6, restart_m=20)
            assert st1 == 0
            iters.append(i1["iters"])
            one = host(u)
            assert np.max(np.abs(blk[k] - one)) <= 1e-12 * np.max(np.abs(one))
            res = np.linalg.norm(f[k] - O.apply_A(m["q"], blk[k])) / np.linalg.norm(f[k])
            assert res <= 1e-6
        assert info["iters"] == max(iters)
    finally:
        h.close()


@pytest.mark.parametrize("name", ["helm2d_n64_homogeneous", "helm2d_n64_slmg"])
def test_born_iteration_matches_oracle(ctx, name):
    """Born+McMg (Appendix, Born-series variant): the iterate u and its true
    residual after k = 1..5 Born steps u <- u + MG(G(f - A u)), G applied by
    FFT with the discrete-Laplacian symbol, match the oracle's, u element by
    element."""
    from paper_2606_30495_b300 import mcmg
    m = workload_model(name)
    feats = O.setup(m["q"], m["w"])
    f = I.point_source(m["shape"])
    q0 = O.born_background(m["q"])
    _, oinfo = O.born_solve(lambda u: O.apply_A(m["q"], u), lambda v: O.apply_G(q0, v),
                            lambda v: O.vcycle(m["w"], feats, v), f, tol=1e-30, max_iters=5)
    h = handle(ctx, m)
    try:
        for k in range(1, 6):
            u = torch.zeros(m["shape"], dtype=torch.complex128, device="cuda")
            st, info = h.solve(dev(f, torch.complex128), u, tol=1e-30, restart_m=1, max_iters=k,
                               flags=mcmg.SOLVE_BORN)
            assert st == -5 and info["iters"] == k
            want = oinfo["history"][k]
            assert abs(info["rel_residual"] - want) <= 1e-4 * want, (k, info, want)
            res = np.linalg.norm(f - O.apply_A(m["q"], host(u))) / np.linalg.norm(f)
            assert abs(res - want) <= 1e-4 * want
            uk, _ = O.born_solve(lambda v: O.apply_A(m["q"], v), lambda v: O.apply_G(q0, v),
                                 lambda v: O.vcycle(m["w"], feats, v), f, tol=1e-30, max_iters=k)
            assert relerr(host(u), uk) < 1e-4, k
        # the server runs FGMRES only
        with pytest.raises(mcmg.McmgError):
            ctx.submit(h, dev(f, torch.complex128), torch.zeros(m["shape"], dtype=torch.complex128,
                       device="cuda"), tol=1e-6, restart_m=1, max_iters=2, flags=mcmg.SOLVE_BORN)
    finally:
        h.close()


@pytest.mark.parametrize("shape", [(64, 64), (32, 128), (16, 8, 32), (4096, 4)])
def test_green_operator_matches_oracle(ctx, shape):
    """The Born-series Green operator G = (-Delta_h - k0^2)^{-1} through this
    library's FFT (Appendix, Eq. discrete_symbol) against the oracle's numpy
    FFT form, element by element at FP64 rounding (1e-12)."""
    d = len(shape)
    chans = [2, 4] if min(shape) >= 8 else [2]
    m = model(shape, chans, mode="random", seed=3, sponge=2 if min(shape) >= 8 else 1)
    q0 = O.born_background(m["q"])
    h = handle(ctx, m)
    try:
        for s in (0, 1):
            x = I.complex_normal(shape, rng(90 + s))
            xd = dev(x, torch.complex128)
            h.apply_G(xd)
            assert relerr(host(xd), O.apply_G(q0, x)) < 1e-12
    finally:
        h.close()


def test_green_operator_needs_power_of_two_axes(ctx):
    from paper_2606_30495_b300 import mcmg
    m = model((24, 16), [2, 2], mode="random", seed=3, sponge=2)
    h = handle(ctx, m)
    try:
        x = torch.zeros((24, 16), dtype=torch.complex128, device="cuda")
        with pytest.raises(mcmg.McmgError) as ei:
            h.apply_G(x)
        assert ei.value.status == -2
    finally:
        h.close()
