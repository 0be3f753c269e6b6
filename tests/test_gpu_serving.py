"""The request server (mcmg_submit / mcmg_poll): each result is the same alone
and in the mix, admission respects the HBM budget, and a request that can
never fit is refused."""
import time

import numpy as np
import pytest

from oracle import mcmg_oracle as O
from paper_2606_30495_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _requests():
    base = I.serving_weights()
    out = []
    for i, (n, nrhs) in enumerate([(64, 2), (128, 1), (64, 3), (128, 2)]):
        req = dict(id=i, n=n, nrhs=nrhs, medium_seed=500 + i, levels=I.serving_levels(max(n, 64)) - 0)
        req["levels"] = 3 if n == 64 else 4
        out.append((req,) + I.serving_request_inputs(req, base))
    return out


def _handles(ctx, reqs, precision):
    from paper_2606_30495_b300 import mcmg
    return [mcmg.Handle(ctx, c, om, 16, 1.0, w, precision=precision) for (_, c, om, w, _) in reqs]


def _run_mix(ctx, hs, reqs):
    from paper_2606_30495_b300 import mcmg
    fs = [torch.from_numpy(f).cuda() for (_, _, _, _, f) in reqs]
    us = [torch.zeros_like(x) for x in fs]
    tickets = [ctx.submit(h, fd, u, tol=1e-6, restart_m=30, max_iters=3000, nrhs=r[0]["nrhs"])
               for h, fd, u, r in zip(hs, fs, us, reqs)]
    done = {}
    t0 = time.time()
    while len(done) < len(tickets) and time.time() - t0 < 120:
        for t in tickets:
            if t not in done:
                st, info = ctx.poll(t)
                if st != mcmg.MCMG_PENDING:
                    done[t] = (st, info)
        time.sleep(0.002)
    assert len(done) == len(tickets)
    out = []
    for k, t in enumerate(tickets):
        st, info = done[t]
        assert st == 0 and info["converged"]
        out.append(us[k].cpu().numpy())
    return out


def test_server_results_equal_alone_and_in_the_mix():
    """Each request's solution is the same alone (mcmg_solve), in the mix with
    cross-request batching (the V-cycles of requests on 64^2 and 128^2 grids,
    3 and 4 levels of one model, run as cohorts: one tensor-core launch per
    level and step for all of them) and in the mix without it."""
    from paper_2606_30495_b300 import mcmg
    ctx = mcmg.Context(0)
    reqs = _requests()
    hs = _handles(ctx, reqs, mcmg.BF16)
    try:
        alone = []
        for h, (req, c, om, w, f) in zip(hs, reqs):
            fd = torch.from_numpy(f).cuda()
            u = torch.zeros_like(fd)
            st, info = h.solve(fd, u, tol=1e-6, restart_m=30, max_iters=3000, nrhs=req["nrhs"])
            assert st == 0 and info["converged"], info
            alone.append(u.cpu().numpy())
        r0, m0 = ctx.batching(True)
        batched = _run_mix(ctx, hs, reqs)
        r1, m1 = ctx.batching()
        assert r1 > r0 and m1 - m0 >= 2 * (r1 - r0), (r0, m0, r1, m1)   # cohorts were formed
        ctx.batching(False)
        apart = _run_mix(ctx, hs, reqs)
        assert ctx.batching()[0] == r1                                  # and none without it
        ctx.batching(True)
        for k in range(len(reqs)):
            for mix in (batched[k], apart[k]):
                assert np.max(np.abs(mix - alone[k])) <= 1e-12 * np.max(np.abs(alone[k]))
            req, c, om, w, f = reqs[k]
            q = O.wavenumber_coef(c, om, 16, 1.0)
            for j in range(req["nrhs"]):
                res = np.linalg.norm(f[j] - O.apply_A(q, batched[k][j])) / np.linalg.norm(f[j])
                assert res <= 1e-6
    finally:
        for h in hs:
            h.close()
        ctx.close()


def test_admission_under_a_small_budget_and_refusal():
    from paper_2606_30495_b300 import mcmg
    reqs = _requests()[:3]
    probe = mcmg.Context(0)
    hs = _handles(probe, reqs, mcmg.BF16)
    held = probe.memory()
    for h in hs:
        h.close()
    probe.close()
    # room for the handles plus about one request's workspaces at a time
    slack = 48 * 2 ** 20
    ctx = mcmg.Context(0, hbm_budget_bytes=held + slack)
    hs = _handles(ctx, reqs, mcmg.BF16)
    try:
        fs = [torch.from_numpy(f).cuda() for (_, _, _, _, f) in reqs]
        us = [torch.zeros_like(x) for x in fs]
        tickets = [ctx.submit(h, fd, u, tol=1e-6, restart_m=30, max_iters=3000, nrhs=r[0]["nrhs"])
                   for h, fd, u, r in zip(hs, fs, us, reqs)]
        ctx.drain()
        for t in tickets:
            try:
                st, info = ctx.poll(t)
            except mcmg.McmgError as e:
                raise AssertionError(f"ticket {t}: {e} (handles hold {held} bytes)")
            assert st == 0 and info["converged"]
        assert ctx.memory() <= held + slack
        # a request far larger than the budget is refused once nothing else runs
        big = torch.zeros((8, 64, 64), dtype=torch.complex128, device="cuda")
        big[:, 32, 32] = 1.0
        t = ctx.submit(hs[0], big, torch.zeros_like(big), tol=1e-6, restart_m=2000, nrhs=8)
        ctx.drain()
        with pytest.raises(mcmg.McmgError) as ei:
            ctx.poll(t)
        assert ei.value.status == -3
        with pytest.raises(mcmg.McmgError):
            ctx.poll(987654)
    finally:
        for h in hs:
            h.close()
        ctx.close()


def test_solve_and_submit_read_inputs_after_the_callers_stream():
    """f and u written on the caller's stream just before the call are what
    the solve reads: u is first filled with NaN, then zeroed on torch's
    current stream behind a GPU sleep of about 0.1 s, and the solve is
    issued at once (a single solve, a batched solve and a server request).
    Without the ordering the first residual would read the NaN."""
    from paper_2606_30495_b300 import mcmg
    ctx = mcmg.Context(0)
    reqs = _requests()
    req, c, om, w, f = reqs[0]                   # 64^2, two right-hand sides
    h = mcmg.Handle(ctx, c, om, 16, 1.0, w, precision=mcmg.BF16)
    try:
        fd = torch.from_numpy(f).cuda()
        ref = torch.zeros_like(fd)
        st, info = h.solve(fd, ref, tol=1e-6, restart_m=30, max_iters=3000, nrhs=req["nrhs"])
        assert st == 0 and info["converged"]
        want = ref.cpu().numpy()

        def poisoned():
            u = torch.full_like(fd, float("nan"))
            torch.cuda.synchronize()
            torch.cuda._sleep(200_000_000)        # ~0.1 s of device time on this stream
            u.zero_()
            return u

        u = poisoned()
        st, info = h.solve(fd, u, tol=1e-6, restart_m=30, max_iters=3000, nrhs=req["nrhs"])
        assert st == 0 and info["converged"], info
        assert np.allclose(u.cpu().numpy(), want, rtol=0, atol=1e-12 * np.abs(want).max())
        u1 = poisoned()[0].contiguous()
        st, info = h.solve(fd[0].contiguous(), u1, tol=1e-6, restart_m=30, max_iters=3000)
        assert st == 0 and info["converged"], info
        assert np.all(np.isfinite(u1.cpu().numpy()))
        u = poisoned()
        t = ctx.submit(h, fd, u, tol=1e-6, restart_m=30, max_iters=3000, nrhs=req["nrhs"])
        t0 = time.time()
        while True:
            st, info = ctx.poll(t)
            if st != mcmg.MCMG_PENDING or time.time() - t0 > 60:
                break
            time.sleep(0.002)
        assert st == 0 and info["converged"], (st, info)
        assert np.allclose(u.cpu().numpy(), want, rtol=0, atol=1e-12 * np.abs(want).max())
    finally:
        h.close()
        ctx.close()


def test_several_frequencies_of_one_medium_share_batched_vcycles():
    """The inverse-problem inner solver (Section 5): one medium at several
    frequencies, each frequency a handle of its own (features from its own
    q = (omega h / c)^2 (1 - i gamma)) with the same weights.  Submitted
    together, their V-cycles run as cohorts (one tensor-core launch per level
    and step for all frequencies), and every solution equals the one of the
    frequency alone; each meets the true FP64 residual 1e-6."""
    from paper_2606_30495_b300 import mcmg
    ctx = mcmg.Context(0)
    req, c, om, w, f = _requests()[1]               # 128^2, 4 levels
    omegas = [0.8 * om, om, 1.2 * om]
    hs = [mcmg.Handle(ctx, c, o, 16, 1.0, w, precision=mcmg.BF16) for o in omegas]
    try:
        fd = torch.from_numpy(f).cuda()
        alone = []
        for h in hs:
            u = torch.zeros_like(fd)
            st, info = h.solve(fd, u, tol=1e-6, restart_m=30, max_iters=3000, nrhs=req["nrhs"])
            assert st == 0 and info["converged"], info
            alone.append(u.cpu().numpy())
        r0, m0 = ctx.batching(True)
        us = [torch.zeros_like(fd) for _ in hs]
        tickets = [ctx.submit(h, fd, u, tol=1e-6, restart_m=30, max_iters=3000, nrhs=req["nrhs"])
                   for h, u in zip(hs, us)]
        done = {}
        t0 = time.time()
        while len(done) < len(tickets) and time.time() - t0 < 120:
            for t in tickets:
                if t not in done:
                    st, info = ctx.poll(t)
                    if st != mcmg.MCMG_PENDING:
                        done[t] = (st, info)
            time.sleep(0.002)
        assert len(done) == len(tickets)
        r1, m1 = ctx.batching()
        assert r1 > r0 and m1 - m0 >= 2 * (r1 - r0)
        for k, t in enumerate(tickets):
            st, info = done[t]
            assert st == 0 and info["converged"]
            got = us[k].cpu().numpy()
            assert np.max(np.abs(got - alone[k])) <= 1e-12 * np.max(np.abs(alone[k]))
            q = O.wavenumber_coef(c, omegas[k], 16, 1.0)
            for j in range(req["nrhs"]):
                assert np.linalg.norm(f[j] - O.apply_A(q, got[j])) / np.linalg.norm(f[j]) <= 1e-6
    finally:
        for h in hs:
            h.close()
        ctx.close()


def test_setup_while_the_server_runs_gives_the_features_of_an_idle_setup():
    """Requests set up and submitted one after another while the earlier ones
    run (as a server's arrivals are): every handle computes the same features
    (bit for bit) as a handle of the same medium set up on an idle GPU, and
    every request converges.  Setup uploads its weights and medium on the
    stream its kernels run on; copies left to the legacy stream could land
    after the kernels had read the buffers once the GPU was busy, which
    corrupted coarse-level features and failed requests at their first step."""
    from paper_2606_30495_b300 import mcmg
    base = I.serving_weights()
    reqs = [r for r in I.serving_requests(count=256) if r["n"] <= 512][:24]
    data = [I.serving_request_inputs(r, base) for r in reqs]
    ctx = mcmg.Context(0)
    hs, bufs, tickets = [], [], []
    try:
        for r, (c, om, w, f) in zip(reqs, data):
            h = mcmg.Handle(ctx, c, om, 16, 1.0, w, precision=mcmg.BF16)
            fd = torch.from_numpy(f).cuda()
            u = torch.zeros_like(fd)
            torch.cuda.synchronize()
            tickets.append(ctx.submit(h, fd, u, tol=1e-6, restart_m=30, max_iters=5000,
                                      nrhs=r["nrhs"]))
            hs.append(h)
            bufs.append((fd, u))
        ctx.drain()
        for k, t in enumerate(tickets):
            st, info = ctx.poll(t)
            assert st == 0 and info["converged"], (k, reqs[k]["n"], st, info)
        for r, h, (c, om, w, f) in zip(reqs, hs, data):
            fresh = mcmg.Handle(ctx, c, om, 16, 1.0, w, precision=mcmg.BF16)
            try:
                for l in range(r["levels"]):
                    n = (r["n"] >> l) ** 2
                    C = w["channels"][l]
                    for which in (0, 1):
                        a1 = torch.zeros((n, C), dtype=torch.complex64, device="cuda")
                        a2 = torch.zeros_like(a1)
                        h.get_feature(l, which, a1)
                        fresh.get_feature(l, which, a2)
                        torch.cuda.synchronize()
                        assert torch.equal(a1, a2), (r["n"], l, which)
            finally:
                fresh.close()
    finally:
        for h in hs:
            h.close()
        ctx.close()
