"""mcmg_cgs2_noalloc against mcmg_cgs2.

The no-allocation variant serves callers that must not call cudaMalloc (code
under another framework's fixed memory budget, or call sites that cannot take
an allocation's device-wide synchronisation).  Its scratch is a static device
array shared by all calls.  This file is collected last so that a run stopping
at its first failure has already run every other test; it passes alone in a
fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

from paper_2606_30495_b300 import inputs as I
from tests._models import model, relerr, rng

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_cgs2_matches_allocating_cgs2_twice():
    from paper_2606_30495_b300 import mcmg
    ctx = mcmg.Context(0)
    m = model((34, 30), [8, 16], mode="random", seed=3)
    h = mcmg.Handle(ctx, m["c"], m["omega"], m["sponge"], m["gamma_max"], m["w"])
    try:
        n = 34 * 30
        for call, k in enumerate((13, 64)):              # two calls in a row
            Q, _ = np.linalg.qr(I.complex_normal((n, k), rng(60 + call)))
            V = torch.from_numpy(np.ascontiguousarray(Q.T)).to("cuda", torch.complex64)
            w0 = torch.from_numpy(I.complex_normal(n, rng(70 + call))).to("cuda", torch.complex64)
            w_ref, w_new = w0.clone(), w0.clone()
            h_ref, n_ref = h.cgs2(V, w_ref)
            h_new, n_new = mcmg.cgs2_noalloc(V, w_new)
            torch.cuda.synchronize()
            assert relerr(h_new, h_ref) < 1e-6
            assert abs(n_new - n_ref) < 1e-5 * n_ref
            assert relerr(w_new.cpu().numpy(), w_ref.cpu().numpy()) < 1e-5
        with pytest.raises(mcmg.McmgError) as ei:        # beyond the stated maximum
            mcmg.cgs2_noalloc(torch.zeros((65, n), dtype=torch.complex64, device="cuda"),
                              torch.zeros(n, dtype=torch.complex64, device="cuda"))
        assert ei.value.status == -1
    finally:
        h.close()
        ctx.close()


def test_noalloc_cgs2_allocates_nothing_and_runs_on_a_side_stream():
    """A warm call leaves torch's reserved memory, the library's accounted
    memory and the device's free memory unchanged, and a call on a
    non-default stream gives the default stream's results."""
    from paper_2606_30495_b300 import mcmg
    ctx = mcmg.Context(0)
    m = model((34, 30), [8, 16], mode="random", seed=4)
    h = mcmg.Handle(ctx, m["c"], m["omega"], m["sponge"], m["gamma_max"], m["w"])
    try:
        n, k = 34 * 30, 20
        Q, _ = np.linalg.qr(I.complex_normal((n, k), rng(80)))
        V = torch.from_numpy(np.ascontiguousarray(Q.T)).to("cuda", torch.complex64)
        w0 = torch.from_numpy(I.complex_normal(n, rng(81))).to("cuda", torch.complex64)
        w_def, w_side = w0.clone(), w0.clone()
        side = torch.cuda.Stream()          # created (and used once) before measuring
        mcmg.cgs2_noalloc(V, w0.clone())                  # warm: modules loaded, address cached
        mcmg.cgs2_noalloc(V, w0.clone(), stream=side)
        torch.cuda.synchronize()
        reserved, ctx_mem = torch.cuda.memory_reserved(), ctx.memory()
        free0, _ = torch.cuda.mem_get_info()
        h_def, n_def = mcmg.cgs2_noalloc(V, w_def)
        side.wait_stream(torch.cuda.current_stream())
        h_side, n_side = mcmg.cgs2_noalloc(V, w_side, stream=side)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert torch.cuda.memory_reserved() == reserved
        assert ctx.memory() == ctx_mem
        assert free1 == free0
        assert relerr(h_side, h_def) < 1e-6
        assert abs(n_side - n_def) < 1e-5 * n_def
        assert relerr(w_side.cpu().numpy(), w_def.cpu().numpy()) < 1e-5
    finally:
        h.close()
        ctx.close()
