"""The two large workload recipes at the sizes the FP64 oracle solves, against
the oracle's stored FGMRES iteration counts (tests/golden/oracle_solves.json,
written by tests/golden/make_oracle_solves.py from the oracle alone).

* ``helm2d_n256_layers``: the 1024^2 recipe (six layers c in [1, 4] plus
  twenty discs of 10x contrast, 6 points per wavelength, 16-cell sponge,
  6 levels 8/16/32/64/64/64, FGMRES(30)) on a 256^2 grid.
* ``helm3d_n64_grf``: the 256^3 recipe (random field c in [1, 3] plus three
  spheres of 5x contrast, 8 points per wavelength, 10-cell sponge, 5 levels
  8/16/32/64/64, FGMRES(30)) on a 64^3 grid.

Each is solved on the GPU in every channel-mixing precision: the iteration
count must be within 10% of the oracle's and the final solution's relative
residual, recomputed with the oracle's FP64 operator, at most 1e-6.
"""
import json
import os

import numpy as np
import pytest

from oracle import mcmg_oracle as O
from paper_2606_30495_b300 import inputs as I
from tests._models import workload_model

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _golden(name):
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_solves.json")
    return json.load(open(path))[name]


@pytest.fixture(scope="module")
def ctx():
    from paper_2606_30495_b300 import mcmg
    c = mcmg.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("name", ["helm3d_n64_grf", "helm2d_n256_layers"])
@pytest.mark.parametrize("precision", ["fp32", "fp32tc", "bf16"])
def test_large_recipe_solve_against_stored_oracle_count(ctx, name, precision):
    from paper_2606_30495_b300 import mcmg
    m = workload_model(name)
    g = _golden(name)
    assert g["converged"] and g["restart"] == m["wl"]["restart"]
    prec = {"fp32": mcmg.FP32, "fp32tc": mcmg.FP32_TC, "bf16": mcmg.BF16}[precision]
    h = mcmg.Handle(ctx, m["c"], m["omega"], m["sponge"], m["gamma_max"], m["w"], precision=prec)
    try:
        f = I.point_source(m["shape"])
        u = torch.zeros(m["shape"], dtype=torch.complex128, device="cuda")
        st, info = h.solve(torch.from_numpy(f).cuda(), u, tol=1e-6, restart_m=g["restart"],
                           max_iters=3 * g["iters"])
        assert st == 0 and info["converged"], info
        torch.cuda.synchronize()
        res = np.linalg.norm(f - O.apply_A(m["q"], u.cpu().numpy())) / np.linalg.norm(f)
        assert res <= 1e-6, res
        assert abs(info["iters"] - g["iters"]) <= 0.1 * g["iters"], (info["iters"], g["iters"])
        assert h.device_error() == 0
    finally:
        h.close()
