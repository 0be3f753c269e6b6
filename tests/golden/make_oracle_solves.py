"""Write tests/golden/oracle_solves.json: FP64 oracle solves of the named workloads.

Calls only the oracle and the seeded input generators.  For each workload it
records the FGMRES(restart) iteration count, restarts and final true relative
residual of the point-source solve at tol 1e-6 (zero initial guess).
Run:  python tests/golden/make_oracle_solves.py [workload ...]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import mcmg_oracle as O  # noqa: E402
from paper_2606_30495_b300 import inputs as I  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_solves.json")
DEFAULT = ["helm2d_n64_homogeneous", "helm2d_n64_slmg", "helm2d_n256_grf", "helm3d_n64_grf",
           "helm2d_n256_layers"]
MAX_ITERS = {"helm2d_n256_layers": 20000}


def solve(name):
    wl = I.workload(name)
    c = I.medium_for(wl)
    omega = I.omega_for_ppw(c.min(), wl["ppw"], wl["n"])
    q = O.wavenumber_coef(c, omega, wl["sponge"], wl["gamma_max"])
    w = I.weights_for(wl)
    feats = O.setup(q, w)
    f = I.point_source(c.shape)
    t0 = time.time()
    _, info = O.fgmres(lambda u: O.apply_A(q, u), lambda v: O.vcycle(w, feats, v), f,
                       m=wl["restart"], tol=wl["tol"], max_iters=MAX_ITERS.get(name, 4000))
    return dict(iters=info["iters"], restarts=info["restarts"],
                rel_residual=info["rel_residual"], converged=info["converged"],
                restart=wl["restart"], tol=wl["tol"], oracle_seconds=round(time.time() - t0, 1))


if __name__ == "__main__":
    names = sys.argv[1:] or DEFAULT
    for n in names:
        res = solve(n)
        print(n, res, flush=True)
        # re-read before writing, so runs of different workloads can overlap
        data = json.load(open(OUT)) if os.path.exists(OUT) else {}
        data[n] = res
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
