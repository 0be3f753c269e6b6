"""CPU-side checks of the boundary: the shared library loads, exports every
entry point include/mcmg.h declares, and the host-side marshalling is right.
No compute call is made (there may be no GPU)."""
import ctypes

import numpy as np
import pytest

from paper_2606_30495_b300 import inputs as I
from paper_2606_30495_b300 import mcmg


def test_library_exports_every_declared_symbol():
    lib = mcmg.load()
    declared = mcmg.declared_symbols()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(mcmg._SIGS), "binding and header disagree"
    assert b"sm_103a" in lib.mcmg_version()


def test_library_built_for_sm103a():
    """Every translation unit is compiled for sm_103a only (the build's one
    -gencode), and the library reports that architecture."""
    from paper_2606_30495_b300 import build as B
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert b"sm_103a" in mcmg.load().mcmg_version()


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """No fallback: without the CUDA library the binding raises."""
    monkeypatch.setattr(mcmg, "_lib", None)
    with pytest.raises(RuntimeError):
        mcmg.load(str(tmp_path / "libmcmg.so"))


@pytest.mark.parametrize("dim,channels", [(2, [1, 4, 8]), (2, [8, 16, 32, 64]), (3, [8, 16])])
def test_weight_blob_length_matches_header_layout(dim, channels):
    L = len(channels)
    pre, post = I.nu_schedule(L)
    w = I.make_weights(dim, channels, pre, post, mode="structured", seed=0)
    s, blob = mcmg.pack_weights(w)
    T, T3 = 2 * dim + 1, 3 ** dim
    n = 2 * channels[0] * 2 * T3 + 2 * channels[0]
    for l, Cc in enumerate(channels):
        ns = pre[l] + post[l]
        n += 2 * T * Cc * Cc + 2 * 2 * Cc * Cc + 2 * ns * Cc * Cc + 2 * Cc * 2 * Cc * T3 + 2 * Cc
        if l < L - 1:
            Cn = channels[l + 1]
            n += 2 * 2 * T3 * Cn * Cc + 2 * Cn * 2 * Cc * T3 + 2 * Cn
    n += 2 * 2 * channels[0]
    assert s.blob_len == n == blob.size
    assert list(s.channels)[:L] == channels
    # first complex entry of level-0 W follows f_lift's weight and bias
    off = 2 * channels[0] * 2 * T3 + 2 * channels[0]
    assert blob[off] == w["lvl"][0]["W"].reshape(-1)[0].real
    assert blob[off + 1] == w["lvl"][0]["W"].reshape(-1)[0].imag


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """ctypes structs have the sizes and field offsets gcc gives the header's."""
    import os
    import subprocess
    src = tmp_path / "layout.c"
    inc = os.path.join(os.path.dirname(mcmg.HERE), "include")
    fields = {"mcmg_medium": ("Medium", ["dim", "n", "c", "sponge_width", "gamma_max"]),
              "mcmg_weights": ("Weights", ["levels", "channels", "nu_pre", "nu_post", "feat_sl",
                                           "feat_eps", "sl_shift_re", "sl_shift_im", "precision",
                                           "blob", "blob_len"]),
              "mcmg_solve_opts": ("SolveOpts", ["tol", "restart_m", "max_iters", "nrhs", "flags",
                                                  "stream"]),
              "mcmg_solve_info": ("SolveInfo", ["iters", "restarts", "rel_residual", "t_solve_s",
                                                "converged"])}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "mcmg.h"', "int main(void){"]
    for cname, (_, fl) in fields.items():
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        for f in fl:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", inc, str(src), "-o", str(exe)], check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    i = 0
    for cname, (pname, fl) in fields.items():
        cls = getattr(mcmg, pname)
        assert ctypes.sizeof(cls) == vals[i], cname
        i += 1
        for f in fl:
            assert getattr(cls, f).offset == vals[i], (cname, f)
            i += 1


def test_context_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(mcmg.McmgError) as ei:
        mcmg.Context(0)
    assert ei.value.status == -4
