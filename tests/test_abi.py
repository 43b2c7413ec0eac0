"""Host-side checks of the C ABI (no GPU needed): the shared library loads and
exports every entry point include/dig_dsmc.h declares, the Python struct
mirrors the C struct byte for byte, and configuration errors are reported."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2501_10965_gb300 import dsmc, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dig_dsmc.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_symbol():
    L = dsmc.load()
    declared = _declared()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(L, name), name
    assert sorted(dsmc.SYMBOLS) == declared
    out = subprocess.run(["nm", "-D", "--defined-only", dsmc.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, flags=re.M))
    assert set(declared) <= exported


def test_config_struct_layout_matches_header():
    fields = [f[0] for f in dsmc.DsmcConfig._fields_]
    prog = "#include <stdio.h>\n#include <stddef.h>\n#include \"dig_dsmc.h\"\nint main(void){\n"
    prog += 'printf("size %zu\\n", sizeof(dsmc_config));\n'
    for f in fields:
        prog += f'printf("{f} %zu\\n", offsetof(dsmc_config, {f}));\n'
    prog += "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(prog)
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(l.split() for l in lines if l)
    assert int(got["size"]) == ctypes.sizeof(dsmc.DsmcConfig)
    for f in fields:
        assert int(got[f]) == getattr(dsmc.DsmcConfig, f).offset, f


def _ws(cfg):
    L = dsmc.load()
    c = dsmc.make_config(cfg)
    n = ctypes.c_size_t()
    return L.dsmc_workspace_size(ctypes.byref(c), ctypes.byref(n)), n.value


def test_workspace_size_and_argument_errors():
    rc, n = _ws(W.cavity_2d_20m())
    assert rc == 0 and n > 2 * 6 * 4 * 20_040_000  # two FP32 particle buffers at least
    rc, n64 = _ws(W.fourier_1d())
    assert rc == 0 and n64 > 2 * 6 * 8 * 10000
    # d_r 2 or 3, VSS alpha in (0, 2]
    assert _ws(W.fourier_1d(d_r=3.0))[0] == 0 and _ws(W.fourier_1d(alpha=1.5))[0] == 0
    assert _ws(W.fourier_1d(d_r=4.0))[0] == -1 and _ws(W.fourier_1d(d_r=2.5))[0] == -1
    assert _ws(W.fourier_1d(alpha=0.0))[0] == -1 and _ws(W.fourier_1d(alpha=2.5))[0] == -1
    # a batch of FP32 general-gas cases has no fused-step instantiation
    L = dsmc.load()
    arr = (dsmc.DsmcConfig * 2)(*[dsmc.make_config(W.fourier_1d(precision="fp32", d_r=3.0, seed=k)) for k in range(2)])
    n = ctypes.c_size_t()
    assert L.dsmc_batch_workspace_size(arr, 2, ctypes.byref(n)) == -1
    assert _ws(W.fourier_1d(nx=0))[0] == -1
    assert _ws(W.fourier_1d(dt=-1.0))[0] == -1
    bad = W.fourier_1d()
    bad["walls"][0] = {"kind": "diffuse", "T": 1.0, "u": (0.5, 0.0, 0.0)}  # moving along its normal
    assert _ws(bad)[0] == -1
    assert _ws(W.couette_1d(bin_slack=0.5))[0] == -1


def test_synth2d_workspace_and_validation():
    """synth2d reserves the banded factorisation of the 2D synthetic solve:
    8 N (20 m + 158) bytes or so (N = 5 nx ny unknowns, m = min(nx, ny));
    it needs a single 2D box case of at least 3 x 3 cells, at most 500 on
    the shorter side."""
    rc0, n0 = _ws(W.cavity_2d(nx=24, ny=20, ppc=4))
    rc1, n1 = _ws(W.cavity_2d(nx=24, ny=20, ppc=4, synth2d=True))
    assert rc0 == 0 and rc1 == 0
    N, m = 5 * 24 * 20, 20
    assert 8 * N * (20 * m + 149) <= n1 - n0 <= 8 * N * (20 * m + 166) + 4096, (n1 - n0, 8 * N * (20 * m + 158))
    # the band follows the shorter side: 20 x 24 costs the same
    assert _ws(W.cavity_2d(nx=20, ny=24, ppc=4, synth2d=True)) == (0, n1)
    assert _ws(W.fourier_1d(synth2d=True))[0] == -1
    assert _ws(W.cavity_2d(nx=2, ny=8, ppc=4, synth2d=True))[0] == -1
    assert _ws(W.cavity_2d(nx=501, ny=501, ppc=1, synth2d=True))[0] == -1
    # the annulus: at least 5 sectors and 3 rings, at most 500 sectors (its band follows the sectors)
    rc0, nc0 = _ws(W.cylinder_2d(ntheta=24, nr=8, ppc=4))
    rc1, nc1 = _ws(W.cylinder_2d(ntheta=24, nr=8, ppc=4, synth2d=True))
    assert rc0 == 0 and rc1 == 0 and nc1 > nc0
    assert _ws(W.cylinder_2d(ntheta=4, nr=8, ppc=4, synth2d=True))[0] == -1
    assert _ws(W.cylinder_2d(ntheta=24, nr=2, ppc=4, synth2d=True))[0] == -1
    assert _ws(W.cylinder_2d(ntheta=501, nr=8, ppc=1, synth2d=True))[0] == -1
    # the wall-refined box: 2D, stretch > 0; its 2D solve takes the box's workspace
    assert _ws(W.cavity_2d_refined(nx=14, ny=12, ppc=4, dx_min=0.02))[0] == 0
    assert _ws(W.cavity_2d_refined(nx=14, ny=12, ppc=4, dx_min=0.02, synth2d=True)) == \
        (0, _ws(W.cavity_2d_refined(nx=14, ny=12, ppc=4, dx_min=0.02))[1] + _ws(W.cavity_2d(nx=14, ny=12, ppc=4,
                                                                                          synth2d=True))[1]
         - _ws(W.cavity_2d(nx=14, ny=12, ppc=4))[1])
    assert _ws(W.cavity_2d_refined(nx=14, ny=12, ppc=4, dx_min=0.02, stretch=0.0))[0] == -1
    assert _ws(W.cavity_2d_refined(nx=14, ny=12, ppc=4, dx_min=0.02, dim=1))[0] == -1
    L = dsmc.load()
    cs = (dsmc.DsmcConfig * 2)(dsmc.make_config(W.cavity_2d(nx=8, ny=6, ppc=4, synth2d=True)),
                               dsmc.make_config(W.cavity_2d(nx=8, ny=6, ppc=4, synth2d=True)))
    n = ctypes.c_size_t()
    assert L.dsmc_batch_workspace_size(cs, 2, ctypes.byref(n)) == -1


def test_init_without_workspace_is_rejected():
    L = dsmc.load()
    c = dsmc.make_config(W.fourier_1d())
    h = ctypes.c_void_p()
    assert L.dsmc_init(ctypes.byref(c), None, 0, None, ctypes.byref(h)) == -1
    assert not h.value
