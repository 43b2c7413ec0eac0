"""The 2D synthetic solve's arithmetic on the CPU (no GPU needed).

tests/synth2d_host.cu compiles the GPU path's __host__ __device__ functions
(csrc/dsmc_synth2d.cuh) as host code and runs them in the order of the
kernels.  Checked here against the oracle (oracle/synth2d.py) and numpy:

* the residual of every cell equals the oracle's (both band orderings);
* the blocked FP32 banded LU with partial pivoting and the FP32
  substitutions solve random band matrices (heavy pivoting, ragged panel
  counts) to FP64 accuracy under FP64 iterative refinement; a wrong factor
  would stall the refinement far above rounding;
* Newton's method with these solves reaches the oracle's discrete solution
  with the oracle's iteration count.
"""
import ctypes
import os
import shutil
import subprocess
import warnings

import numpy as np
import pytest

from oracle import synth2d
from oracle.fields import F_RHO, F_TR, F_TT, F_U, kappa_coefficients, mu_ref_of
from paper_2501_10965_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2501_10965_gb300", "csrc")
P = ctypes.POINTER(ctypes.c_double)


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    so = str(tmp_path_factory.mktemp("s2host") / "libs2host.so")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-x", "cu", "-I", CSRC,
                    os.path.join(HERE, "synth2d_host.cu"), "-o", so], check=True)
    return ctypes.CDLL(so)


def _p(a):
    return a.ctypes.data_as(P)


def _consts(cfg):
    kt, kr = kappa_coefficients(cfg["a_matrix"], float(cfg["d_r"]))
    return np.array([float(cfg["d_r"]), float(cfg["omega"]), mu_ref_of(float(cfg["kn"])), float(cfg["z_rot"]), kt, kr])


def _smooth(nx, ny, seed=0, hot_amp=1e-3):
    n = nx * ny
    X, Y = np.meshgrid((np.arange(nx) + 0.5) / nx, (np.arange(ny) + 0.5) / ny)
    d = np.zeros((ny, nx, 18))
    d[..., F_RHO] = 1 + 0.02 * np.cos(np.pi * X)
    d[..., F_U] = 0.05 * np.sin(np.pi * X) * np.cos(np.pi * Y) * np.sin(np.pi * Y)
    d[..., F_U + 1] = -0.05 * np.cos(np.pi * X) * np.sin(np.pi * X) * np.sin(np.pi * Y)
    d[..., F_U + 2] = 0.003
    d[..., F_TT] = 1 + 0.01 * Y
    d[..., F_TR] = 1 + 0.012 * Y
    return d.reshape(n, 18), hot_amp * np.random.default_rng(seed).standard_normal((n, 12))


@pytest.mark.parametrize("nx,ny", [(9, 6), (6, 9), (12, 12)])
def test_residual_equals_oracle(lib, nx, ny):
    cfg = W.cavity_2d(nx=nx, ny=ny, ppc=4, kn=0.05, precision="fp64")
    d, h = _smooth(nx, ny, seed=nx)
    x = synth2d.initial_state(d) * (1.0 + 0.01 * np.random.default_rng(1).standard_normal(5 * nx * ny))
    R0 = synth2d.residual(x, d, h, cfg)
    R1 = np.zeros_like(R0)
    lib.h_residual(nx, ny, ctypes.c_double(cfg["lx"] / nx), ctypes.c_double(cfg["ly"] / ny), _p(_consts(cfg)),
                   _p(np.ascontiguousarray(d)), _p(np.ascontiguousarray(h)), _p(x), _p(R1))
    assert np.max(np.abs(R1 - R0)) <= 1e-12 * max(1.0, np.max(np.abs(R0)))


def _refined(lib, cfg):
    """Hand the wall-refined grid's edges to the harness (kept alive by the
    returned arrays)."""
    from oracle.fields import box_edges
    xe = np.ascontiguousarray(box_edges(cfg["nx"], cfg["lx"], cfg["stretch"]))
    ye = np.ascontiguousarray(box_edges(cfg["ny"], cfg["ly"], cfg["stretch"]))
    lib.h_set_edges(_p(xe), _p(ye), ctypes.c_double(cfg["lx"] * cfg["ly"]))
    return xe, ye


@pytest.mark.parametrize("nx,ny", [(9, 6), (6, 9), (12, 12)])
def test_residual_equals_oracle_on_the_wall_refined_grid(lib, nx, ny):
    cfg = W.cavity_2d_refined(nx=nx, ny=ny, ppc=4, kn=0.05, dx_min=0.04, precision="fp64")
    d, h = _smooth(nx, ny, seed=nx)
    x = synth2d.initial_state(d) * (1.0 + 0.01 * np.random.default_rng(1).standard_normal(5 * nx * ny))
    R0 = synth2d.residual(x, d, h, cfg)
    R1 = np.zeros_like(R0)
    keep = _refined(lib, cfg)
    try:
        lib.h_residual(nx, ny, ctypes.c_double(cfg["lx"] / nx), ctypes.c_double(cfg["ly"] / ny), _p(_consts(cfg)),
                       _p(np.ascontiguousarray(d)), _p(np.ascontiguousarray(h)), _p(x), _p(R1))
    finally:
        lib.h_set_edges(None, None, ctypes.c_double(0.0))
    del keep
    assert np.max(np.abs(R1 - R0)) <= 1e-12 * max(1.0, np.max(np.abs(R0)))


@pytest.mark.parametrize("N,kl,nb", [(40, 5, 4), (200, 30, 16), (333, 37, 32), (400, 54, 32), (300, 100, 8)])
def test_blocked_band_lu_refines_to_fp64(lib, N, kl, nb):
    rng = np.random.default_rng(N + kl)
    A = rng.standard_normal((N, N))
    A[np.abs(np.subtract.outer(np.arange(N), np.arange(N))) > kl] = 0.0
    b = rng.standard_normal(N)
    xe = np.linalg.solve(A, b)

    def solve(rhs):
        out = np.zeros(N)
        lib.h_band_test(N, kl, nb, _p(np.ascontiguousarray(A)), _p(np.ascontiguousarray(rhs)), _p(out))
        return out

    x = solve(b)
    first = np.max(np.abs(x - xe)) / np.max(np.abs(xe))
    assert first < 1e-2  # FP32 factors and substitutions
    for _ in range(6):
        x = x + solve(b - A @ x)
    err = np.max(np.abs(x - xe)) / np.max(np.abs(xe))
    assert err < 1e-11, (first, err)


@pytest.mark.parametrize("nx,ny", [(10, 8), (7, 11), (16, 5)])
@pytest.mark.parametrize("reuse", [0, 1])
def test_newton_reaches_the_oracle_solution(lib, nx, ny, reuse):
    """Without reuse every Newton step factorises and the iterates follow
    the oracle's step for step.  With the GPU's reuse policy (1 refinement
    sweep after a fresh factorisation, 3 when reusing) fewer steps
    factorise; the reused steps are exact only to the refinement's accuracy
    (~1e-6), which may cost one more Newton step, and the solution is the
    oracle's."""
    cfg = W.cavity_2d(nx=nx, ny=ny, ppc=4, kn=0.05, precision="fp64")
    d, h = _smooth(nx, ny)
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        out0, it0, res0 = synth2d.synth_solve_2d(d, h, cfg, tol=1e-12, max_iter=50)
    out1 = np.zeros((nx * ny, 6))
    it, res, st, nf = ctypes.c_int(), ctypes.c_double(), ctypes.c_int(), ctypes.c_int()
    lib.h_solve_blk(nx, ny, ctypes.c_double(cfg["lx"] / nx), ctypes.c_double(cfg["ly"] / ny), _p(_consts(cfg)),
                    _p(np.ascontiguousarray(d)), _p(np.ascontiguousarray(h)), 50, ctypes.c_double(1e-12), 32, 1,
                    reuse, 3, _p(out1), ctypes.byref(it), ctypes.byref(res), ctypes.byref(st), ctypes.byref(nf))
    assert st.value == 0 and res.value < 1e-11
    if reuse:
        assert it0 <= it.value <= it0 + 1 and 1 <= nf.value < it.value, (it0, it.value, nf.value)
    else:
        assert it.value == it0 and nf.value == it0
    np.testing.assert_allclose(out1, out0, rtol=0, atol=1e-12)


@pytest.mark.parametrize("nx,ny", [(10, 8), (7, 11)])
def test_newton_reaches_the_oracle_solution_on_the_wall_refined_grid(lib, nx, ny):
    """The GPU's Newton steps (reuse policy included) on the wall-refined
    grid, with the volume-weighted total-mass row: the oracle's solution."""
    cfg = W.cavity_2d_refined(nx=nx, ny=ny, ppc=4, kn=0.05, dx_min=0.04, precision="fp64")
    d, h = _smooth(nx, ny)
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        out0, it0, res0 = synth2d.synth_solve_2d(d, h, cfg, tol=1e-12, max_iter=50)
    out1 = np.zeros((nx * ny, 6))
    it, res, st, nf = ctypes.c_int(), ctypes.c_double(), ctypes.c_int(), ctypes.c_int()
    keep = _refined(lib, cfg)
    try:
        lib.h_solve_blk(nx, ny, ctypes.c_double(cfg["lx"] / nx), ctypes.c_double(cfg["ly"] / ny), _p(_consts(cfg)),
                        _p(np.ascontiguousarray(d)), _p(np.ascontiguousarray(h)), 50, ctypes.c_double(1e-12), 32, 1,
                        1, 3, _p(out1), ctypes.byref(it), ctypes.byref(res), ctypes.byref(st), ctypes.byref(nf))
    finally:
        lib.h_set_edges(None, None, ctypes.c_double(0.0))
    del keep
    assert st.value == 0 and res.value < 1e-11
    assert it0 <= it.value <= it0 + 1, (it0, it.value)
    np.testing.assert_allclose(out1, out0, rtol=0, atol=1e-12)


# ---------------------------------------------------------------------------
# the annulus around a cylinder
# ---------------------------------------------------------------------------

def _ann_cfg(nt, nr, **kw):
    base = dict(ntheta=nt, nr=nr, ppc=4, kn=0.1, mach=0.5, r_in=0.5, r_out=1.5, dr1=0.1, precision="fp64")
    base.update(kw)
    return W.cylinder_2d(**base)


def _ann_state(cfg, seed=0, hot_amp=1e-3):
    from oracle import synth_annulus as SA
    nt, nr, R, rc, dth, thc = SA.geometry(cfg)
    r, th = np.meshgrid(rc, thc, indexing="ij")
    x, y, r = (r * np.cos(th)).ravel(), (r * np.sin(th)).ravel(), r.ravel()
    n = nt * nr
    d = np.zeros((n, 18))
    d[:, F_RHO] = 1.0 + 0.05 * np.cos(x)
    d[:, F_U] = 0.2 * (1.0 - 0.5 / r) * np.sin(y)
    d[:, F_U + 1] = -0.1 * x * y
    d[:, F_U + 2] = 0.01
    d[:, F_TT] = 1.0 + 0.1 * np.exp(-r)
    d[:, F_TR] = 1.0 + 0.08 * np.exp(-r)
    return d, hot_amp * np.random.default_rng(seed).standard_normal((n, 12)), R


@pytest.mark.parametrize("nt,nr", [(10, 6), (7, 5), (16, 4)])
def test_annulus_residual_equals_oracle(lib, nt, nr):
    from oracle import synth_annulus as SA
    cfg = _ann_cfg(nt, nr)
    d, h, R = _ann_state(cfg, seed=nt)
    x = SA.initial_state(d) * (1.0 + 0.01 * np.random.default_rng(2).standard_normal(5 * nt * nr))
    R0 = SA.residual(x, d, h, cfg)
    R1 = np.zeros_like(R0)
    Rk = np.ascontiguousarray(R)
    lib.h_set_annulus(_p(Rk))
    try:
        lib.h_residual(nt, nr, ctypes.c_double(1.0), ctypes.c_double(1.0), _p(_consts(cfg)),
                       _p(np.ascontiguousarray(d)), _p(np.ascontiguousarray(h)), _p(x), _p(R1))
    finally:
        lib.h_set_annulus(None)
    assert np.max(np.abs(R1 - R0)) <= 1e-12 * max(1.0, np.max(np.abs(R0)))


@pytest.mark.parametrize("nt,nr", [(10, 6), (12, 5)])
def test_annulus_newton_reaches_the_oracle_solution(lib, nt, nr):
    """The GPU's Newton steps on the annulus (no total-mass row; the reuse
    policy): the oracle's solution."""
    from oracle import synth_annulus as SA
    cfg = _ann_cfg(nt, nr)
    d, h, R = _ann_state(cfg)
    out0, it0, res0 = SA.synth_solve_annulus(d, h, cfg, tol=1e-12, max_iter=50)
    out1 = np.zeros((nt * nr, 6))
    it, res, st, nf = ctypes.c_int(), ctypes.c_double(), ctypes.c_int(), ctypes.c_int()
    Rk = np.ascontiguousarray(R)
    lib.h_set_annulus(_p(Rk))
    try:
        lib.h_solve_blk(nt, nr, ctypes.c_double(1.0), ctypes.c_double(1.0), _p(_consts(cfg)),
                        _p(np.ascontiguousarray(d)), _p(np.ascontiguousarray(h)), 50, ctypes.c_double(1e-12), 32, 1,
                        1, 3, _p(out1), ctypes.byref(it), ctypes.byref(res), ctypes.byref(st), ctypes.byref(nf))
    finally:
        lib.h_set_annulus(None)
    assert st.value == 0 and res.value < 1e-11 and res0 < 1e-11
    assert it0 <= it.value <= it0 + 1, (it0, it.value)
    np.testing.assert_allclose(out1, out0, rtol=0, atol=1e-12)
