"""synth_solve_noalloc: the synthetic solve for callers that cannot allocate
device memory (their device memory belongs to another allocator, or they run
where cudaMalloc is not allowed).  It keeps its scratch in a fixed array inside
the library instead of a caller-provided workspace.  Its output must equal the
ordinary synth_solve's on the same inputs, on two calls in a row (the second
call reuses the array the first one left behind).

This file is collected last on purpose, so that a run which stops at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2501_10965_gb300 import dsmc, workloads as W

pytestmark = pytest.mark.gpu


def _inputs(cfg, seed):
    n = cfg["nx"]
    rng = np.random.default_rng(seed)
    x = (np.arange(n) + 0.5) / n
    f = np.zeros((n, dsmc.NFIELDS))
    f[:, 0] = 1.0 + 0.05 * rng.standard_normal(n)
    f[:, 2] = -0.3 + 0.6 * x + 0.01 * rng.standard_normal(n)
    f[:, 4] = 1.0 + 0.3 * x + 0.01 * rng.standard_normal(n)
    f[:, 5] = 1.0 + 0.28 * x + 0.01 * rng.standard_normal(n)
    hot = 0.003 * rng.standard_normal((n, dsmc.NHOT))
    return torch.tensor(f, device="cuda"), torch.tensor(hot, device="cuda")


@pytest.mark.parametrize("nx", [150, 1030, "max"])
def test_noalloc_synth_equals_synth_solve_on_two_calls(nx):
    """150 cells run the 128-thread solver; 1030 the 1024-thread one with
    strided loops; the largest slab accepted fills nearly all of the fixed
    array."""
    nx = dsmc_max() if nx == "max" else nx
    cfg = W.couette_1d(kn=0.05, nx=nx, ppc=4, synth_tol=1e-12, n_m=60, precision="fp64")
    ref_sim = dsmc.Dsmc(cfg)
    for call, seed in enumerate((1, 2)):
        fields, hot = _inputs(cfg, seed)
        ref, it_ref, res_ref = ref_sim.synth_solve(fields, hot)
        out, it, res, rc = dsmc.synth_solve_noalloc(cfg, fields, hot)
        torch.cuda.synchronize()
        assert rc == 0, (call, rc)
        assert it == it_ref and res_ref < 1e-9
        assert np.allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=1e-12, atol=1e-14), call


def test_noalloc_synth_rejects_oversized_slab_through_the_c_abi():
    L = dsmc.load()
    cfg = dsmc.make_config(W.couette_1d(nx=dsmc_max() + 1, ppc=1, precision="fp64"))
    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(t.data_ptr())
    rc = L.synth_solve_noalloc(ctypes.byref(cfg), p, p, p, None, None, None)
    assert rc == -2


def dsmc_max():
    import re
    import os
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "dig_dsmc.h")
    return int(re.search(r"#define DSMC_SYNTH_NOALLOC_MAX_CELLS (\d+)", open(hdr).read()).group(1))
