"""Oracle runs that the GPU tests farm out to worker processes (spawned,
so that no worker inherits a CUDA context): plain functions of picklable
arguments that import nothing but the oracle and the workload table."""
import oracle
from oracle.fields import fields_from_sums
from paper_2501_10965_gb300 import workloads as W


def couette_fields(kn, seed, warm, ns):
    """Time-averaged fields of the oracle's 1D Couette flow (200 x 200, FP64)
    over steps warm .. warm + ns."""
    o = oracle.OracleSim(W.couette_1d(kn=kn, precision="fp64", seed=seed))
    o.step(warm)
    o.reset_accumulators()
    o.step(ns, sample=True)
    c = o.constants()
    return fields_from_sums(o.accumulators(), o.nsamples, c["fnum"], c["vcell"], 2.0)


def pool(n):
    """A process pool of n spawned workers."""
    import concurrent.futures
    import multiprocessing
    return concurrent.futures.ProcessPoolExecutor(max_workers=n, mp_context=multiprocessing.get_context("spawn"))
