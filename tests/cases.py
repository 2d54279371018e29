"""Seeded parity cases: oracle factorizations of the paper's workloads at sizes the oracle
builds in seconds (several nodes per level, ragged segment lengths, odd and even L)."""
import functools

import numpy as np

from oracle import idbf, kernels
from paper_1809_10573_gb300 import inputs

CASES = {
    # name: (N, n0, kernel, grid, eps, build kwargs)
    "dft_1024": (1024, 16, ("dft", -1, 0), "uniform", 1e-8, {}),
    "dft_jit_2048_oddL": (2048, 16, ("dft", -1, 0), "jitter", 1e-6, {}),            # L = 7
    "fio_base_4096": (4096, 64, ("fio", 0, 0), "uniform", 1e-8, dict(t=2, t_leaf=4)),  # N = 4096, eps = 1e-8 FIO
    "fio_paper_2048": (2048, 8, ("fio", 0, 1), "uniform", 1e-6, {}),                # Example 1, L = 8
    "fio_base_8192_oddL": (8192, 64, ("fio", 0, 0), "uniform", 1e-6, dict(t=2, t_leaf=4)),  # L = 7
    "j0_2048": (2048, 16, ("j0", 0, 0), "schlomilch", 1e-8, dict(t=2, t_leaf=4)),   # Example 2, L = 7
    # the benchmark's FIO at N = 2^14 (L = 8): 256 nodes per level, blocks of up to 181 rows and
    # 324 columns, the tall shapes of the N = 2^20 benchmark's middle levels
    "fio_base_16384": (16384, 64, ("fio", 0, 0), "uniform", 1e-6, dict(t=2, t_leaf=4)),
}


def kernel_of(spec):
    kind, sign, prof = spec
    kinds = {"fio": kernels.KIND_FIO, "dft": kernels.KIND_DFT, "j0": kernels.KIND_J0}
    return kernels.Kernel(kinds[kind], sign=sign, c_profile=prof)


def grid_of(name, N):
    grid = CASES[name][3]
    if grid == "uniform":
        return inputs.uniform_grid(N)
    if grid == "schlomilch":
        return inputs.schlomilch_grid(N)
    return inputs.jittered_grid(N, seed=N)


@functools.lru_cache(maxsize=None)
def oracle_case(name):
    N, n0, kspec, _, eps, kw = CASES[name]
    x, xi = grid_of(name, N)
    K = kernel_of(kspec)
    F = idbf.build(K, x, xi, eps, n0, **kw)
    return dict(N=N, n0=n0, x=x, xi=xi, K=K, F=F, ex=idbf.export(F), eps=eps)
