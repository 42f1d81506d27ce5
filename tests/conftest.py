import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def build_library():
    """Compile libadc_gb300.so if needed (build.py loaded by path, not via the package)."""
    import importlib.util
    path = os.path.join(ROOT, "paper_2511_21640_gb300", "build.py")
    spec = importlib.util.spec_from_file_location("_adc_gb300_build", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build()


# ---- oracle rows on the host cores (spawn-started processes, one row per task)
_POOL_STATE = {}


def _pool_init(cfg_name, kind, X):
    from synthetic import config_problem
    _POOL_STATE.update(p=config_problem(cfg_name), kind=kind, X=X)


def _pool_row(task):
    from oracle.rows import ea_satellite_rows, ee_doubles_rows, ip_satellite_rows
    order, x, dd_order, row = task
    p, kind, X = _POOL_STATE["p"], _POOL_STATE["kind"], _POOL_STATE["X"]
    if kind == "EE":
        return ee_doubles_rows(p.B, p.eps_occ, p.eps_vir, order, x, X, [row], dd_order=dd_order)[:, 0]
    fn = ea_satellite_rows if kind == "EA" else ip_satellite_rows
    return fn(p.B, p.eps_occ, p.eps_vir, order, x, X, [row])[:, 0]


def oracle_rows_pool(cfg_name, kind, order, x, X, rows, dd_order=1, workers=None):
    """Satellite (IP/EA) or doubles (EE) rows of S = M X from oracle/rows.py for
    the seeded inputs of a named workload, computed in parallel: one spawn-
    started process per host core (at most one per row), each rebuilding the
    inputs from their seed. Returns [len(X), len(rows)]."""
    import multiprocessing as mp
    import numpy as np
    n = max(1, min(workers or os.cpu_count() or 1, len(rows)))
    with mp.get_context("spawn").Pool(n, initializer=_pool_init, initargs=(cfg_name, kind, X)) as pool:
        cols = pool.map(_pool_row, [(order, x, dd_order, r) for r in rows], chunksize=1)
    return np.stack(cols, axis=1)
