"""Helpers shared by the GPU parity tests: run the CUDA path and the CPU oracle on the
same seeded inputs and compare field by field."""
import numpy as np

import oracle
from paper_2511_10257_gb300 import inputs as I

ALL_FIELDS = [I.PHI, I.HE, I.T, I.FL, I.P, I.U, I.V, I.C, I.MUC, I.RHO, I.MX, I.MY, I.FSPREV]


# Liquid and solid fractions live on [0, 1]: their scale is 1 even when a case has
# almost no solid (then the oracle's field is rounding noise of order 1e-16).
SCALE_FLOOR = {I.FL: 1.0, I.FSPREV: 1.0}


def rel_err(a, b, floor=1e-30):
    """max |a - b| relative to the reference field's largest magnitude"""
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), floor))


def compare(solver, case_id, ref, fields=ALL_FIELDS):
    got = solver.fields(case_id, fields)
    return {I.FIELD_NAMES[f]: rel_err(got[f], ref.get(f), SCALE_FLOOR.get(f, 1e-30)) for f in fields}


def assert_parity(solver, case_id, ref, tol, fields=ALL_FIELDS):
    errs = compare(solver, case_id, ref, fields)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"fields beyond {tol:g}: {bad}"
    return errs


def set_both(solver, case_id, ref, state):
    solver.set_fields(case_id, state)
    ref.set_state(state)


def _oracle_job(job):
    """worker of oracle_pool: (case, steps, fields, state) -> {field: array}"""
    case, steps, fields, state = job
    o = oracle.Oracle(case, threads=1)
    if state:
        o.set_state(state)
    o.step(steps)
    return {f: o.get(f) for f in fields}


def oracle_pool(jobs, processes=None):
    """Run independent oracle cases in parallel worker processes started with spawn
    (safe after the CUDA context exists).  jobs: (case, steps, fields, state or None)."""
    import multiprocessing as mp
    import os
    n = processes or min(len(jobs), os.cpu_count() or 1)
    oracle.build()
    with mp.get_context("spawn").Pool(n) as pool:
        return pool.map(_oracle_job, jobs)
