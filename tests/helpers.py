"""Shared test helpers: build the oracle problem and the GPU grid from one seeded spec."""
import numpy as np

from oracle import constraints as ocs, discrete as odz


def oracle_problem(spec):
    pb = odz.problem_from(spec)
    rows = ocs.rows_from_intents(pb, spec.get("intents", []))
    return pb, rows


def gpu_grid(spec, precision):
    from paper_2607_26082_b300 import rows as prow
    return prow.setup_grid(spec, precision)


def rel_l2(a, b):
    d = np.linalg.norm(np.asarray(a) - np.asarray(b))
    n = np.linalg.norm(np.asarray(b))
    return d / n if n > 0 else d


def dof_masks(pb):
    return np.stack([pb.dof_mask(c) for c in range(3)])
