"""The stored operation count of one evaluation of F per node (tests/golden/ops_per_node.txt, written by
tests/golden/make_ops_per_node.py from the oracle) is what the oracle counts now, and the count itself
behaves as its definition says."""
import importlib.util
import os

import numpy as np
import pytest

from paper_2302_10988_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _script():
    spec = importlib.util.spec_from_file_location("make_ops", os.path.join(GOLDEN, "make_ops_per_node.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_stored_counts_are_the_oracles(oracle):
    m = _script()
    stored = {}
    for line in open(os.path.join(GOLDEN, "ops_per_node.txt")):
        f = line.split()
        if not line.startswith("#") and len(f) == 5:
            stored[(f[0], int(f[1]), int(f[2]))] = (int(f[3]), int(f[4]))
    for name, b, s in (("weld_batch", 7, 17), ("weld_single", 0, 9)):
        ops, n = m.count(m.workload(name), b, s)
        so, sn = stored[(name, b, s)]
        assert n == sn
        # libm may round a last digit differently on another machine and flip a near-tie
        assert ops == pytest.approx(so, rel=1e-3)
    per = m.read()
    assert 150 < per["weld_batch"] < 600 and 150 < per["weld_single"] < 600


def test_count_of_a_plane_wave_in_isotropic_steel(oracle):
    """In an isotropic medium every stencil time costs 38 operations and a node's count is made of its
    stencils, metrics and choice: a plane wave along +x frozen on the first column gives every other node the
    same neighbourhood away from the edges, so the count per node is the same there."""
    n = 12
    mats = [oracle.mat_from_voigt(*W.PARENT_ISO)]
    M = oracle.OMedium(n, n, 1e-3, np.zeros(n * n, np.int32), np.zeros(n * n), mats)
    frozen = np.zeros(n * n, np.uint8)
    frozen.reshape(n, n)[:, :2] = 1
    v = oracle.phase_velocity(mats[0], 0.0)
    tau0 = np.where(frozen == 1, (np.arange(n * n) % n) * 1e-3 / v, np.inf)
    tau = oracle.fmm(M, frozen, tau0)[0]
    counts = []
    for j in (4, 5, 6):
        one = np.zeros(n * n, np.uint8)
        one[:] = 1
        one[j * n + 6] = 0  # evaluate F at node (6, j) alone: every other node frozen
        ops, k = oracle.ops_of_F_all(M, one, tau)
        assert k == 1
        counts.append(ops)
    assert counts[0] == counts[1] == counts[2] > 38
