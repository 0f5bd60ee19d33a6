"""Pins of the oracle's stencil table (Sec. 4.1), single-stencil update (Sec. 4.2) and choice (Sec. 4.3)."""
import numpy as np
import pytest

from paper_2302_10988_gb300 import workloads as W


def test_stencil_table_structure(oracle):
    """Sec. 4.1: 16 square and 16 triangular stencils, in pairs that share A and D with B and C swapped."""
    T = oracle.stencil_table()  # [32, 3 (A, B, C), 2 (di, dj)]
    rows = {tuple(T[r].ravel()) for r in range(32)}
    assert len(rows) == 32
    for p in range(16):
        s1, s2 = T[2 * p], T[2 * p + 1]
        assert (s1[0] == s2[0]).all() and (s1[1] == s2[2]).all() and (s1[2] == s2[1]).all()
    for r in range(16):  # squares: A, B, C, D are the corners of a square, A opposite D
        A, B, C = T[r]
        assert (B + C - A == 0).all()
        assert np.dot(B - A, C - A) == 0 and np.dot(B - A, B - A) == np.dot(C - A, C - A)
        assert np.dot(B - A, B - A) == (1 if r < 8 else 2)
    for r in range(16, 32):  # triangles: A two cells along an axis, an axis point and a diagonal point
        A, B, C = T[r]
        assert sorted(np.abs(A)) == [0, 2]
        axis, diag = (B, C) if 0 in B else (C, B)
        assert (axis * 2 == A).all()
        assert np.abs(diag).tolist() == [1, 1] and np.dot(diag - axis, diag - axis) == 1


def _plane_wave_medium(oracle, theta_mat, n=5):
    c6, rho = W.WELD_TI
    m = oracle.mat_from_voigt(c6, rho)
    M = oracle.OMedium(n, n, 1e-3, np.zeros(n * n), np.full(n * n, theta_mat), [m])
    return M, m


def test_linear_field_exactness_every_stencil(oracle):
    """Sec. 4.2: with exact samples of a plane wave tau = x.n / v(n) at A, B, C, the wavefront EB is an
    iso-line and every feasible stencil returns the exact time at D."""
    T = oracle.stencil_table()
    rng = np.random.default_rng(5)
    hits = np.zeros(32, int)
    for trial in range(400):
        th_mat = rng.uniform(-np.pi, np.pi)
        M, m = _plane_wave_medium(oracle, th_mat)
        ang = rng.uniform(-np.pi, np.pi)
        nvec = np.array([np.cos(ang), np.sin(ang)])
        slow = M.h / oracle.phase_velocity(m, ang - th_mat)
        jj, ii = np.mgrid[0:5, 0:5]
        tau = ((ii - 2) * nvec[0] + (jj - 2) * nvec[1]) * slow
        for r in range(32):
            A, B, C = [tau[2 + T[r, k, 1], 2 + T[r, k, 0]] for k in range(3)]
            if not (A < B <= C):
                continue
            if B + C - A <= 0 and r < 16:  # D would not be downwind
                continue
            got = oracle.stencil_value(M, tau, 2, 2, r)
            if got <= C:
                continue
            hits[r] += 1
            assert got == pytest.approx(0.0, abs=1e-12 * slow)
    assert (hits > 0).all()


def _choice_case(oracle, ang_deg, drop=()):
    """Node D at the centre of a 5x5 plane-wave patch; returns F_D and its record."""
    M, m = _plane_wave_medium(oracle, 0.0)
    a = np.radians(ang_deg)
    slow = M.h / oracle.phase_velocity(m, a)
    jj, ii = np.mgrid[0:5, 0:5]
    tau = ((ii - 2) * np.cos(a) + (jj - 2) * np.sin(a)) * slow
    for di, dj in drop:
        tau[2 + dj, 2 + di] = np.inf
    frozen = np.zeros(25, np.uint8)
    F, rec = oracle.F_all(M, frozen, tau)
    return F[2, 2], rec[2, 2]


def test_choice_worked_examples(oracle):
    """Sec. 4.3 by hand.  A plane wave along 30 deg: of the squares only 1 (A lower-left) and
    5 (A two cells left) have A earliest; |tau_C - tau_B| is 0.37 cell-times for square 1 and 1.0 for
    square 5, so square 1 is used, with B = (i-1, j) (the earlier of its two points): stencil 1-2."""
    F, rec = _choice_case(oracle, 30.0)
    assert rec == 1 and abs(F) < 1e-18
    # along 60 deg square 1 again, now B = (i, j-1): stencil 1-1
    F, rec = _choice_case(oracle, 60.0)
    assert rec == 0 and abs(F) < 1e-18
    # along +x (0 deg) no small square has A earliest; square 5 (A = (i-2, j)) is used, member 1 on the tie
    F, rec = _choice_case(oracle, 0.0)
    assert rec == 8 and abs(F) < 1e-18
    # without the node (i-1, j-1) square 5 and triangle 16 are incomplete: only triangle 13 is left,
    # whose axis point (i-1, j) is earlier than its diagonal point: B = axis, stencil 13-1
    F, rec = _choice_case(oracle, 0.0, drop=[(-1, -1)])
    assert rec == 24 and abs(F) < 1e-18
    # with nothing but (i-1, j) known, no stencil exists: straight-ray fallback through that slot
    drop = [(di, dj) for di in range(-2, 3) for dj in range(-2, 3) if (di, dj) not in ((-1, 0), (0, 0))]
    F, rec = _choice_case(oracle, 0.0, drop=drop)
    assert rec == 32 + 0
