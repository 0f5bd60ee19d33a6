"""Independent reference computations used to pin the oracle.

Nothing here calls the oracle: each function derives its result another way
(a library eigen-solver on the full 3x3 Christoffel matrix, a brute-force
maximisation, a textbook closed form), so that a mistake in the oracle's
formulas shows up as a disagreement.
"""
import numpy as np


def voigt_to_tensor(c6):
    """C_ijkl from the 6x6 Voigt matrix through the index map of Sec. 3.2:
    f(i, j) = i if i == j else 9 - i - j (1-based)."""
    def f(i, j):
        return i if i == j else 9 - i - j
    C = np.zeros((3, 3, 3, 3))
    for i in range(1, 4):
        for j in range(1, 4):
            for k in range(1, 4):
                for l in range(1, 4):
                    C[i - 1, j - 1, k - 1, l - 1] = c6[f(i, j) - 1, f(k, l) - 1]
    return C


def christoffel(c6, n):
    """M_ik = C_ijkl n_j n_l for a unit 3-vector n."""
    C = voigt_to_tensor(np.asarray(c6, float))
    return np.einsum("ijkl,j,l->ik", C, n, n)


def qp_phase(c6, rho, theta):
    """qP phase speed and polarisation for phase direction (0, cos theta, sin theta) in the YZ plane."""
    n = np.array([0.0, np.cos(theta), np.sin(theta)])
    w, V = np.linalg.eigh(christoffel(c6, n))
    return np.sqrt(w[-1] / rho), V[:, -1]


def energy_velocity(c6, rho, theta):
    """Group velocity vector d(omega)/dk_m from the Christoffel equation of Sec. 3.1,
    rho omega^2 = C_ijql k_j k_l p_i p_q, which gives V_m = C_imql p_i p_q n_l / (rho v).
    (The derivation printed in Sec. 3.1 places both polarisation indices in one index pair; taken
    from the Christoffel equation as printed, they sit in different pairs.)
    Returned as (angle in the YZ plane, magnitude)."""
    C = voigt_to_tensor(np.asarray(c6, float))
    n = np.array([0.0, np.cos(theta), np.sin(theta)])
    v, p = qp_phase(c6, rho, theta)
    Vm = np.einsum("imql,i,q,l->m", C, p, p, n) / (rho * v)
    return np.arctan2(Vm[2], Vm[1]), np.hypot(Vm[1], Vm[2])


def hopf_lax_group_speed(phase_speed, psi, n=4001):
    """Group speed along psi from the phase-speed curve: 1/V = max_theta cos(theta - psi) / v(theta),
    maximised by a dense scan and two refinements."""
    lo, hi = psi - np.pi / 2, psi + np.pi / 2
    best = None
    for _ in range(3):
        th = np.linspace(lo, hi, n)
        vals = np.cos(th - psi) / phase_speed(th)
        k = int(np.argmax(vals))
        best = vals[k]
        step = (hi - lo) / (n - 1)
        lo, hi = th[k] - 2 * step, th[k] + 2 * step
    return 1.0 / best


def qp_phase_many(c6, rho, theta):
    """qP phase speeds for an array of phase angles (the batched form of qp_phase)."""
    th = np.asarray(theta, float).reshape(-1)
    C = voigt_to_tensor(np.asarray(c6, float))
    n = np.stack([np.zeros_like(th), np.cos(th), np.sin(th)], 1)
    M = np.einsum("ijkl,bj,bl->bik", C, n, n)
    w = np.linalg.eigvalsh(M)
    return np.sqrt(w[:, -1] / rho).reshape(np.shape(theta))


def exact_group_speed(c6, rho, psi):
    """Ray (energy) speed along the angle psi from the material axis, by the Hopf-Lax maximum over
    phase directions of cos(theta - psi) / v(theta), with the eigen-solver's phase speeds."""
    return hopf_lax_group_speed(lambda th: qp_phase_many(c6, rho, th), psi)


def paper_group_speed(c6, rho, psi):
    """The paper's group speed along psi (Sec. 3.2): the phase angle theta whose qP polarisation (from the
    eigen-solver) lies along psi, found by a scan and bisection, and V = v(theta) / cos(theta - psi)."""
    from scipy.optimize import brentq

    def mismatch(th):
        _, p = qp_phase(c6, rho, th)
        d = np.arctan2(p[2], p[1]) - psi
        return (d + np.pi / 2) % np.pi - np.pi / 2

    grid = np.linspace(psi - np.pi / 2 + 1e-9, psi + np.pi / 2 - 1e-9, 721)
    f = np.array([mismatch(t) for t in grid])
    roots = []
    for k in range(len(grid) - 1):
        # a sign change through zero (not a jump of the wrapped angle across +-pi/2)
        if f[k] == 0.0:
            roots.append(grid[k])
        elif f[k] * f[k + 1] < 0 and abs(f[k]) < 0.5 and abs(f[k + 1]) < 0.5:
            roots.append(brentq(mismatch, grid[k], grid[k + 1], xtol=1e-15, rtol=1e-15))
    assert len(roots) == 1, roots
    th = roots[0]
    v, _ = qp_phase(c6, rho, th)
    return v / np.cos(th - psi)
