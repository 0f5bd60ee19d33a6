"""Pins of the oracle's velocity model (Sec. 3) against independent computations."""
import numpy as np
import pytest

from paper_2302_10988_gb300 import workloads as W
from tests import pins

MATS = {"weld_ti": W.WELD_TI, "parent_iso": W.PARENT_ISO, "paper_cubic": W.PAPER_CUBIC}


@pytest.mark.parametrize("name", list(MATS))
def test_phase_speed_equals_largest_christoffel_eigenvalue(oracle, name):
    c6, rho = MATS[name]
    m = oracle.mat_from_voigt(c6, rho)
    for th in np.linspace(-np.pi, np.pi, 73):
        v_ref, _ = pins.qp_phase(c6, rho, th)
        assert oracle.phase_velocity(m, th) == pytest.approx(v_ref, rel=1e-12)


def test_phase_speed_axes_closed_form(oracle):
    c6, rho = W.WELD_TI
    m = oracle.mat_from_voigt(c6, rho)
    assert oracle.phase_velocity(m, 0.0) == pytest.approx(np.sqrt(234e9 / 8100), rel=1e-14)
    assert oracle.phase_velocity(m, np.pi / 2) == pytest.approx(np.sqrt(216e9 / 8100), rel=1e-14)
    iso = oracle.mat_from_voigt(*W.PARENT_ISO)
    for th in np.linspace(0, np.pi, 13):
        assert oracle.phase_velocity(iso, th) == np.sqrt(273e9 / 7850)


@pytest.mark.parametrize("name", ["weld_ti", "paper_cubic"])
def test_paper_group_model_polarisation(oracle, name):
    """Sec. 3.2: the inversion returns the phase angle whose qP polarisation lies along the group
    angle; lambda is the qP eigenvalue there and V = v / cos(theta - phi)."""
    c6, rho = MATS[name]
    m = oracle.mat_from_voigt(c6, rho)
    oracle.lib().om_reset_counters()
    for phi in np.radians(np.arange(-179.5, 180.0, 2.5)):
        th, V = oracle.group_paper(m, phi)
        v, p = pins.qp_phase(c6, rho, th)
        pol = np.arctan2(p[2], p[1])
        d = (pol - phi + np.pi / 2) % np.pi - np.pi / 2
        assert abs(d) < 1e-9
        assert V == pytest.approx(v / np.cos(th - phi), rel=1e-12)
        assert abs(th - phi) < np.pi / 2
    # the printed root rule picks the qP root everywhere for these materials
    assert oracle.lib().om_counter(0) == 0
    assert oracle.lib().om_counter(1) == 0


def test_paper_group_model_axis_rounding(oracle):
    """End of Sec. 3.2: within 0.01 deg of a multiple of 90 the angle is rounded onto it."""
    c6, rho = W.WELD_TI
    m = oracle.mat_from_voigt(c6, rho)
    for base, lam in ((0.0, 234e9), (90.0, 216e9), (180.0, 234e9), (-90.0, 216e9)):
        for eps in (0.0, 0.004, -0.009):
            th, V = oracle.group_paper(m, np.radians(base + eps))
            assert V == pytest.approx(np.sqrt(lam / rho), rel=1e-13)


@pytest.mark.parametrize("name", ["weld_ti", "paper_cubic"])
def test_exact_group_model_matches_energy_velocity(oracle, name):
    """Exact ray velocity = the energy velocity of Sec. 3.1 (library eigenvectors) and the Hopf-Lax
    support function of the phase-speed curve."""
    c6, rho = MATS[name]
    m = oracle.mat_from_voigt(c6, rho)
    for th in np.radians(np.arange(-85.0, 90.0, 7.0)):
        psi, Vref = pins.energy_velocity(c6, rho, th)
        th_o, V = oracle.group_exact(m, psi)
        assert V == pytest.approx(Vref, rel=1e-9)
        assert th_o == pytest.approx(th, abs=1e-8)

    def vphase(t):
        return np.array([oracle.phase_velocity(m, x) for x in np.atleast_1d(t)])
    for psi in np.radians([3.0, 31.0, 58.0, 77.0, 122.0]):
        assert oracle.group_exact(m, psi)[1] == pytest.approx(pins.hopf_lax_group_speed(vphase, psi, 801),
                                                              rel=1e-7)


def test_isotropic_group_equals_phase(oracle):
    m = oracle.mat_from_voigt(*W.PARENT_ISO)
    for phi in np.radians([0.0, 17.0, 45.0, 90.0, 133.0]):
        for f in (oracle.group_paper, oracle.group_exact):
            th, V = f(m, phi)
            assert th == pytest.approx(phi)
            assert V == np.sqrt(273e9 / 7850)


def test_paper_vs_exact_group_speed_gap(oracle):
    """The paper's model takes the polarisation as the ray direction; for the weld TI it is faster
    than the exact ray velocity by at most about half a percent, and exact on the axes."""
    m = oracle.mat_from_voigt(*W.WELD_TI)
    gaps = [oracle.group_paper(m, p)[1] / oracle.group_exact(m, p)[1] - 1 for p in np.radians(np.arange(0, 181))]
    assert 0.003 < max(gaps) < 0.006
    assert min(gaps) > -1e-9
    assert abs(gaps[0]) < 1e-12 and abs(gaps[90]) < 1e-12
