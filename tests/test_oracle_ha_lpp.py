"""Pins for the oracle's Heine-Abarenkov local pseudopotential, Eq. (E4A).

The closed form is checked against a radial quadrature of the model it is
the transform of (v = -A inside rc, -Z/r outside), its G -> 0 constant
against the real-space integral, its pressure weight against a numerical
q-derivative, and forces and pressure against finite differences of the
minimised free energy.  Parameters are the ones printed for H.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad

import oracle as O
from paper_1406_0835_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_parameters_are_the_printed_ones():
    gold = json.load(open(os.path.join(GOLD, "paper_constants.json")))["ha_lpp_H"]
    assert O.HA_H == {"rc": gold["rc"], "A": gold["A"], "qc": gold["qc"]}


@pytest.mark.parametrize("Z", [1.0, 2.5])
@pytest.mark.parametrize("q", [0.3, 1.7, 6.0, 19.0, 31.0])
def test_form_is_the_transform_of_the_model(Z, q):
    """Omega w(q)/f(q) = -4 pi Z/q^2 + (4 pi/q) int_0^rc (Z - A r) sin(q r) dr:
    the Coulomb tail plus the compact core correction (v + Z/r) r."""
    rc, A, qc = O.HA_H["rc"], O.HA_H["A"], O.HA_H["qc"]
    omega = 7.0
    core = quad(lambda r: (Z - A * r) * math.sin(q * r), 0.0, rc, epsabs=1e-15, epsrel=1e-13)[0]
    ref = -4.0 * math.pi * Z / q ** 2 + 4.0 * math.pi / q * core
    w = O.lpp_form_ha(np.array([q * q]), omega, Z, rc, A, qc)[0]
    f = math.exp(-(q / qc) ** 6)
    assert omega * w / f == pytest.approx(ref, rel=1e-11, abs=1e-13)


@pytest.mark.parametrize("Z", [1.0, 3.0])
def test_long_wavelength_constant(Z):
    """Omega w(q) + 4 pi Z/q^2 -> int (v(r) + Z/r) d^3r = int_0^rc 4 pi (Z r - A r^2) dr."""
    rc, A, qc = O.HA_H["rc"], O.HA_H["A"], O.HA_H["qc"]
    ref = quad(lambda r: 4.0 * math.pi * (Z * r - A * r * r), 0.0, rc)[0]
    assert O.alpha_z_ha(Z, rc, A) == pytest.approx(ref, rel=1e-13)
    q = 1e-3
    w = O.lpp_form_ha(np.array([q * q]), 1.0, Z, rc, A, qc)[0]
    assert w + 4.0 * math.pi * Z / q ** 2 == pytest.approx(ref, rel=1e-5)


@pytest.mark.parametrize("q", [0.4, 2.0, 9.0, 27.0])
def test_pressure_weight_is_the_dilation_derivative(q):
    """wp = w + (q/3) dw/dq, the derivative taken by central differences."""
    rc, A, qc = O.HA_H["rc"], O.HA_H["A"], O.HA_H["qc"]
    h = 1e-5 * q
    w = lambda x: O.lpp_form_ha(np.array([x * x]), 3.0, 1.0, rc, A, qc)[0]
    dw = (w(q - 2 * h) - 8 * w(q - h) + 8 * w(q + h) - w(q + 2 * h)) / (12 * h)
    wp = O.lpp_pform_ha(np.array([q * q]), 3.0, 1.0, rc, A, qc)[0]
    assert wp == pytest.approx(w(q) + q * dw / 3.0, rel=1e-9, abs=1e-12 * abs(w(q)))


def _system(fn="fttf", L=None, ions=None, grid=12):
    cfg = I.config_single_point()
    return O.System(cfg["L"] if L is None else L, (grid, grid, grid),
                    cfg["ions"] if ions is None else ions, cfg["Z"], 1e5, fn, lpp="ha")


@pytest.mark.parametrize("fn", ["fttf", "sga"])
def test_forces_are_derivatives_of_minimised_energy(fn):
    """Eq. (M12) with the Eq. (E4A) potential: F_I = -dF_tot/dR_I at equilibrium."""
    s = _system(fn)
    phi, ev, _ = O.minimize(s, gtol=1e-11)
    F = O.forces(s, ev)
    R0 = s.R.copy()
    h = 2e-4
    for I_, a in ((0, 0), (5, 1)):
        E = []
        for k in (-1, 1):
            R = R0.copy()
            R[I_, a] += k * h
            s.set_positions(R)
            E.append(O.minimize(s, phi, gtol=1e-11)[1]["F_tot"])
        s.set_positions(R0)
        fd = -(E[1] - E[0]) / (2 * h)
        assert fd == pytest.approx(F[I_, a], rel=1e-5, abs=1e-7)


def test_pressure_is_volume_derivative():
    """Eq. (pressure) with the Eq. (E4A) potential: P = -dF_tot/dOmega at fixed
    fractional coordinates and grid count; the LPP term uses the dilation weight."""
    cfg = I.config_single_point()
    L0 = np.array(cfg["L"])
    frac = cfg["ions"] / L0

    def F_at(lam, phi0=None):
        s = _system("sga", L=L0 * lam, ions=frac * L0 * lam)
        phi, ev, _ = O.minimize(s, phi0, gtol=1e-11)
        return s, phi, ev

    s, phi, ev = F_at(1.0)
    d = 1e-4
    Fp = F_at(1.0 + d, phi)[2]["F_tot"]
    Fm = F_at(1.0 - d, phi)[2]["F_tot"]
    dFdOmega = (Fp - Fm) / (s.grid.omega * ((1 + d) ** 3 - (1 - d) ** 3))
    assert ev["P"] == pytest.approx(-dFdOmega, rel=2e-6)
    assert ev["E_alphaZ"] == pytest.approx(
        s.Ne * 8 * O.alpha_z_ha(1.0, 0.25, 6.18) / s.grid.omega, rel=1e-14)


def test_gaussian_and_ha_share_the_coulomb_tail():
    """Both potentials are -Z/r far from the ion: at small q their difference
    tends to the difference of the two G = 0 constants."""
    g = O.Grid((9.0, 9.0, 9.0), (8, 8, 8))
    q2 = np.array([1e-6])
    wg = O.lpp_form(q2, g.omega, 0.25)[0]
    wh = O.lpp_form_ha(q2, g.omega, 1.0, 0.25, 6.18, 29.97)[0]
    ref = (O.alpha_z_ha(1.0, 0.25, 6.18) - math.pi * 0.25 ** 2) / g.omega
    assert wh - wg == pytest.approx(ref, rel=1e-5)
