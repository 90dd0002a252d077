"""Pins of the oracle's forward of an object of several materials
(orc_forward_fields: per-line phase and attenuation line integrals, Eq. 6
before the single-material substitution of Eq. 7, Eqs. 2, 3 and 5).

* One material: Phi_s = delta_s tau, A_s = mu_s tau is the non-local forward
  of tau (the single-material model), to rounding.
* Mass: the prediction plus the mass that left the grid is sum_s f_s sum
  exp(-A_s) (the splat conserves mass, Eq. 3).
* Zero phase: no transport, P = sum_s f_s exp(-A_s) pixel by pixel.
* A constant added to a line's phase changes nothing (only its gradient
  enters the shift).
* material_fields of one material at the reference indices gives back the
  per-line delta_s and mu_s of the spectrum's scalings.

A shift of the wrong sign or scale, the attenuation taken from the phase
field, or a dropped weight fails one of these."""
import numpy as np
import pytest

from paper_2601_22793_gb300 import phantoms as ph


@pytest.fixture(scope="module")
def case(oracle):
    Es, d, b, w = ph.spectrum(3, 60.0, 120.0, 85.0, 30.0, ph.BONE[0], ph.BONE[1], 80.0, 12)
    ln = oracle.Lines(Es, d, b, w, L=30.0, pixel=20e-6)
    ells = ph.random_ellipsoids(64, 96, 10, 3.0, 18.0, seed=81)
    chords = ph.project_materials(ells, 64, 96, 20e-6)
    tau = ph.project_ellipsoids(ells, 64, 96, 20e-6)
    return ln, chords, tau


def test_one_material_is_the_single_thickness_forward(oracle, case):
    ln, _, tau = case
    _, mu, *_ = ln.params()
    Phi = np.stack([ln.delta[s] * tau for s in range(ln.n)])
    A = np.stack([mu[s] * tau for s in range(ln.n)])
    P, Ps, dr = oracle.forward_fields(ln, Phi, A, per_line=True)
    Pr, Psr, drr = oracle.forward(ln, tau, per_line=True)
    assert np.allclose(P, Pr, rtol=1e-12, atol=0)
    assert np.allclose(Ps, Psr, rtol=1e-12, atol=1e-300)
    assert np.allclose(dr, drr, rtol=1e-9, atol=1e-15)


def test_mass_and_zero_phase(oracle, case):
    ln, chords, _ = case
    Phi, A = oracle.material_fields(ln, chords, [ph.TISSUE[0], ph.BONE[0]],
                                    [ph.TISSUE[1], ph.BONE[1]], 80.0)
    f = ln.w / ln.w.sum()
    I = np.stack([f[s] * np.exp(-A[s]) for s in range(ln.n)])
    P, Ps, dr = oracle.forward_fields(ln, Phi, A, per_line=True)
    for s in range(ln.n):
        assert abs(Ps[s].sum() + dr[s] - I[s].sum()) <= 1e-12 * I[s].sum()
    P0 = oracle.forward_fields(ln, np.zeros_like(Phi), A)
    assert np.allclose(P0, I.sum(0), rtol=1e-14, atol=0)
    # the mismatch is real: the two-material prediction differs from the
    # single-material one of the phase-equivalent thickness
    tau_pe = (ph.TISSUE[0] / ph.BONE[0]) * chords[0] + chords[1]
    Pm = oracle.forward(ln, tau_pe)
    assert np.linalg.norm(P - Pm) > 1e-3 * np.linalg.norm(Pm)


def test_constant_phase_offset_changes_nothing(oracle, case):
    ln, chords, _ = case
    Phi, A = oracle.material_fields(ln, chords, [ph.TISSUE[0], ph.BONE[0]],
                                    [ph.TISSUE[1], ph.BONE[1]], 80.0)
    P = oracle.forward_fields(ln, Phi, A)
    P2 = oracle.forward_fields(ln, Phi + 3e-9, A)
    assert np.allclose(P, P2, rtol=1e-9, atol=0)


def test_material_fields_reproduce_the_line_scalings(oracle, case):
    ln, _, tau = case
    _, mu, *_ = ln.params()
    Phi, A = oracle.material_fields(ln, tau[None], [ph.BONE[0]], [ph.BONE[1]], 80.0)
    for s in range(ln.n):
        assert np.allclose(Phi[s], ln.delta[s] * tau, rtol=1e-14, atol=0)
        assert np.allclose(A[s], mu[s] * tau, rtol=1e-13, atol=0)
