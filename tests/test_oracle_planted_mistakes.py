"""Planted mistakes in the oracle (on the CPU) must each be caught by a pin.

Each case monkeypatches one plausible error into the oracle and checks that
the corresponding pin computation then reports a large error.
"""
import numpy as np
import pytest

from oracle import basis, fem
from tests import oracle_pins as pins


def test_transposed_jacobian_convention_is_caught(monkeypatch):
    # the literal J^-T |J| J^-1 of Eq. (localStiffnessMapped) read with J_ij = dx_i/dxi_j
    orig = fem.Operator.geometry

    def transposed(self, es):
        detJ, Jinv = orig(self, es)
        return detJ, np.swapaxes(Jinv, -1, -2)

    monkeypatch.setattr(fem.Operator, "geometry", transposed)
    eK, _ = pins.energy_error(2, 4)
    assert eK > 1e-3


def test_dropped_mass_term_is_caught(monkeypatch):
    orig = fem.Operator.__init__

    def no_mass(self, mesh, alpha, nu, *a, **k):
        orig(self, mesh, 0.0, nu, *a, **k)

    monkeypatch.setattr(fem.Operator, "__init__", no_mass)
    assert pins.volume_error(2, 4) > 0.5


def test_wrong_derivative_sign_is_caught(monkeypatch):
    # flip the sign of one basis function's derivative column (a plausible sign slip in D)
    orig = basis.lagrange_derivatives
    flip = lambda nodes, x: orig(nodes, x) * np.where(np.arange(len(nodes)) == 0, -1.0, 1.0)
    monkeypatch.setattr(fem, "lagrange_derivatives", flip)
    assert pins.box_element_error(2, 4) > 1e-3


def test_wrong_gauss_weight_is_caught(monkeypatch):
    orig = basis.gauss_rule

    def bad(q):
        x, w = orig(q)
        w = w.copy()
        w[0] *= 1.001
        return x, w

    monkeypatch.setattr(fem, "gauss_rule", bad)
    assert pins.volume_error(2, 4) > 1e-5


def test_too_few_quadrature_points_is_caught():
    # q = p (under-integration) no longer reproduces the exact energy
    eK, eM = pins.energy_error(3, 3)
    assert max(eK, eM) > 1e-8


def test_swapped_restriction_is_caught(monkeypatch):
    orig = fem.structured_restriction

    def swapped(nx, ny, nz, p):
        R = orig(nx, ny, nz, p).copy()
        R[:, [1, p + 1]] = R[:, [p + 1, 1]]   # swap local nodes (1,0,0) and (0,1,0)
        return R

    monkeypatch.setattr(fem, "structured_restriction", swapped)
    eK, eM = pins.energy_error(2, 4)
    assert max(eK, eM) > 1e-3
