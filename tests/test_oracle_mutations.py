"""The oracle's pins have teeth (CPU only).

Each case plants one plausible mistake in the oracle (a wrong Gauss abscissa,
a sign, a transposed operand, a dropped term or factor, the wrong inner
product) by patching the oracle module for the duration of the case, then runs
the pin that must catch it and expects it to fail.  The planted mistakes never
leave this file: monkeypatch undoes each one when the case ends.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import test_oracle_graded as GRADED
import test_oracle_ks as KSPINS
import test_oracle_mg as MGPINS
import test_oracle_pins as PINS
from oracle import ks as KS
from oracle import mg as MG
from oracle import paro as O


def _fails(pin, *args):
    with pytest.raises((AssertionError, np.linalg.LinAlgError, FloatingPointError)):
        pin(*args)


def test_pins_pass_unmutated():
    # the same pins, without a planted mistake, pass (so the failures below are theirs)
    PINS.test_stiffness_and_mass_are_kronecker_products((4, 5, 6), (1.0, 1.5, 2.0))
    PINS.test_product_potential_is_exact_integral()
    PINS.test_free_box_sine_mode_fixed_point()
    PINS.test_rayleigh_ritz_conditions_and_interlacing()
    PINS.test_paro_converges_to_dense_spectrum()
    KSPINS.test_hartree_of_a_gaussian_charge_converges_at_second_order()
    KSPINS.test_slater_energy_of_a_gaussian_density()
    MGPINS.test_prolongation_evaluates_the_coarse_function((8, 6, 4))
    KSPINS.test_mixing_moves_the_input_density_toward_the_output_by_the_mixing_fraction()
    GRADED.test_graded_stiffness_and_mass_are_kronecker_products((6, 5, 7), (2.0, 1.5, 3.0), (1.5, 0.8, 2.5))


def test_wrong_gauss_abscissa_is_caught(monkeypatch):
    def bad():  # 1/3 in place of 1/sqrt(3)
        return np.array([(1 - 1 / 3) / 2, (1 + 1 / 3) / 2]), np.array([0.5, 0.5])

    monkeypatch.setattr(O, "gauss_1d", bad)
    _fails(PINS.test_stiffness_and_mass_are_kronecker_products, (4, 5, 6), (1.0, 1.5, 2.0))


def test_wrong_shape_derivative_sign_is_caught(monkeypatch):
    orig = O.q1_shape

    def bad(t):
        l, dl = orig(t)
        return l, np.stack([dl[0], -dl[1]])

    monkeypatch.setattr(O, "q1_shape", bad)
    _fails(PINS.test_stiffness_and_mass_are_kronecker_products, (4, 5, 6), (1.0, 1.5, 2.0))


def test_potential_read_in_the_wrong_gauss_point_order_is_caught(monkeypatch):
    orig = O.element_matrices
    # q = qx + 2 qy + 4 qz read as qz + 2 qy + 4 qx
    perm = [((q >> 2) & 1) | (q & 2) | ((q & 1) << 2) for q in range(8)]

    def bad(h):
        Ke, Me, P, wq = orig(h)
        return Ke, Me, P[perm], wq

    monkeypatch.setattr(O, "element_matrices", bad)
    # a potential linear along one axis cannot show it (on the interior nodes the
    # cell-local linear part assembles to the same matrix along any axis); x y z can
    _fails(PINS.test_product_potential_is_exact_integral)


def test_dropped_shift_in_the_source_operator_is_caught(monkeypatch):
    monkeypatch.setattr(O.Operators, "A", property(lambda self: (0.5 * self.K + self.MV).tocsr()))
    _fails(PINS.test_free_box_sine_mode_fixed_point)


def test_unshifted_right_hand_side_is_caught(monkeypatch):
    orig = O.pcg

    def bad_source(ops, U, lam, tol, maxit):  # lambda_i M u_i in place of (lambda_i + sigma) M u_i
        return orig(ops.A, (ops.M @ U) * np.asarray(lam)[None, :], U, tol, maxit)

    monkeypatch.setattr(O, "source_problems", bad_source)
    _fails(PINS.test_free_box_sine_mode_fixed_point)


def test_euclidean_in_place_of_mass_inner_product_is_caught(monkeypatch):
    orig = O.rayleigh_ritz

    def bad(ops, X):
        eye = sp.identity(ops.M.shape[0], format="csr")
        return orig(O.Operators(ops.mesh, ops.K, eye, ops.MV, ops.sigma), X)

    monkeypatch.setattr(O, "rayleigh_ritz", bad)
    _fails(PINS.test_rayleigh_ritz_conditions_and_interlacing)


def test_transposed_rotation_is_caught(monkeypatch):
    orig = O.rayleigh_ritz

    def bad(ops, X):
        rr = orig(ops, X)
        return O.RRResult(X @ rr.C.T, rr.lam, rr.GA, rr.GB, rr.C)

    monkeypatch.setattr(O, "rayleigh_ritz", bad)
    _fails(PINS.test_rayleigh_ritz_conditions_and_interlacing)


def test_skipped_source_problems_are_caught(monkeypatch):
    def bad(ops, U, lam, tol, maxit):  # Rayleigh-Ritz on the old orbitals
        n = U.shape[1]
        return O.PCGResult(U.copy(), np.zeros(n, int), np.zeros(n), np.ones(n, bool))

    monkeypatch.setattr(O, "source_problems", bad)
    _fails(PINS.test_paro_converges_to_dense_spectrum)


def test_hartree_without_four_pi_is_caught(monkeypatch):
    orig = KS.hartree

    def bad(mesh, rho_q):
        r = orig(mesh, rho_q)
        return KS.HartreeResult(r.VH_q / (4 * math.pi), r.VH_nodes / (4 * math.pi), r.Q, r.xc)

    monkeypatch.setattr(KS, "hartree", bad)
    _fails(KSPINS.test_hartree_of_a_gaussian_charge_converges_at_second_order)


def test_wrong_slater_constant_is_caught(monkeypatch):
    monkeypatch.setattr(KS, "slater_potential",
                        lambda rho_q: -np.cbrt(3.0 * np.maximum(rho_q, 0.0) / (4 * np.pi)))
    _fails(KSPINS.test_slater_energy_of_a_gaussian_density)


def test_wrong_prolongation_weight_is_caught(monkeypatch):
    orig = MG.prolongation_1d

    def bad(nf):  # neighbours weighted 1/4 in place of 1/2
        P = orig(nf).tocoo()
        v = np.where(P.data == 0.5, 0.25, P.data)
        return sp.csr_matrix((v, (P.row, P.col)), shape=P.shape)

    monkeypatch.setattr(MG, "prolongation_1d", bad)
    _fails(MGPINS.test_prolongation_evaluates_the_coarse_function, (8, 6, 4))


def test_swapped_mixing_direction_is_caught(monkeypatch):
    # rho_in <- mix rho_in + (1 - mix) rho_out: the roles of the two densities swapped
    monkeypatch.setattr(KS, "mix_density", lambda rho_in, rho_out, mix: mix * rho_in + (1.0 - mix) * rho_out)
    _fails(KSPINS.test_mixing_moves_the_input_density_toward_the_output_by_the_mixing_fraction)


def test_graded_stiffness_with_the_axes_swapped_is_caught(monkeypatch):
    # the unit cell's gradient parts paired with the wrong cell sizes (x with h_z):
    # invisible on a uniform mesh, and on a graded mesh with equal spacing per axis
    orig = O._unit_stiffness_parts
    monkeypatch.setattr(O, "_unit_stiffness_parts", lambda: orig()[::-1].copy())
    _fails(GRADED.test_graded_stiffness_and_mass_are_kronecker_products, (6, 5, 7), (2.0, 1.5, 3.0), (1.5, 0.8, 2.5))
