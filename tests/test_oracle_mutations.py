"""Planted mistakes: each test plants one plausible error in the oracle (on
the CPU, through monkeypatch) and checks that one of the oracle's pins
fails on it.  This shows that the pins constrain the part they are meant to
constrain: a wrong weight, a dropped factor, a flipped sign or a swapped
index in the oracle would not go unnoticed."""
import numpy as np
import pytest

from oracle import dg, quadrature, solvers, transfer

import test_oracle_multigrid as mg
import test_oracle_operator as op
import test_oracle_quadrature as qd


def _fails(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


def test_pins_pass_unmutated():
    """The pins used below pass on the oracle as it is."""
    op.test_interior_penalty_closed_form(2)
    op.test_dirichlet_penalty_closed_form(1)
    op.test_weighted_average_closed_form(2)
    op.test_volume_and_reaction_closed_form(1)
    op.test_upwind_closed_form(1)
    op.test_advection_discrete_solution(2)
    op.test_discrete_solution_reproduced(2)
    mg.test_prolongation_reproduces_trilinear_functions()
    mg.test_q1_rediscretisation_equals_galerkin_product(True, True)
    mg.test_thomas_solve_brute_force()
    mg.test_vcycle_symmetric_with_exact_blocks()
    mg.test_tridiagonal_preconditioner_exact_on_tridiagonal_block()
    mg.test_multicolour_sor_properties()
    mg.test_p0_galerkin_matrix_is_modified_fv(True)
    qd.test_gauss3_closed_form()


def test_arithmetic_instead_of_harmonic_mean(monkeypatch):
    monkeypatch.setattr(dg, "harmonic", lambda a, b: 0.5 * (a + b))
    _fails(op.test_interior_penalty_closed_form, 2)


def test_penalty_with_p_p_plus_1(monkeypatch):
    def wrong(self, dm, k):
        a, b = self.tangential_axes(k)
        return self.alpha * self.p * (self.p + 1) * dm * self.h[a] * self.h[b] / np.prod(self.h)
    monkeypatch.setattr(dg.Problem, "penalty_boundary", wrong)
    _fails(op.test_dirichlet_penalty_closed_form, 1)


def test_own_coefficient_on_both_sides_of_a_face(monkeypatch):
    """The face flux of T^+ computed with the K of T^- (an index slip)."""
    orig = dg.Problem.interior_face_matrix

    def wrong(self, cm, k):
        cx = list(self.cell_coords(cm))
        cx[k] += 1
        cp = self.cell_index(*cx)
        saved = self.K[cp].copy()
        self.K[cp] = self.K[cm]
        try:
            return orig(self, cm, k)
        finally:
            self.K[cp] = saved
    monkeypatch.setattr(dg.Problem, "interior_face_matrix", wrong)
    _fails(op.test_weighted_average_closed_form, 2)


def test_reaction_counted_twice(monkeypatch):
    orig = dg.Problem.c_of
    monkeypatch.setattr(dg.Problem, "c_of", lambda self, c: 2.0 * orig(self, c))
    _fails(op.test_volume_and_reaction_closed_form, 1)


def test_advection_field_with_the_wrong_sign(monkeypatch):
    """(The upwind closed form cannot see this one: on piecewise constants
    u^T A u is even in b; the consistency pin can.)"""
    orig = dg.Problem.b_at
    monkeypatch.setattr(dg.Problem, "b_at", lambda self, c, xi: -orig(self, c, xi))
    op.test_upwind_closed_form(1)
    _fails(op.test_advection_discrete_solution, 2)


def test_dirichlet_terms_on_the_opposite_face(monkeypatch):
    orig = dg.Problem.boundary_face_block
    monkeypatch.setattr(dg.Problem, "boundary_face_block", lambda self, c, k, side: orig(self, c, k, 1 - side))
    _fails(op.test_discrete_solution_reproduced, 2)


def test_swapped_q1_hat_functions(monkeypatch):
    orig = transfer.hat
    monkeypatch.setattr(transfer, "hat", lambda o, x: orig(1 - o, x))
    _fails(mg.test_prolongation_reproduces_trilinear_functions)


def test_q1_gradient_with_the_wrong_sign(monkeypatch):
    orig = transfer.hat_deriv
    monkeypatch.setattr(transfer, "hat_deriv", lambda o: -orig(o))
    _fails(mg.test_q1_rediscretisation_equals_galerkin_product, True, True)


def test_thomas_on_the_transposed_band(monkeypatch):
    orig = solvers.thomas_solve
    monkeypatch.setattr(solvers, "thomas_solve",
                        lambda sub, diag, sup, r: orig(np.roll(sup, 1), diag, np.roll(sub, -1), r))
    _fails(mg.test_thomas_solve_brute_force)


def test_vcycle_without_post_smoothing(monkeypatch):
    orig = solvers.HybridVCycle.__init__

    def wrong(self, *a, **kw):
        orig(self, *a, **kw)
        self.npost = 0
    monkeypatch.setattr(solvers.HybridVCycle, "__init__", wrong)
    _fails(mg.test_vcycle_symmetric_with_exact_blocks)


def test_gauss_nodes_left_on_minus_one_to_one(monkeypatch):
    orig = quadrature.gauss_legendre
    monkeypatch.setattr(quadrature, "gauss_legendre", lambda m: (2 * orig(m)[0] - 1, orig(m)[1]))
    _fails(qd.test_gauss3_closed_form)


def test_thomas_preconditioner_dropped(monkeypatch):
    monkeypatch.setattr(solvers, "thomas_solve", lambda sub, diag, sup, r: r / diag)
    _fails(mg.test_tridiagonal_preconditioner_exact_on_tridiagonal_block)


def test_colouring_by_x_parity_only(monkeypatch):
    """Colours that let face neighbours in y or z share a colour."""
    orig = solvers.MulticolourBlockSOR.__init__

    def wrong(self, A, N, nc, *a, **kw):
        orig(self, A, N, nc, *a, **kw)
        c = np.arange(int(np.prod(nc)))
        self.colour = c % nc[0] % 2
    monkeypatch.setattr(solvers.MulticolourBlockSOR, "__init__", wrong)
    _fails(mg.test_multicolour_sor_properties)


def test_p0_coarse_values_spread_with_weight_one_half(monkeypatch):
    orig = transfer.p0_prolongation
    monkeypatch.setattr(transfer, "p0_prolongation", lambda prob: 0.5 * orig(prob))
    _fails(mg.test_p0_galerkin_matrix_is_modified_fv, True)
