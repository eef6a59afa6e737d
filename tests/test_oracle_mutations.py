"""The pins catch plausible mistakes in the oracle: each test plants one mistake in the oracle
(on the CPU, through monkeypatching) and checks that a pin of `test_oracle_macro.py` or
`test_oracle_pins.py` fails."""
import numpy as np
import pytest

import test_oracle_adjoint as adj_pins
import test_oracle_macro as pins
import test_oracle_pins as cell_pins
from oracle import adjoint, cell, fe, macro, plan

_assemble = macro.assemble
_source = macro.source_point


def _dropped_cross_terms(M, d, H, E_grid, fbar_grid):
    # mistake: the terms coupling U_i and d_m U_j (B^m, Bbar^n) are left out
    E = np.array(E_grid, dtype=np.float64, copy=True)
    N = E.shape[1] // (1 + d)
    E[:, :N, N:] = 0.0
    E[:, N:, :N] = 0.0
    return _assemble(M, d, H, E, fbar_grid)


def _dropped_grad_grad(M, d, H, E_grid, fbar_grid):
    # mistake: the permeability block B^mn is left out
    E = np.array(E_grid, dtype=np.float64, copy=True)
    N = E.shape[1] // (1 + d)
    E[:, N:, N:] = 0.0
    return _assemble(M, d, H, E, fbar_grid)


def _load_without_corner_weight(M, d, H, E_grid, fbar_grid):
    # mistake: int_K N_b taken as |K| instead of |K| / 2^d
    A, rhs, g = _assemble(M, d, H, E_grid, fbar_grid)
    return A, rhs * 2 ** d, g


def _source_element_weight(*args, **kw):
    # mistake: int_e phi taken as h^d times the corner sum (no 1/2^d)
    wl = args[0]
    return _source(*args, **kw) * 2 ** wl.dim


def _source_region_volume(*args, **kw):
    # mistake: normalised by twice the volume of R_p
    return _source(*args, **kw) * 0.5


@pytest.mark.parametrize("mutant", [_dropped_cross_terms])
def test_kronecker_pin_catches_dropped_cross_terms(monkeypatch, mutant):
    monkeypatch.setattr(macro, "assemble", mutant)
    with pytest.raises(AssertionError):
        pins.test_assembly_matches_kronecker(2)


def test_manufactured_pin_catches_dropped_grad_grad(monkeypatch):
    monkeypatch.setattr(macro, "assemble", _dropped_grad_grad)
    with pytest.raises((AssertionError, RuntimeError, ValueError)):
        pins.test_manufactured_solution_second_order(2, (16, 32, 64))


def test_manufactured_pin_catches_wrong_load(monkeypatch):
    monkeypatch.setattr(macro, "assemble", _load_without_corner_weight)
    with pytest.raises(AssertionError):
        pins.test_manufactured_solution_second_order(2, (16, 32, 64))


@pytest.mark.parametrize("mutant", [_source_element_weight, _source_region_volume])
def test_source_pin_catches_wrong_weights(monkeypatch, mutant):
    monkeypatch.setattr(macro, "source_point", mutant)
    with pytest.raises(AssertionError):
        pins.test_source_constant_per_continuum_is_volume_fraction()


# --------------------------------------------------------------------------- cell problems

_stiffness = fe.stiffness_full
_targets = fe.targets
_rows = fe.constraint_rows
_prolong = cell.prolong_medium


def _stiffness_h_power(g, kappa):
    # mistake: element stiffness scaled by h^d instead of h^(d-2)
    return _stiffness(g, kappa) * g.h ** 2


def _targets_sign(g, labels, n_cont, periods, overs):
    # mistake: linear targets int (c_mj - y_m) psi_j instead of int (y_m - c_mj) psi_j
    G = _targets(g, labels, n_cont, periods, overs).copy()
    G[:, n_cont:] *= -1.0
    return G


def _rows_wrong_continuum(g, labels, n_cont, periods):
    # mistake: the constraint of continuum j built from the elements of continuum j + 1
    return _rows(g, (np.asarray(labels) + 1) % n_cont, n_cont, periods)


def _prolong_swapped_axes(values, d, n_coarse, rho):
    # mistake: the child's medium prolonged with x and y exchanged
    v = np.asarray(values).reshape((n_coarse,) * d).swapaxes(-1, -2).reshape(-1)
    return _prolong(v, d, n_coarse, rho)


@pytest.mark.parametrize("target,attr,mutant", [
    (fe, "stiffness_full", _stiffness_h_power),
    (fe, "targets", _targets_sign),
    (fe, "constraint_rows", _rows_wrong_continuum),
])
def test_dense_kkt_pin_catches_cell_mistakes(monkeypatch, target, attr, mutant):
    monkeypatch.setattr(target, attr, mutant)
    with pytest.raises(AssertionError):
        cell_pins.test_level1_matches_dense_kkt("channel2d_17x17_L3", 16, 2)


def test_child_pin_catches_wrong_prolongation(monkeypatch):
    monkeypatch.setattr(cell, "prolong_medium", _prolong_swapped_axes)
    with pytest.raises(AssertionError):
        cell_pins.test_child_correction_matches_dense_kkt()


# --------------------------------------------------------------------------- plan and adjoint

_level_plan = plan.level_plan
_point_adjoint = adjoint._point_adjoint


def _plan_weights_on_wrong_vertices(wl):
    # mistake: the multilinear weights attached to the vertices in reverse order
    levels = _level_plan(wl)
    for lev in levels:
        lev["parents"] = [[(lv, pos, w) for (lv, pos, _), (_, _, w) in zip(par, par[::-1])]
                          for par in lev["parents"]]
    return levels


def _adjoint_without_parent_seeds(wl, ops, kap, lab, r, W, V):
    # mistake: the hierarchy is ignored in the reverse sweep (nothing pushed to the parents)
    g, U = _point_adjoint(wl, ops, kap, lab, r, W, V)
    return g, (None if U is None else np.zeros_like(U))


def _adjoint_seed_sign(wl, ops, kap, lab, r, W, V):
    # mistake: the terms added to the incoming seed V enter with the wrong sign
    g, U = _point_adjoint(wl, ops, kap, lab, r, W, V)
    return g, (None if U is None else 2 * V - U)


def test_parent_pin_catches_weights_on_wrong_vertices(monkeypatch):
    monkeypatch.setattr(plan, "level_plan", _plan_weights_on_wrong_vertices)
    with pytest.raises(AssertionError):
        cell_pins.test_level_plan_parents("channel2d_17x17_L3")


@pytest.mark.parametrize("mutant", [_adjoint_without_parent_seeds, _adjoint_seed_sign])
def test_difference_pin_catches_adjoint_mistakes(monkeypatch, mutant):
    monkeypatch.setattr(adjoint, "_point_adjoint", mutant)
    with pytest.raises(AssertionError):
        adj_pins.test_central_differences((2, 1), 16, 3, 0)
    with pytest.raises(AssertionError):
        adj_pins.test_central_differences((2, 1), 32, 3, 1)


@pytest.mark.parametrize("mutant", [_adjoint_without_parent_seeds, _adjoint_seed_sign])
def test_euler_identity_is_blind_to_the_hierarchical_terms(monkeypatch, mutant):
    """Documents why the differences are needed: the Euler identity still holds with these
    mistakes (scaling every kappa leaves the cell functions unchanged)."""
    monkeypatch.setattr(adjoint, "_point_adjoint", mutant)
    adj_pins.test_euler_identity((2, 1), 16, 3, 0)


# --------------------------------------------------------------------------- more cell pieces

_saddle = cell.saddle_solve
_region = fe.Grid.region_mask
_grid_from_levels = macro.grid_from_levels


def _correction_rhs_sign(A, C, b, g, *args, **kw):
    # mistake: the correction right-hand side taken as +P^T A_1 I
    return _saddle(A, C, -b, g, *args, **kw)


def _region_ignores_overs(self, periods, overs):
    # mistake: E integrated over the whole RVE whatever the oversampling
    return _region(self, periods, 0)


def _grid_y_fastest(pl, M, d, per_level):
    # mistake: macro order with y fastest
    g = _grid_from_levels(pl, M, d, per_level)
    return g.reshape((M,) * d + g.shape[1:]).swapaxes(0, 1).reshape(g.shape)


def test_child_pin_catches_correction_sign(monkeypatch):
    monkeypatch.setattr(cell, "saddle_solve", _correction_rhs_sign)
    with pytest.raises(AssertionError):
        cell_pins.test_child_correction_matches_dense_kkt()


def test_oversampling_pin_catches_ignored_region(monkeypatch):
    monkeypatch.setattr(fe.Grid, "region_mask", _region_ignores_overs)
    with pytest.raises(AssertionError):
        cell_pins.test_oversampling_matches_dense_kkt(2, 16, 4, 1)


def test_macro_order_pin_catches_transposed_grid(monkeypatch):
    monkeypatch.setattr(macro, "grid_from_levels", _grid_y_fastest)
    with pytest.raises(AssertionError):
        pins.test_grid_from_levels_places_points_by_macro_index()


_prolongation = fe.prolongation


def _prolongation_swapped_coarse_axes(gc, gf):
    # mistake: the coarse nodal values read with x and y exchanged
    P = _prolongation(gc, gf).tocsc()
    W = gc.n + 1
    k = np.arange(gc.n_nodes)
    swapped = (k % W) * W + (k // W) % W + (k // (W * W)) * W * W
    return P[:, swapped].tocsr()


def test_galerkin_pin_catches_wrong_prolongation(monkeypatch):
    monkeypatch.setattr(fe, "prolongation", _prolongation_swapped_coarse_axes)
    with pytest.raises(AssertionError):
        cell_pins.test_galerkin_identities()

