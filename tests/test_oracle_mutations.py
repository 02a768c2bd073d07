"""The pins catch plausible mistakes in the oracle.

Each case plants one mistake in the oracle's source -- a dropped term, a wrong
sign, a transposed operand, another reading of a formula -- by recompiling the
one function that holds it with a single textual change (on the CPU, in this
process only, undone after the test), then runs the pins meant to catch it.
At least one of them must fail with an AssertionError; a mutation that no pin
notices means the oracle is not pinned there.
"""
import inspect
import textwrap

import numpy as np
import pytest

from oracle import couette, dg, ops, velset
from tests import test_oracle_cavity_symmetry as tsym
from tests import test_oracle_dg as tdg
from tests import test_oracle_ops as tops
from tests import test_oracle_velset as tvs


def _mutate(monkeypatch, module, owner, name, old, new):
    """Recompile owner.name (a function or method defined in `module`) with
    `old` replaced by `new`, and install it for this test."""
    fn = getattr(owner, name)
    src = textwrap.dedent(inspect.getsource(fn))
    assert src.count(old) == 1, f"mutation anchor not unique in {name}: {old!r}"
    ns = dict(vars(module))
    exec(compile(src.replace(old, new), f"<mutant {name}>", "exec"), ns)
    monkeypatch.setattr(owner, name, ns[name])


def _caught(pins):
    """Run the pins; return how many failed with an AssertionError."""
    failed = 0
    for pin in pins:
        try:
            pin()
        except AssertionError:
            failed += 1
    return failed


RHS = (dg, dg.Problem, "rhs")
P0_FV = tdg.test_p0_is_first_order_upwind_finite_volume
ENERGY = tdg.test_central_flux_is_energy_neutral_upwind_dissipates
FREE = tdg.test_free_stream_periodic_is_steady
REST = lambda: (tdg.test_rest_state_with_resting_walls_is_steady("diffuse"),
                tdg.test_rest_state_with_resting_walls_is_steady("eq"))
WALL_MASS = tdg.test_diffuse_walls_conserve_mass_eq_walls_do_not
CONSERVE = lambda: [tdg.test_collision_conserves_mass_and_momentum(vs, o)
                    for vs, o in ((("gh", 4), 2), (("gh", 4), 3), (("nc", 16), 2))]
LOW_MACH = tdg.test_equilibrium_low_mach_expansion_of_maxwellian
TAU = lambda: (tdg.test_tau_from_kn(), tdg.test_couette_closed_form_matches_linearized_solve_and_tau_reading())
LSRK = lambda: (tdg.test_lsrk_order_conditions(), tdg.test_lsrk_fourth_order_in_time())
DERIV = lambda: [tops.test_derivatives_exact_on_polynomials(p) for p in range(1, 5)]
MASSM = lambda: [tops.test_mass_matrix_integrates_products(p) for p in range(1, 5)]
FACEM = lambda: [tops.test_face_mass_integrates_edge_polynomials(p) for p in range(1, 5)]
GEOM = tops.test_geometry_structured_mesh
GH = lambda: (tvs.test_table1_d1q4_d1q5_closed_forms(), tvs.test_table1_d1q6_printed_values(),
              [tvs.test_gh_exact_to_degree_2n_minus_1(n) for n in (3, 4, 6)])
NC = lambda: [tvs.test_nc_even_moments_corrected(n, s) for n, s in ((16, 1.0), (33, np.sqrt(2.0)))]
COUETTE = tdg.test_couette_closed_form_matches_linearized_solve_and_tau_reading
SYM = tsym.pins

MUTATIONS = {
    # numerical flux (Sec. II.B.1): upwind weight with the wrong sign
    "flux_upwind_sign": (RHS, "0.5 * (en - self.ab * np.abs(en))", "0.5 * (en + self.ab * np.abs(en))",
                         [P0_FV, ENERGY]),
    # outward normal flipped in e.n of the flux
    "flux_normal_sign": (RHS, "en = ex[None, :] * nx + ey[None, :] * ny",
                         "en = -(ex[None, :] * nx + ey[None, :] * ny)", [P0_FV, ENERGY]),
    # surface term dropped (no LIFT of the flux difference)
    "dropped_lift": (RHS, 'out += np.einsum("nj,kjq->knq", ops.LIFT, flux)',
                     'out += 0.0 * np.einsum("nj,kjq->knq", ops.LIFT, flux)', [P0_FV, ENERGY]),
    # exterior trace taken from the element itself instead of its neighbour
    "own_trace_as_neighbour": (RHS, "fp = f[self.mapk[elems, fc], self.mapn[elems, fc], :]",
                               "fp = fe[:, ops.fmask[fc], :].copy()", [P0_FV, ENERGY]),
    # volume derivative with the differentiation matrix transposed
    "transposed_dr": (RHS, 'fr = np.einsum("nm,kmq->knq", ops.Dr, fe)',
                      'fr = np.einsum("mn,kmq->knq", ops.Dr, fe)', [FREE, ENERGY]),
    # volume term with the wrong sign
    "volume_sign": (RHS, "out = -(ar[:, None, :] * fr + as_[:, None, :] * fs)",
                    "out = (ar[:, None, :] * fr + as_[:, None, :] * fs)", [P0_FV, ENERGY]),
    # metric term of the volume derivative taken from the wrong axis
    "metric_sx_for_ry": (RHS, 'ey[None, :] * g["ry"][elems, None]', 'ey[None, :] * g["sx"][elems, None]',
                         [SYM, ENERGY]),
    # wall velocity components exchanged in the wall equilibrium (a moving lid
    # then pushes along its normal instead of along the wall)
    "lid_velocity_components_swapped": ((dg, dg.Problem, "_wall_states"), "equilibrium(1.0, u[0], u[1]",
                                        "equilibrium(1.0, u[1], u[0]", [SYM]),
    # BGK term with the wrong sign, or multiplied by tau
    "collision_sign": (RHS, "out -= (fe - feq) / self.tau", "out += (fe - feq) / self.tau", [P0_FV]),
    "collision_times_tau": (RHS, "out -= (fe - feq) / self.tau", "out -= (fe - feq) * self.tau", [P0_FV]),
    # eq. FullBC: numerator summed over the incoming instead of the outgoing half
    "diffuse_numerator_half": (RHS, "np.where(e_n > 0, e_n, 0.0)[None, :] * fm[idx]",
                               "np.where(e_n < 0, -e_n, 0.0)[None, :] * fm[idx]", [WALL_MASS]),
    # wall state imposed on the outgoing instead of the incoming velocities
    "wall_incoming_flipped": (RHS, "fp[idx] = np.where(e_n[None, :] < 0, inc, fm[idx])",
                              "fp[idx] = np.where(e_n[None, :] > 0, inc, fm[idx])", [WALL_MASS, REST]),
    # eq. feq: sign of u^2 in the second-order term
    "feq_u2_sign": ((dg, dg, "equilibrium"), "0.5 * (eu * eu - uu)", "0.5 * (eu * eu + uu)",
                    [CONSERVE, LOW_MACH]),
    # eq. Herm3a: third-order term dropped, or its second part dropped
    "feq_third_dropped": ((dg, dg, "equilibrium"), "poly = poly + eu * eu * eu / 6.0 - 0.5 * eu * uu",
                          "poly = poly + 0.0 * eu", [LOW_MACH]),
    "feq_third_half": ((dg, dg, "equilibrium"), "poly = poly + eu * eu * eu / 6.0 - 0.5 * eu * uu",
                       "poly = poly + eu * eu * eu / 6.0", [CONSERVE, LOW_MACH]),
    # momentum from the wrong velocity component
    "moment_component": ((dg, dg, "moments"), "jx = f @ ex", "jx = f @ ey", [CONSERVE]),
    # eq. KnTau: the other typesetting reading, tau = Kn sqrt(3)
    "tau_reading": ((dg, dg, "tau_from_kn"), "kn * L / (np.sqrt(3.0) * cs)", "kn * L * np.sqrt(3.0) / cs",
                    [TAU]),
    # reference operators: transposed derivative matrix, mass-matrix quadrature
    # without the Jacobian of the collapsed coordinates, LIFT without M^-1
    "refops_dr_transposed": ((ops, ops.RefOps, "__init__"), "self.Dr = Vr @ Vinv", "self.Dr = (Vr @ Vinv).T",
                             [DERIV]),
    "quadrature_no_collapse_jacobian": ((ops, ops, "triangle_quadrature"), "w = WA * WB * 0.5 * (1.0 - B)",
                                        "w = WA * WB * 0.5", [MASSM]),
    "refops_lift_no_minv": ((ops, ops.RefOps, "__init__"), "self.LIFT = np.linalg.solve(self.M, E)",
                            "self.LIFT = E", [FACEM]),
    # geometry: inward normal, Fscale inverted
    "geometry_normal_inward": ((ops, ops, "geometry"), "nx[:, f] = dy / length", "nx[:, f] = -dy / length",
                               [GEOM, P0_FV]),
    "geometry_fscale_inverted": ((ops, ops, "geometry"), "Fscale=sJ / J[:, None]", "Fscale=J[:, None] / sJ",
                                 [GEOM, P0_FV]),
    # velocity sets: GH weights not normalised; NC moment correction dropped
    "gh_weights_unnormalised": ((velset, velset, "gauss_hermite_1d"), "/ np.sqrt(2.0 * np.pi)", "/ 2.5", [GH]),
    "nc_correction_dropped": ((velset, velset, "newton_cotes_1d"),
                              "w = w * (abc[0] + abc[1] * xi ** 2 + abc[2] * xi ** 4)", "w = w", [NC]),
    # eq. exact: the two readings the garbled closed form needs
    "couette_minus_in_z": ((couette, couette, "exact_ux"),
                           "* np.cosh(a)\n                           + 2.0 * (mu * kn",
                           "* np.cosh(a)\n                           - 2.0 * (mu * kn", [COUETTE]),
    "couette_eta_from_wall": ((couette, couette, "exact_ux"), "eta = y - 0.5 * L", "eta = y + 0.5 * L",
                              [COUETTE]),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(monkeypatch, name):
    (module, owner, fname), old, new, pins = MUTATIONS[name]
    _mutate(monkeypatch, module, owner, fname, old, new)
    assert _caught(pins) >= 1, f"no pin caught the planted mistake {name!r}"


def test_lsrk_coefficient_typo_is_caught(monkeypatch):
    b = dg.LSRK_B.copy()
    b[2] *= 1.0 + 1e-6
    monkeypatch.setattr(dg, "LSRK_B", b)
    assert _caught([LSRK]) >= 1


def test_unmutated_pins_pass():
    # the same pin groups pass on the oracle as committed
    groups = [P0_FV, ENERGY, FREE, REST, WALL_MASS, CONSERVE, LOW_MACH, TAU, LSRK, DERIV, MASSM, FACEM,
              GEOM, GH, NC, COUETTE, SYM]
    assert _caught(groups) == 0
