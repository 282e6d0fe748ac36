"""The oracle's pins, tested against planted mistakes (CPU only).

Each case below plants one plausible error in the oracle with monkeypatch -- a
dropped term, a wrong sign, a swapped index or weight, a misread formula -- and
checks that at least one of the oracle's pins then fails. A pin that passes for
the right and for the wrong arithmetic pins nothing; these cases show the pins
cover each part of the method (Eq. CS, the Maxwell rule, the shaped EOS, the
equilibrium, the MRT moments, the Shan-Chen force, the Li and Guo forcing,
the two-phase relaxation time, the walls and their ghost densities, the
surface-tension control)."""
import numpy as np
import pytest

from oracle import eos as E
from oracle import lbm as L

import test_oracle_eos as TE  # noqa: E402
import test_oracle_fd as TF  # noqa: E402
import test_oracle_lbm as TL  # noqa: E402
import test_oracle_surface_tension as TS  # noqa: E402


def _eos06():
    e = E.make_eos(E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834)
    e.solve_eps()
    return e


def some_pin_fails(*pins):
    """True if any of the pins fails its assertion (other exceptions propagate, so a
    mutant that merely breaks is not counted as caught)."""
    for pin in pins:
        try:
            pin()
        except AssertionError:
            return True
    return False


def test_pins_pass_unmutated():
    """The same pins pass on the oracle as it stands (the baseline of every case)."""
    e = _eos06()
    assert not some_pin_fails(TE.test_critical_point_matches_printed_constants,
                              lambda: TE.test_maxwell_equals_equal_chemical_potential(0.6),
                              lambda: TE.test_smooth_junctions_are_C1(e),
                              TL.test_equilibrium_moments_closed_form,
                              TL.test_mrt_rows_are_the_velocity_moments,
                              lambda: TL.test_collision_sigma0_equals_guo_in_population_space(e, (1, 1, 1, 1, 1, 1)),
                              TL.test_two_phase_tau_endpoints,
                              lambda: TL.test_bounce_back_is_no_slip_for_free_streaming_packets(e, 5),
                              lambda: TL.test_wall_ghosts_exert_no_force_on_their_own_phase(e))


def test_cs_without_the_cubic_term(monkeypatch):
    """Eq. CS with (1 + eta + eta^2) instead of (1 + eta + eta^2 - eta^3)."""
    monkeypatch.setattr(E, "_cs_Z", lambda eta: (1.0 + eta + eta**2) / (1.0 - eta) ** 3)
    assert some_pin_fails(TE.test_critical_point_matches_printed_constants,
                          TE.test_cs_derivative_against_central_differences,
                          TE.test_maxwell_density_ratios_and_psat_match_paper)


def test_maxwell_densities_off_by_1e4(monkeypatch):
    """A Maxwell construction that lands 1e-4 off (e.g. a loose root tolerance)."""
    orig = E.maxwell
    monkeypatch.setattr(E, "maxwell", lambda a, b, R, T: (lambda r: (r[0] * (1 + 1e-4), r[1], r[2]))(orig(a, b, R, T)))
    assert some_pin_fails(lambda: TE.test_maxwell_equals_equal_chemical_potential(0.6))


def test_cubic_of_the_shaped_eos_in_unnormalised_rho(monkeypatch):
    """Region 2's cubic evaluated in rho - rho_max instead of the normalised t."""
    orig = E.EOS.pressure

    def pressure(self, rho):
        p = np.atleast_1d(np.array(orig(self, rho), dtype=np.float64))
        r = np.atleast_1d(np.asarray(rho, dtype=np.float64))
        if self.mode in (E.MODE_SMOOTH,):
            m = (r > self.rho_max) & (r < self.rho_min)
            d = r[m] - self.rho_max
            p[m] = 2.0 * (self.p_max - self.p_min) * d**3 + 3.0 * (self.p_min - self.p_max) * d**2 + self.p_max
        return p if np.ndim(rho) else float(p[0])

    monkeypatch.setattr(E.EOS, "pressure", pressure)
    assert some_pin_fails(lambda: TE.test_smooth_junctions_are_C1(E.make_eos(E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834)),
                          lambda: TE.test_smooth_obeys_maxwell_rule_independent_quadrature(
                              E.make_eos(E.MODE_SMOOTH, 0.6, 0.387, 2.0, 0.834)))


def test_equilibrium_second_order_coefficient(monkeypatch):
    """f_eq with 4 instead of 1/(2 c_s^4) = 4.5 in front of (c.u)^2."""
    def equilibrium(rho, ux, uy):
        feq = np.empty((9,) + np.shape(rho))
        for i in range(9):
            cu = L.C[i, 0] * ux + L.C[i, 1] * uy
            feq[i] = L.W[i] * rho * (1.0 + 3.0 * cu + 4.0 * cu * cu - 1.5 * (ux * ux + uy * uy))
        return feq

    monkeypatch.setattr(L, "equilibrium", equilibrium)
    assert some_pin_fails(TL.test_equilibrium_moments_closed_form)


def test_mrt_shear_rows_swapped(monkeypatch):
    """Rows 7 and 8 of Eq. MatrixMRT exchanged."""
    M = L.M.copy()
    M[[7, 8]] = M[[8, 7]]
    monkeypatch.setattr(L, "M", M)
    monkeypatch.setattr(L, "MINV", np.linalg.inv(M))
    assert some_pin_fails(TL.test_mrt_rows_are_the_velocity_moments)


def test_shan_chen_weights_swapped(monkeypatch):
    """w(1) = 1/12, w(2) = 1/3 instead of w(1) = 1/3, w(2) = 1/12 in Eq. ShanChenForce."""
    w = L.W_SC.copy()
    w[1:5], w[5:9] = 1.0 / 12.0, 1.0 / 3.0
    monkeypatch.setattr(L, "W_SC", w)
    assert some_pin_fails(lambda: TF.test_interface_response_matches_fd((0.8, 0.5, 0.5, 0.342), 0.03))


def test_shan_chen_force_sign(monkeypatch):
    """F = +G psi sum ... instead of -G psi sum ... (Eq. ShanChenForce)."""
    orig = L.shan_chen_force
    monkeypatch.setattr(L, "shan_chen_force", lambda *a, **k: tuple(-v for v in orig(*a, **k)))
    assert some_pin_fails(lambda: TF.test_interface_response_matches_fd((0.8, 0.5, 0.5, 0.342), 0.03))


def test_li_term_sign(monkeypatch):
    """The sigma terms of Eq. LiFS with the opposite sign."""
    orig = L.li_source
    monkeypatch.setattr(L, "li_source", lambda ux, uy, Fx, Fy, psi, sigma, te, tz:
                        orig(ux, uy, Fx, Fy, psi, -sigma, te, tz))
    assert some_pin_fails(lambda: TF.test_interface_response_matches_fd((0.6, 0.387, 2.0, 0.834), 0.10))


def test_forcing_without_the_half_factor(monkeypatch):
    """m* = m - Lambda (m - m_eq) + S instead of + (I - Lambda/2) S: with Lambda = I
    this doubles the source (Eq. GFS)."""
    orig = L.li_source
    monkeypatch.setattr(L, "li_source", lambda *a: 2.0 * orig(*a))
    e = _eos06()
    assert some_pin_fails(lambda: TL.test_collision_sigma0_equals_guo_in_population_space(e, (1, 1, 1, 1, 1, 1)))


def test_two_phase_relaxation_times_swapped(monkeypatch):
    """tau(rho) of Eq. RelaxationTime with tau_v at rho_l and tau_l at rho_v."""
    orig = L.relaxation_rates
    monkeypatch.setattr(L, "relaxation_rates", lambda relax, rho, rv, rl: orig(relax, rho, rl, rv))
    assert some_pin_fails(TL.test_two_phase_tau_endpoints)


def test_specular_walls_instead_of_bounce_back(monkeypatch):
    """Walls that reflect only the normal velocity (free slip) instead of bouncing the
    populations back (Sec. IV)."""
    monkeypatch.setattr(L, "OPP", np.array([0, 3, 4, 1, 2, 8, 7, 6, 5]))
    e = _eos06()
    assert some_pin_fails(lambda: TL.test_bounce_back_is_no_slip_for_free_streaming_packets(e, 5),
                          lambda: TL.test_bounce_back_is_no_slip_for_free_streaming_packets(e, 6))


def test_wall_ghost_densities_swapped(monkeypatch):
    """The vapour density inside the bottom wall and the liquid density inside the top
    wall (Sec. IV states the opposite)."""
    orig = L.Lattice.__post_init__

    def post_init(self):
        orig(self)
        self.psi_ghost_bottom, self.psi_ghost_top = self.psi_ghost_top, self.psi_ghost_bottom

    monkeypatch.setattr(L.Lattice, "__post_init__", post_init)
    e = _eos06()
    assert some_pin_fails(lambda: TL.test_wall_ghosts_exert_no_force_on_their_own_phase(e))


def test_fd_pressure_tensor_epsilon_sign(monkeypatch):
    """The finite-difference scheme's eps term (App. A, Eq. FDforce) with the wrong sign."""
    from oracle import fd as F

    class Mutant(F.FDSolver):
        def __init__(self, eos, eps, *a, **k):
            super().__init__(eos, -eps, *a, **k)

    monkeypatch.setattr(F, "FDSolver", Mutant)
    assert some_pin_fails(lambda: TF.test_interface_response_matches_fd((0.6, 0.387, 2.0, 0.834), 0.10),
                          lambda: TF.test_interface_response_matches_fd((0.8, 0.5, 0.5, 0.342), 0.03))


def test_fd_maccormack_with_forward_differences_only(monkeypatch):
    """A MacCormack corrector that reuses the predictor's forward differences (App. A)."""
    from oracle import fd as F

    class Mutant(F.FDSolver):
        def d1(self, a, axis, kind):
            return super().d1(a, axis, "f" if kind == "b" else kind)

    monkeypatch.setattr(F, "FDSolver", Mutant)
    assert some_pin_fails(lambda: TF.test_sound_wave_single_phase_matches_fd("liquid"),
                          lambda: TF.test_interface_response_matches_fd((0.8, 0.5, 0.5, 0.342), 0.03))


def test_fd_bottom_wall_without_no_slip(monkeypatch):
    """The FD bottom layer b1 keeping the fluid's tangential velocity (a free-slip
    wall) instead of U_b1 = 0 (Eq. B1)."""
    from oracle import fd as F

    orig = F.FDSolver._padded

    def padded(self, rho, u):
        R, U, S, P = orig(self, rho, u)
        U[0][1] = u[0][0]
        return R, U, S, P

    monkeypatch.setattr(F.FDSolver, "_padded", padded)
    assert some_pin_fails(lambda: TF.test_fd_walls_are_no_slip_shear_mode_decays_at_the_viscous_rate(1.0))


def test_surface_tension_source_row7_sign(monkeypatch):
    """The surface-tension source with +l_nu (Q_xx - Q_yy) in row 7."""
    orig = L.surface_tension_source

    def src(qxx, qyy, qxy, lam):
        c = orig(qxx, qyy, qxy, lam)
        c[7] = -c[7]
        return c

    monkeypatch.setattr(L, "surface_tension_source", src)
    assert some_pin_fails(TS.test_unit_tau_second_moments_shift_by_minus_q_plus_three_quarters_trace,
                          TS.test_planar_interface_evolves_identically_at_unit_tau)


def test_surface_tension_q_without_the_centre_subtraction(monkeypatch):
    """Q from sum_i w_i psi(x + c_i) c_i c_i instead of the differences psi(x + c_i) - psi(x)."""
    orig = L.surface_tension_q

    def q(psi, G, kappa, bc, *ghosts):
        qxx, qyy, qxy = orig(psi, G, kappa, bc, *ghosts)
        k = kappa * G / 2.0 * psi * psi
        return qxx + k, qyy + k, qxy

    monkeypatch.setattr(L, "surface_tension_q", q)
    assert some_pin_fails(TS.test_q_is_exact_for_a_quadratic_psi, TS.test_planar_interface_evolves_identically_at_unit_tau)


def test_fd_surface_tension_term_sign(monkeypatch):
    """The finite-difference pressure tensor with the surface-tension term's sign reversed."""
    from oracle import fd as F

    orig = F.FDSolver.__init__

    def init(self, *args, **kw):
        orig(self, *args, **kw)
        self.kappa = -self.kappa

    monkeypatch.setattr(F.FDSolver, "__init__", init)
    assert some_pin_fails(TS.test_droplet_response_to_kappa_matches_fd)


def test_torch_restatement_surface_tension_row8_sign(monkeypatch):
    """The oracle adjoint's torch restatement with +Q_xy in row 8 of the surface-tension
    source: it no longer equals the numpy oracle's step."""
    pytest.importorskip("torch")
    from oracle import adjoint as A
    import test_oracle_adjoint as TA

    orig = A._surface_tension_source

    def src(qxx, qyy, qxy, z, lam):
        c = orig(qxx, qyy, qxy, z, lam)
        return c.index_copy(0, A.torch.tensor([8]), -c[8:9])

    monkeypatch.setattr(A, "_surface_tension_source", src)
    assert some_pin_fails(lambda: TA.test_torch_step_equals_numpy_oracle(TA.PER, 0.6),
                          lambda: TA.test_torch_step_equals_numpy_oracle(TA.WALLS, 0.6))


def test_peng_theta_weights_swapped(monkeypatch):
    """Eq. PengTheta with r_theta weighting the vapour slope and 1 - r_theta the liquid's."""
    import test_oracle_peng as TP

    def theta(self, rho_m):
        rv, rl = self.rho_v, self.rho_l
        self.theta = (self.r_theta / ((rv - rho_m) * (rv - rl)) * self.dpdrho_v
                      + (1.0 - self.r_theta) / ((rl - rho_m) * (rl - rv)) * self.dpdrho_l)

    monkeypatch.setattr(E.EOS, "_peng_theta", theta)
    assert some_pin_fails(TP.test_peng_theta_gives_the_weighted_branch_its_slope)


def test_fd_two_phase_relaxation_times_swapped(monkeypatch):
    """The FD scheme's tau_nu(rho) of Eq. RelaxationTime with tau_l at rho_v and tau_v at rho_l."""
    from oracle import fd as F

    def tau_nu(self, rho):
        if self.tau_l is None:
            return self.tau_nu, 0.0
        e = self.eos
        tau_v = 0.5 + self.visc_ratio * (self.tau_l - 0.5)
        tau = tau_v * (rho - e.rho_v) / (e.rho_l - e.rho_v) + self.tau_l * (rho - e.rho_l) / (e.rho_v - e.rho_l)
        return tau, (tau_v - self.tau_l) / (e.rho_l - e.rho_v)

    monkeypatch.setattr(F.FDSolver, "_tau_nu", tau_nu)
    assert some_pin_fails(lambda: TF.test_fd_two_phase_viscosity_shear_waves_decay_at_each_phase_rate("liquid"),
                          lambda: TF.test_fd_two_phase_viscosity_shear_waves_decay_at_each_phase_rate("vapour"))


def test_torch_restatement_two_phase_rate_inverted(monkeypatch):
    """The torch restatement relaxing rows 7, 8 with tau(rho) instead of 1/tau(rho)
    (Eq. RelaxationTime misread): it no longer equals the numpy oracle's step."""
    pytest.importorskip("torch")
    from oracle import adjoint as A
    import test_oracle_adjoint as TA

    orig = A.relaxation_diagonal

    def diag(lat, rho):
        lam = orig(lat, rho)
        return A.torch.cat([lam[:7], 1.0 / lam[7:]])

    monkeypatch.setattr(A, "relaxation_diagonal", diag)
    assert some_pin_fails(lambda: TA.test_two_phase_torch_step_equals_numpy_oracle(TA.PER, 0.0),
                          lambda: TA.test_two_phase_torch_step_equals_numpy_oracle(TA.WALLS, 0.0))
