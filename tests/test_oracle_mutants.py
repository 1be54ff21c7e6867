"""Planted mistakes in the oracle, on the CPU: each mutant below (one edit of
the oracle's source: a dropped term, a flipped sign, a wrong index or
operand) must fail at least one of the pins aimed at it, so the pins can
tell the oracle from a plausible slip in it.

A mutant is built in memory from the oracle's source and put in place of
its module (and of the modules that import from it) for one check; the
pins are the functions of tests/test_oracle_*.py, imported afresh so that
they bind the mutant.  The files on disk are not touched, and the module
table is restored afterwards.  Edits that change only a convention with no
observable consequence (the sign of the DFT's exponent, which of sin / cos
drives which normal, the direction of the CPML's alpha grading, the
boundary condition at the ends of the envelope's domain, where the bound
state has decayed to ~e^-32) are not planted here: the oracle's convention
there is fixed by the GPU path's bit-exact Philox and field parity instead.
"""
import importlib
import os
import sys
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_MODULES = ("test_oracle_maxwell", "test_oracle_gain", "test_oracle_cpml_probes",
               "test_oracle_adjoint", "test_oracle_philox", "test_oracle_gp", "test_oracle_analysis",
               "test_oracle_modemap")
ORACLE_MODULES = ("mb_oracle", "mb_adjoint", "mb_analysis", "gp_oracle")

# pins: (test module, function, keyword arguments)
CAVITY = [("test_oracle_maxwell", "test_pec_cavity_eigenmode",
           dict(grid=(9, 16, 11), modes=(2, 1, 3), amp_dir=(1.0, 0.2, -0.4), eps_r=2.5)),
          ("test_oracle_maxwell", "test_yee_energy_invariant_pec_box", {})]
CPML = [("test_oracle_cpml_probes", "test_cpml_coefficients_shape", {}),
        ("test_oracle_cpml_probes", "test_cpml_reflection_against_larger_box", {})]
LORENTZ = [("test_oracle_gain", "test_lorentz_recursion_harmonic_response", dict(lam=590e-9)),
           ("test_oracle_gain", "test_lorentz_recursion_continuous_limit_is_the_lorentzian", {})]
NOISE = [("test_oracle_gain", "test_langevin_force_amplitude_after_one_step", {}),
         ("test_oracle_gain", "test_lorentz_noise_stationary_variance", {})]
RATES = [("test_oracle_gain", "test_rate_steady_state_closed_form", {}),
         ("test_oracle_gain", "test_rate_crank_nicolson_matches_matrix_exponential", {})]
COUPLING = [("test_oracle_gain", "test_field_and_atoms_exchange_energy_exactly", {}),
            ("test_oracle_gain", "test_field_transfer_direction", {}),
            ("test_oracle_gain", "test_inverted_medium_amplifies_and_absorber_absorbs", {}),
            ("test_oracle_gain", "test_populations_conserved_in_noisy_run", {})]
PROBES = [("test_oracle_cpml_probes", "test_point_probe_dft_of_cavity_mode", {}),
          ("test_oracle_cpml_probes", "test_face_flux_balances_interior_energy_exactly", {})]
FACE = [("test_oracle_cpml_probes", "test_face_spectra_parseval", dict(every=1, stride=2))]
PHILOX = [("test_oracle_philox", "test_philox_known_answers", "every known-answer row"),
          ("test_oracle_philox", "test_philox_vectorised_matches_scalar", {}),
          ("test_oracle_philox", "test_unit_map_is_open_interval_and_exact_in_fp32", {}),
          ("test_oracle_philox", "test_box_muller_moments", {})]
GP = [("test_oracle_gp", "test_near_threshold_closed_form", {}),
      ("test_oracle_gp", "test_integral_identities", dict(E=4.0)),
      ("test_oracle_gp", "test_integral_identities", dict(E=20.0)),
      ("test_oracle_gp", "test_thomas_fermi_limit", dict(E=150.0)),
      ("test_oracle_gp", "test_shooting_and_boundary_value_solve_agree", {}),
      ("test_oracle_gp", "test_features_from_the_fourier_transform", dict(E=20.0)),
      ("test_oracle_gp", "test_threshold_and_pump_relation", {}),
      ("test_oracle_gp", "test_peak_grows_and_width_is_finite_above_threshold", {})]
ANALYSIS = [("test_oracle_analysis", "test_sampled_gaussian_gives_back_centre_and_width", {}),
            ("test_oracle_analysis", "test_flat_spectrum_std_width_is_uniform", {}),
            ("test_oracle_analysis", "test_two_lines_std_width_is_half_the_spacing", {}),
            ("test_oracle_analysis", "test_sweep_threshold_is_first_level_that_halves_the_width", {}),
            ("test_oracle_analysis", "test_emission_threshold_finds_the_kink_of_an_s_curve", {})]
MODEMAP = [("test_oracle_modemap", "test_energy_density_planes_sum_to_the_energy", {}),
           ("test_oracle_modemap", "test_plane_probe_equals_point_probes_on_its_cells", {}),
           ("test_oracle_modemap", "test_plane_probe_sampling_interval_does_not_change_the_map", {}),
           ("test_oracle_modemap", "test_cw_waveform_closed_form", {})]
ADJ = [("test_oracle_adjoint", "test_adjoint_gradient_matches_central_differences", dict(case=c))
       for c in ("pulse", "noise", "strong")] + \
      [("test_oracle_adjoint", "test_objective_is_the_face_flux", {}),
       ("test_oracle_adjoint", "test_crank_nicolson_pump_derivative", {})]

MUTANTS = {
    # Maxwell part
    "H curl: a sign": ("mb_oracle", "Hx -= dt / MU0 * (dEz_dy - dEy_dz", "Hx -= dt / MU0 * (dEz_dy + dEy_dz", CAVITY),
    "H curl: backward difference": ("mb_oracle", "dEz_dy = d_fwd(Ez, AX_Y) / dx", "dEz_dy = d_bwd(Ez, AX_Y) / dx", CAVITY),
    "E curl: forward difference": ("mb_oracle", "dHx_dz = d_bwd(Hx, AX_Z) / dx", "dHx_dz = d_fwd(Hx, AX_Z) / dx", CAVITY),
    "E update: 1/eps_r dropped": ("mb_oracle", "ce = dt / (EPS0 * self.eps_r)", "ce = dt / EPS0", CAVITY),
    "E update: mu0 for eps0": ("mb_oracle", "Hy -= dt / MU0 *", "Hy -= dt / EPS0 *", CAVITY),
    "PEC: a wall left open": ("mb_oracle", "        Ey[:, :, 0] = 0.0\n", "", CAVITY),
    "E update: current with the wrong sign": ("mb_oracle", "- Jtot[2])", "+ Jtot[2])", COUPLING),
    # CPML
    "CPML: memory dropped from the H curl": ("mb_oracle", "Hz -= dt / MU0 * (dEy_dx - dEx_dy + psH[(\"z\", \"x\")] - psH[(\"z\", \"y\")])",
                                             "Hz -= dt / MU0 * (dEy_dx - dEx_dy)", CPML),
    "CPML: memory not decaying": ("mb_oracle", "    b[inside] = bb[inside]\n", "    b[inside] = 1.0\n", CPML),
    "CPML: grading exponent": ("mb_oracle", "sigma = sigma_max * depth ** p.pml_order", "sigma = sigma_max * depth", CPML),
    "CPML: E memory from the H profile": ("mb_oracle", "            b, c = be[w]\n", "            b, c = bh[w]\n", CPML),
    # Lorentz polarization and noise
    "Lorentz: restoring force sign": ("mb_oracle", "- w0 * w0 * P + force", "+ w0 * w0 * P + force", LORENTZ),
    "Lorentz: damping sign": ("mb_oracle", "J_new = ((1.0 - a) * J", "J_new = ((1.0 + a) * J", LORENTZ),
    "Lorentz: P from the old J": ("mb_oracle", "P_new = P + dt * J_new", "P_new = P + dt * J", LORENTZ),
    "Lorentz: inversion reversed": ("mb_oracle", "dN = N1 - N2", "dN = N2 - N1", COUPLING),
    "noise: amplitude from N1": ("mb_oracle", "np.sqrt((np.maximum(N2, 0.0) + N_floor)", "np.sqrt((np.maximum(N1, 0.0) + N_floor)", NOISE),
    "noise: 1/dt dropped from the variance": ("mb_oracle", "/ (dx ** 3 * dt))", "/ (dx ** 3))", NOISE),
    # populations
    "rates: pump into N2": ("mb_oracle", "    A[3, 0] = W_p\n", "    A[2, 0] = W_p\n", RATES),
    "rates: decay N2 -> N1 missing its loss": ("mb_oracle", "    A[2, 2] = -1.0 / p.tau21\n", "", RATES),
    "rates: explicit Euler for Crank-Nicolson": ("mb_oracle", "M = np.linalg.solve(L, I + 0.5 * dt * A)", "M = I + dt * A", RATES),
    "populations: field drive dropped": ("mb_oracle", "+ m.reshape((4,) + (1,) * (N.ndim - 1)) * s", "+ 0.0 * s", COUPLING),
    "populations: drive with E^n only": ("mb_oracle", "0.5 * (E_old[c] + self.E[c]) * self.J[c]", "E_old[c] * self.J[c]", COUPLING),
    # Philox and the unit map
    "Philox: Weyl constant": ("mb_oracle", "PHILOX_W1 = 0xBB67AE85", "PHILOX_W1 = 0xBB67AE84", PHILOX),
    "Philox: words 1 and 3 swapped in the mix": ("mb_oracle", "c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0",
                                                 "c0, c1, c2, c3 = hi1 ^ c3 ^ k0, lo1, hi0 ^ c1 ^ k1, lo0", PHILOX),
    "unit map: 24 bits": ("mb_oracle", ">> np.uint32(9)).astype(np.float64) + 0.5) * 2.0 ** -23",
                          ">> np.uint32(8)).astype(np.float64) + 0.5) * 2.0 ** -23", PHILOX),
    "Box-Muller: radius without the 2": ("mb_oracle", "r01 = np.sqrt(-2.0 * np.log(u0))", "r01 = np.sqrt(-np.log(u0))", PHILOX),
    # probes and flux
    "DFT: dt weight dropped": ("mb_oracle", "self.E[c][k, j, i], pr[\"omegas\"], t, self.dt)", "self.E[c][k, j, i], pr[\"omegas\"], t, 1.0)", PROBES),
    "flux: E x H pairing sign": ("mb_oracle", "F = float(np.sum(Ea * Hb - Eb * Ha)) * dA", "F = float(np.sum(Ea * Hb + Eb * Ha)) * dA", PROBES),
    "flux: outward sign of the low faces": ("mb_oracle", "out.append(F if face % 2 == 1 else -F)", "out.append(F)", PROBES),
    "point spectrum: modulus not squared": ("mb_oracle", "return np.sum(np.abs(pr[\"acc\"]) ** 2, axis=0), pr[\"lams\"].copy()",
                                            "return np.sum(np.abs(pr[\"acc\"]), axis=0), pr[\"lams\"].copy()", PROBES),
    "face spectrum: E x H pairing sign": ("mb_oracle", "S = np.real(Ea * np.conj(Hb) - Eb * np.conj(Ha))",
                                          "S = np.real(Ea * np.conj(Hb) + Eb * np.conj(Ha))", FACE),
    "face spectrum: low faces not turned outward": ("mb_oracle", "return (S if face % 2 == 1 else -S), fp[\"lams\"].copy()",
                                                    "return S, fp[\"lams\"].copy()", FACE),
    "face spectrum: sub-grid area": ("mb_oracle", "S = S.reshape(-1, K).sum(axis=0) * (fp[\"stride\"] * self.dx) ** 2",
                                     "S = S.reshape(-1, K).sum(axis=0) * self.dx ** 2", FACE),
    # NEXT-1: CW source, plane probes, energy density
    "CW: rise inverted": ("mb_oracle", "* (1.0 - math.exp(-((t - t0) / tau) ** 2))", "* math.exp(-((t - t0) / tau) ** 2)", MODEMAP),
    "plane probe: sampling interval left out of the weight": ("mb_oracle", "ph = np.exp(1j * pp[\"omegas\"] * t) * (pp[\"every\"] * self.dt)",
                                                              "ph = np.exp(1j * pp[\"omegas\"] * t) * self.dt", MODEMAP),
    "plane probe: E^n sampled": ("mb_oracle", "pp[\"acc\"][:, c] += self.E[c][pp[\"k\"]]", "pp[\"acc\"][:, c] += E_old[c][pp[\"k\"]]", MODEMAP),
    "energy density: eps_r dropped": ("mb_oracle", "* EPS0 * self.eps_r[k]", "* EPS0", MODEMAP),
    # NEXT-4: bound state of -phi'' + tau^2 phi + phi^3 = E phi
    "GP: potential sign": ("gp_oracle", "(tau * tau + phi * phi - E) * phi", "(-tau * tau + phi * phi - E) * phi", GP),
    "GP: nonlinearity dropped": ("gp_oracle", "(tau * tau + phi * phi - E) * phi", "(tau * tau - E) * phi", GP),
    "GP: nonlinearity sign": ("gp_oracle", "(tau * tau + phi * phi - E) * phi", "(tau * tau - phi * phi - E) * phi", GP),
    "GP: carried int phi'^2 of phi": ("gp_oracle", "phi * phi, dphi * dphi, tau", "phi * phi, phi * dphi, tau", GP),
    "GP: carried int tau^2 phi^2 without tau": ("gp_oracle", "tau * tau * phi * phi, phi ** 4", "phi * phi, phi ** 4", GP),
    "GP: shooting verdicts swapped": ("gp_oracle", "        if kind < 0:\n            lo = mid", "        if kind > 0:\n            lo = mid", GP),
    "GP: spectral peak normalisation": ("gp_oracle", "p_phi = st.I0 ** 2 / (4.0 * math.pi ** 2)", "p_phi = st.I0 ** 2 / (2.0 * math.pi)", GP),
    "GP: waist from int phi^2": ("gp_oracle", "sig2 = st.I2 / st.I1", "sig2 = st.I3 / st.I1", GP),
    "GP: waist without the 2 pi": ("gp_oracle", "return math.sqrt(sig2) / (2.0 * math.pi), p_phi", "return math.sqrt(sig2), p_phi", GP),
    "GP: E(p) with p for sqrt p": ("gp_oracle", "return (p - 1.0) / (kappa * np.sqrt(p))", "return (p - 1.0) / (kappa * p)", GP),
    "GP: threshold root sign": ("gp_oracle", "+ kappa * math.sqrt(4.0 + kappa ** 2) / 2.0", "- kappa * math.sqrt(4.0 + kappa ** 2) / 2.0", GP),
    # NEXT-2: spectral statistics
    "analysis: emission slope against the energy ratio alone": ("mb_analysis",
        "g = math.log(emitted[q + 1] / emitted[q]) / math.log(levels[q + 1] / levels[q])",
        "g = math.log(emitted[q + 1] / emitted[q])", ANALYSIS),
    "analysis: emitted energy from the peak bin": ("mb_analysis",
        "em = [float(np.sum(spectra[i])) for i in idx]", "em = [float(np.max(spectra[i])) for i in idx]", ANALYSIS),
    "analysis: unweighted mean": ("mb_analysis", "mean = (S * w).sum() / tot", "mean = w.mean()", ANALYSIS),
    "analysis: width over bins": ("mb_analysis", "return math.sqrt((S * (w - mean) ** 2).sum() / tot)",
                                  "return math.sqrt((S * (w - mean) ** 2).sum() / S.size)", ANALYSIS),
    "analysis: fit centre sign": ("mb_analysis", "return float(x0 - b / (2.0 * c))", "return float(x0 + b / (2.0 * c))", ANALYSIS),
    "analysis: fit width without the 2": ("mb_analysis", "float(math.sqrt(-1.0 / (2.0 * c)))", "float(math.sqrt(-1.0 / c))", ANALYSIS),
    "analysis: threshold at a tenth off": ("mb_analysis", "if r[\"std_w\"] <= 0.5 * rows[0][\"std_w\"]:", "if r[\"std_w\"] <= 0.9 * rows[0][\"std_w\"]:", ANALYSIS),
    # the discrete adjoint
    "adjoint: psi_E memory coefficient dropped": ("mb_adjoint", "coef = sign * u[_COMP[c]] + cc * tot", "coef = sign * u[_COMP[c]]", ADJ),
    "adjoint: psi_H memory coefficient dropped": ("mb_adjoint", "coef = sign * v[_COMP[c]] + cc * tot\n            F = _COMP[_other(key)]\n            lE0",
                                                  "coef = sign * v[_COMP[c]]\n            F = _COMP[_other(key)]\n            lE0", ADJ),
    "adjoint: noise amplitude derivative dropped": ("mb_adjoint", "lN[2] += gf * cF * dsig", "lN[2] += 0.0 * gf * cF * dsig", ADJ),
    "adjoint: PEC mask dropped": ("mb_adjoint", "lEt = [mask[c] * lE1[c] for c in range(3)]", "lEt = [lE1[c] for c in range(3)]", ADJ),
    "adjoint: population source sign": ("mb_adjoint", "lJ1[c] += ls * 0.5", "lJ1[c] -= ls * 0.5", ADJ),
    "adjoint: inversion derivative dropped": ("mb_adjoint", "lN[1] += ldN", "lN[1] += 0 * ldN", ADJ),
    "adjoint: M untransposed": ("mb_adjoint", "np.tensordot(M.T, lN", "np.tensordot(M, lN", ADJ),
    "adjoint: P -> J term dropped": ("mb_adjoint", "lJt = [lJ1[c] + dt * lP[c]", "lJt = [lJ1[c] + 0 * lP[c]", ADJ),
    "adjoint: objective's E^n half dropped": ("mb_adjoint", "lE0[0][p, sy, sx] += 0.5 * w", "lE0[0][p, sy, sx] += 0.0 * w", ADJ),
    "adjoint: pump derivative of m dropped": ("mb_adjoint", "+ dm.reshape(4, 1, 1, 1) * s", "+ 0 * dm.reshape(4, 1, 1, 1) * s", ADJ),
    "adjoint: noise of the next step": ("mb_adjoint", "langevin_normals(o.seed, o.cell_index, s0[\"n\"])",
                                        "langevin_normals(o.seed, o.cell_index, s1[\"n\"])", ADJ),
    "adjoint: coupling term sign": ("mb_adjoint", "lE0[c] += gf * cF * gc[\"xi\"] * dNn", "lE0[c] -= gf * cF * gc[\"xi\"] * dNn", ADJ),
}


def _mutant_module(name, old, new):
    path = os.path.join(ROOT, "oracle", name + ".py")
    with open(path) as f:
        src = f.read()
    assert src.count(old) == 1, f"edit site not found exactly once in oracle/{name}.py: {old!r}"
    mod = types.ModuleType("oracle." + name)
    mod.__file__ = path
    mod.__package__ = "oracle"
    sys.modules[mod.__name__] = mod
    exec(compile(src.replace(old, new), f"<mutant of oracle/{name}.py>", "exec"), mod.__dict__)
    return mod


def _fails_a_pin(name, old, new, pins):
    import oracle
    keys = tuple("oracle." + m for m in ORACLE_MODULES) + PIN_MODULES
    saved = {k: sys.modules.get(k) for k in keys}
    saved_attr = {m: getattr(oracle, m, None) for m in ORACLE_MODULES}
    try:
        for m in ORACLE_MODULES:
            importlib.import_module("oracle." + m)
        _mutant_module(name, old, new)
        if name == "mb_oracle":             # modules that import names from the forward oracle
            for m in ("mb_adjoint", "mb_analysis"):
                sys.modules.pop("oracle." + m, None)
                importlib.import_module("oracle." + m)
        for m in ORACLE_MODULES:            # `from oracle import m` reads the package attribute
            setattr(oracle, m, sys.modules["oracle." + m])
        for k in PIN_MODULES:
            sys.modules.pop(k, None)
        for module, fn, kwargs in pins:
            tm = importlib.import_module(module)
            pin = getattr(tm, fn)
            # a pin parametrized over the golden rows runs on all of them
            calls = [dict(zip(("ctr", "key", "expect"), r)) for r in tm._kat_rows()] \
                if isinstance(kwargs, str) else [kwargs]
            try:
                with np.errstate(all="ignore"):
                    for kw in calls:
                        pin(**kw)
            except Exception:               # an assertion, or the mutant breaking down
                return True
        return False
    finally:
        for k, v in saved.items():
            if v is None:
                sys.modules.pop(k, None)
            else:
                sys.modules[k] = v
        for m, v in saved_attr.items():
            if v is None:
                if hasattr(oracle, m):
                    delattr(oracle, m)
            else:
                setattr(oracle, m, v)


def test_pins_pass_on_the_oracle_itself():
    """The harness itself: with an edit that changes nothing, every pin set passes."""
    for pins in (CAVITY, CPML, LORENTZ, NOISE, RATES, COUPLING, PROBES, FACE, PHILOX, MODEMAP, GP, ANALYSIS, ADJ):
        assert not _fails_a_pin("mb_oracle", "def rate_matrix(", "def rate_matrix(", pins)


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(mutant):
    name, old, new, pins = MUTANTS[mutant]
    assert _fails_a_pin(name, old, new, pins), f"no pin fails with the mutant '{mutant}'"
