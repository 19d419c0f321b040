"""The oracle's pins catch planted mistakes.  Each case copies evd_oracle.c,
plants one plausible mistake (a dropped term, a flipped sign, swapped operands,
the wrong wall rule; the corrective forcing terms of Eq.
improved_forcing_scheme included), compiles the copy and runs the fast pins
against it: at least one pin must fail, and the pin expected to catch it must
be among them.  The unmodified copy, compiled the same way, passes every pin
(control).  The mistakes are planted in the oracle only, on the CPU."""
import gc
import inspect
import itertools

import pytest

from oracle import oracle as O

import test_oracle_collision as TC
import test_oracle_forcing as TF
import test_oracle_lattice as TL
import test_oracle_physics as TP
import test_oracle_stream as TS
import test_oracle_tau as TT


def _expand(fn):
    """Keyword sets of a test function's parametrize marks (their product)."""
    axes = []
    for m in getattr(fn, "pytestmark", []):
        if m.name != "parametrize":
            continue
        names = [n.strip() for n in m.args[0].split(",")] if isinstance(m.args[0], str) else list(m.args[0])
        sets = []
        for v in m.args[1]:
            vals = v.values if hasattr(v, "values") else ((v,) if len(names) == 1 else tuple(v))
            sets.append(dict(zip(names, vals)))
        axes.append(sets)
    out = []
    for combo in itertools.product(*axes):
        kw = {}
        for d in combo:
            kw.update(d)
        out.append(kw)
    return out


def _pins():
    pins = []
    for mod in (TC, TS, TT, TL, TF):
        for name, fn in inspect.getmembers(mod, inspect.isfunction):
            if name.startswith("test_") and fn.__module__ == mod.__name__:
                for kw in _expand(fn):
                    if set(inspect.signature(fn).parameters) == set(kw):
                        pins.append((name, fn, kw))
    # fast whole-step pins (no fixtures)
    for name in ("test_initial_state_is_at_rest_and_reads_back_its_fields",
                 "test_periodic_box_momentum_grows_by_the_total_force",
                 "test_shear_wave_decays_with_the_common_viscosity",
                 "test_force_field_of_zeros_and_uniform_field_reduce_to_plain_gravity"):
        fn = getattr(TP, name)
        for kw in _expand(fn):
            pins.append((name, fn, kw))
    return pins


PINS = _pins()


def _failing_pins(path):
    failed = set()
    with O.swapped_library(path):
        for name, fn, kw in PINS:
            try:
                fn(**kw)
            except Exception:   # an assertion, or the mutant oracle rejecting its own state
                failed.add(name)
        gc.collect()            # oracle states made by this library are freed by it
    return failed


# name: (text in evd_oracle.c, its replacement, a pin expected to fail)
MUTANTS = {
    "forcing-term-dropped-from-update": (
        "fstar[i * Q + a] = f[i * Q + a] + om_self + om_cross + (1.0 - dt / (2.0 * tau_i)) * S;",
        "fstar[i * Q + a] = f[i * Q + a] + om_self + om_cross;",
        "test_node_identities"),
    "forcing-second-order-sign": (
        "v += (ei[k] * ei[l] - cs2 * (k == l ? 1.0 : 0.0)) / (cs2 * cs2) * u[l];",
        "v -= (ei[k] * ei[l] - cs2 * (k == l ? 1.0 : 0.0)) / (cs2 * cs2) * u[l];",
        "test_node_identities"),
    "cross-collision-sign": (
        "om = -(1.0 / tau_x[i * ns + j])",
        "om = (1.0 / tau_x[i * ns + j])",
        "test_node_identities"),
    "half-force-shift-dropped": (
        "ueq[i][k] = mom[k] / rho[i] + F[i][k] * dt / (2.0 * rho[i]);",
        "ueq[i][k] = mom[k] / rho[i];",
        "test_node_identities"),
    "mixture-velocity-unweighted": (
        "u[k] += (rho[i] / rho_mix) * ueq[i][k];",
        "u[k] += ueq[i][k] / ns;",
        "test_node_identities"),
    "equilibrium-velocity-square-sign": (
        "- usq / (2.0 * cs2));",
        "+ usq / (2.0 * cs2));",
        "test_node_identities"),
    "f0-projection-without-mixture-velocity": (
        "proj += emu[k] * (ueq[i][k] - u[k]);",
        "proj += ei[k] * (ueq[i][k] - u[k]);",
        "test_node_identities"),
    "ternary-tau-diffusivities-swapped": (
        "const double t23 = (A23 - r1 * r2 / (A13 * D13 * D23)) / (B23 - r1 * B13 / (A13 * D23));",
        "const double t23 = (A23 - r1 * r2 / (A13 * D13 * D23)) / (B23 - r1 * B13 / (A13 * D13));",
        "test_ternary_closed_form_solves_the_system"),
    "ternary-tau12-species-index": (
        "const double t12 = 1.0 / (B12 / A12 - r3 / (A12 * D12 * t23));",
        "const double t12 = 1.0 / (B12 / A12 - r2 / (A12 * D12 * t23));",
        "test_ternary_closed_form_solves_the_system"),
    "species-speed-inverted": (
        "c[i] = sqrt(M1 / cfg->M[i]);",
        "c[i] = sqrt(cfg->M[i] / M1);",
        "test_species_speeds_and_equal_viscosity"),
    "viscosity-ratio-inverted": (
        "tau[i] = 0.5 + (cfg->tau1 - 0.5) * (cs2[0] / cs2[i]);",
        "tau[i] = 0.5 + (cfg->tau1 - 0.5) * (cs2[i] / cs2[0]);",
        "test_species_speeds_and_equal_viscosity"),
    "interpolation-weight-sign": (
        "return -s * (1.0 - s) / 2.0;",
        "return s * (1.0 - s) / 2.0;",
        "test_streaming_conserves_each_species_mass"),
    "wall-rule-reversed": (
        "const int b = (dot > 0) ? st->opp[a] : a;",
        "const int b = (dot < 0) ? st->opp[a] : a;",
        "test_wall_equations_of_appendix_a"),
    "s-diff-factor": (
        "Xc[k] += dt / (2.0 * tau_i - dt) * th;",
        "Xc[k] += dt / (2.0 * tau_i) * th;",
        "test_s_diff_adds_no_mass_or_momentum_and_the_symmetric_second_moment"),
    "s-p-sign": (
        "Xc[k] -= cs2 * grad[i * 3 + k];",
        "Xc[k] += cs2 * grad[i * 3 + k];",
        "test_gradient_terms_on_densities_linear_in_x"),
    "s-rho-without-mass-fraction": (
        "Yc[k] = (rho[i] / rho_mix) * grad[ns * 3 + k];",
        "Yc[k] = grad[ns * 3 + k];",
        "test_gradient_terms_on_densities_linear_in_x"),
    "lattice-gradient-scale": (
        "for (k = 0; k < 3; ++k) g[k] *= 3.0;",
        "for (k = 0; k < 3; ++k) g[k] *= 2.0;",
        "test_gradient_terms_on_densities_linear_in_x"),
    "initial-velocity-sign": (
        "ui0[k] = 0.0 - rho_i * a0[k] * dt / (2.0 * rho_i);",
        "ui0[k] = 0.0 + rho_i * a0[k] * dt / (2.0 * rho_i);",
        "test_initial_state_is_at_rest_and_reads_back_its_fields"),
    "readout-mole-fraction-without-molar-mass": (
        "if (x) x[(long)i * nsites + X] = dg.rho[i] / (dg.n * st->cfg.M[i]);",
        "if (x) x[(long)i * nsites + X] = dg.rho[i] / dg.n;",
        "test_initial_state_is_at_rest_and_reads_back_its_fields"),
    "force-field-ignored": (
        "a[k] = st->cfg.g[k] + (st->acc ? st->acc[(long)k * st->nsites + X] : 0.0);",
        "a[k] = st->cfg.g[k];",
        "test_force_field_of_zeros_and_uniform_field_reduce_to_plain_gravity"),
    "d3q19-weights-swapped": (
        "w[a] = (a == 0) ? 1.0 / 3.0 : (a <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);",
        "w[a] = (a == 0) ? 1.0 / 3.0 : (a <= 6 ? 1.0 / 36.0 : 1.0 / 18.0);",
        "test_weights_are_isotropic_with_cs2_one_third"),
    "z-stencil-dropped": (
        "for (d[2] = (Dm == 3 ? -1 : 0); d[2] <= (Dm == 3 ? 1 : 0); ++d[2])",
        "for (d[2] = 0; d[2] <= 0; ++d[2])",
        "test_streaming_conserves_each_species_mass"),
    "opposite-table-ignores-z": (
        "if (e[b][0] == -e[a][0] && e[b][1] == -e[a][1] && e[b][2] == -e[a][2]) opp[a] = b;",
        "if (e[b][0] == -e[a][0] && e[b][1] == -e[a][1] && e[b][2] == e[a][2]) opp[a] = b;",
        "test_weights_are_isotropic_with_cs2_one_third"),
    "wall-tie-to-opposite": (
        "const int b = (dot > 0) ? st->opp[a] : a;",
        "const int b = (dot >= 0) ? st->opp[a] : a;",
        "test_scatter_matches_gather_restatement"),
}


def test_unmodified_copy_passes_every_pin():
    assert len(PINS) > 40
    path = O.compile_variant(O.source(), "control")
    assert _failing_pins(path) == set()


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistake_is_caught(name):
    old, new, expected = MUTANTS[name]
    src = O.source()
    assert src.count(old) == 1, "the mutation's anchor must occur exactly once"
    path = O.compile_variant(src.replace(old, new), name.replace("-", "_"))
    failed = _failing_pins(path)
    assert expected in failed, (name, sorted(failed))
