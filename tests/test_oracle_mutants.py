"""Planted mistakes in the oracles, each failing a pin (test infrastructure, CPU only).

A pin earns its name only if a plausible mistake in the oracle fails it.  Each case below plants
one such mistake -- a dropped term, a wrong sign, factor or index, a one-sided choice -- in a copy
of an oracle source and checks that the named pin fails on that copy: the C++ hydro oracle is
rebuilt from its copy (same compiler flags) and swapped in through `oracle.load`; a Python oracle
module is executed from its copy and swapped into the pin's module.  The unmodified oracles pass
the same pins in their own files.  Nothing here touches the CUDA library.
"""
import os
import shutil
import subprocess
import time
import types

import pytest

import oracle
from oracle import build as obuild

import test_oracle_amr as pins_amr
import test_oracle_mhd as pins_mhd
import test_oracle_octs as pins_octs
import test_oracle_pins as pins_hydro
import test_oracle_ppm as pins_ppm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORK = os.path.join(ROOT, "tests", "_mutants")

# ------------------------------------------------------------------ C++ hydro oracle
# name: (source file, original text, planted text, pin, pin arguments)
HPP = "euler_oracle.hpp"
CPP = {
    "recovery: kinetic energy without its 1/2":
        (HPP, "T kin = T(0.5) * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / rho;",
         "T kin = (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / rho;",
         "test_first_step_of_single_jump_is_godunov_hllc", ()),
    "recovery: gamma in place of gamma - 1":
        (HPP, "T p = T(c.gamma - 1.0) * (U[4] - kin);", "T p = T(c.gamma) * (U[4] - kin);",
         "test_first_step_of_single_jump_is_godunov_hllc", ()),
    "MinMod: the larger difference":
        (HPP, "return (std::fabs(value(a)) <= std::fabs(value(b))) ? a : b;",
         "return (std::fabs(value(a)) >= std::fabs(value(b))) ? a : b;",
         "test_contact_advection_maximum_principle", ("minmod",)),
    "MC: 1 b in place of 2 b":
        (HPP, "T two_b = T(2.0) * b;", "T two_b = T(1.0) * b;", "test_mirror_symmetry", ("mc",)),
    "MC: slope kept at an extremum":
        (HPP, "  if (value(a) * value(b) <= 0.0) return T(0.0);\n  if (limiter == 0)",
         "  if (limiter == 0 && value(a) * value(b) <= 0.0) return T(0.0);\n  if (limiter == 0)",
         "test_first_step_of_a_zigzag_is_first_order_godunov", ("mc",)),
    "predictor: pressure equation without gamma":
        (HPP, "out[4] = T(c.gamma) * q[4] * dq[n] + un * dq[4];", "out[4] = q[4] * dq[n] + un * dq[4];",
         "test_sound_wave_second_order", ("none", 1.8, 4.0)),
    "predictor: dp * rho in place of dp / rho":
        (HPP, "out[n] = out[n] + dq[4] / q[0];", "out[n] = out[n] + dq[4] * q[0];",
         "test_sound_wave_second_order", ("none", 1.8, 4.0)),
    "predictor: density equation without rho du":
        (HPP, "out[0] = un * dq[0] + q[0] * dq[n];", "out[0] = un * dq[0];",
         "test_tangent_matches_central_differences", ("none",)),
    "flux: pressure dropped from the normal momentum flux":
        (HPP, "F[n] = F[n] + q[4];", "F[n] = F[n];", "test_hllc_consistency_equal_states", (0,)),
    "flux: energy flux without p u":
        (HPP, "F[4] = q[n] * (E + q[4]);", "F[4] = q[n] * E;", "test_hllc_consistency_equal_states", (0,)),
    "flux: kinetic energy without its 1/2":
        (HPP, "T E = q[4] / T(c.gamma - 1.0) + T(0.5) * q[0] * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);",
         "T E = q[4] / T(c.gamma - 1.0) + q[0] * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);",
         "test_hllc_consistency_equal_states", (0,)),
    "HLLC: Davis S_L takes the larger speed":
        (HPP, "T SL = (value(aL) <= value(bL)) ? aL : bL;", "T SL = (value(aL) >= value(bL)) ? aL : bL;",
         "test_mirror_symmetry", ("minmod",)),
    "HLLC: pressure difference reversed in S*":
        (HPP, "T Sstar = (qR[4] - qL[4] + qL[n] * mL - qR[n] * mR) / (mL - mR);",
         "T Sstar = (qL[4] - qR[4] + qL[n] * mL - qR[n] * mR) / (mL - mR);",
         "test_contact_advection_maximum_principle", ("minmod",)),
    "HLLC: star energy without the pressure term":
        (HPP, "Us[4] = fac * (UK[4] / q[0] + (Sstar - q[n]) * (Sstar + q[4] / mK));",
         "Us[4] = fac * (UK[4] / q[0] + (Sstar - q[n]) * Sstar);",
         "test_sound_wave_second_order", ("mc", 1.8, 1.0)),
    "HLLC: star state of the wrong side":
        (HPP, "const bool left = (0.0 <= value(Sstar));", "const bool left = (0.0 >= value(Sstar));",
         "test_contact_advection_maximum_principle", ("minmod",)),
    "face state: low side extrapolated the wrong way":
        (HPP, "qL[v] = qh.f[v][a] + T(0.5) * slope[d].f[v][a];", "qL[v] = qh.f[v][a] - T(0.5) * slope[d].f[v][a];",
         "test_mirror_symmetry", ("minmod",)),
    "face state: high side with the low cell's slope":
        (HPP, "qR[v] = qh.f[v][b] - T(0.5) * slope[d].f[v][b];", "qR[v] = qh.f[v][b] - T(0.5) * slope[d].f[v][a];",
         "test_mirror_symmetry", ("minmod",)),
    "predictor: a full step in place of a half step":
        (HPP, "const double hdt = 0.5 * dt / dx;", "const double hdt = dt / dx;",
         "test_sound_wave_second_order", ("none", 1.8, 4.0)),
    "update: z flux differenced against the y neighbour":
        (HPP, "(flux[2].f[v][a] - flux[2].f[v][mz]);", "(flux[2].f[v][a] - flux[2].f[v][my]);",
         "test_first_step_of_single_jump_is_godunov_hllc", ()),
    "CFL: one sound speed in place of three":
        (HPP, "double s = ((std::fabs(q[1]) + std::fabs(q[2])) + std::fabs(q[3])) + 3.0 * cs;",
         "double s = ((std::fabs(q[1]) + std::fabs(q[2])) + std::fabs(q[3])) + cs;", "test_cfl_bruteforce", ()),
    "initial map: kinetic energy without rho":
        (HPP, "U[4] = q[4] / T(c.gamma - 1.0) + T(0.5) * q[0] * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);",
         "U[4] = q[4] / T(c.gamma - 1.0) + T(0.5) * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);",
         "test_first_step_of_a_zigzag_is_first_order_godunov", ("minmod",)),
    # the derivative scalar types behind the oracle's tangent (J v) and tape adjoint (J^T w)
    "tangent: quotient rule with a plus":
        ("scalars.hpp", "return Dual(q, (a.d - q * b.d) / b.v);", "return Dual(q, (a.d + q * b.d) / b.v);",
         "test_tangent_matches_central_differences", ("none",)),
    "tangent: derivative of sqrt without the 1/2":
        ("scalars.hpp", "return Dual(s, a.d / (2.0 * s));", "return Dual(s, a.d / s);",
         "test_tangent_matches_central_differences", ("none",)),
    "adjoint: product partials exchanged":
        ("scalars.hpp", "return tv_make(a.v * b.v, a.i, b.v, b.i, a.v);", "return tv_make(a.v * b.v, a.i, a.v, b.i, b.v);",
         "test_adjoint_dot_product", ("none",)),
    "adjoint: quotient partial with the wrong sign":
        ("scalars.hpp", "return tv_make(q, a.i, 1.0 / b.v, b.i, -q / b.v);", "return tv_make(q, a.i, 1.0 / b.v, b.i, q / b.v);",
         "test_adjoint_dot_product", ("none",)),
    "adjoint: difference partial +1 for the subtrahend":
        ("scalars.hpp", "return tv_make(a.v - b.v, a.i, 1.0, b.i, -1.0);", "return tv_make(a.v - b.v, a.i, 1.0, b.i, 1.0);",
         "test_adjoint_dot_product", ("none",)),
    "adjoint: reverse sweep overwrites instead of accumulating":
        ("scalars.hpp", "if (n.b >= 0) adj[(size_t)n.b] += n.db * g;", "if (n.b >= 0) adj[(size_t)n.b] = n.db * g;",
         "test_adjoint_dot_product", ("none",)),
    "op count: division not counted":
        ("scalars.hpp", "{ ++op_counter(); ++op_kinds()[2]; return Counted(a.v / b.v); }",
         "{ ++op_kinds()[2]; return Counted(a.v / b.v); }", "test_op_counts_match_stage_formulas", ()),
}
CPP_SOURCES = ("oracle_capi.cpp", "euler_oracle.hpp", "scalars.hpp")


def _slug(name):
    return "".join(ch if ch.isalnum() else "_" for ch in name)[:60]


@pytest.fixture(scope="module")
def cpp_mutants():
    """Every C++ mutant built under tests/_mutants, one compiler per core at a time (removed
    afterwards)."""
    shutil.rmtree(WORK, ignore_errors=True)
    procs, libs = {}, {}
    width = max(1, os.cpu_count() or 1)
    for name, (fname, old, new, _, _) in CPP.items():
        d = os.path.join(WORK, _slug(name))
        os.makedirs(d)
        for src in CPP_SOURCES:
            with open(os.path.join(ROOT, "oracle", src)) as f:
                text = f.read()
            if src == fname:
                assert text.count(old) == 1, name
                text = text.replace(old, new)
            with open(os.path.join(d, src), "w") as f:
                f.write(text)
        libs[name] = os.path.join(d, "mutant.so")
        while sum(p.poll() is None for p in procs.values()) >= width:
            time.sleep(0.05)
        procs[name] = subprocess.Popen(obuild.command([os.path.join(d, "oracle_capi.cpp")], libs[name]))
    for name, p in procs.items():
        assert p.wait() == 0, name
    yield libs
    shutil.rmtree(WORK, ignore_errors=True)


@pytest.mark.parametrize("name", sorted(CPP))
def test_cpp_oracle_mutant_fails_its_pin(name, cpp_mutants, monkeypatch):
    _, _, _, pin, args = CPP[name]
    monkeypatch.setattr(oracle, "_lib", oracle.load(cpp_mutants[name]))
    with pytest.raises(AssertionError):
        getattr(pins_hydro, pin)(*args)


# ------------------------------------------------------------------ Python oracles
# name: (module, original text, planted text, pin module, pin, pin arguments)
PY = {
    # MHD with GLM cleaning
    "MHD: magnetic pressure |B|^2 in place of |B|^2/2":
        ("mhd", "pt = p + 0.5 * B2", "pt = p + B2", pins_mhd, "test_linear_magnetosonic_waves_converge",
         ("fast", "none", 1.9)),
    "MHD: energy flux without B (u.B)":
        ("mhd", "F[4] = (E + pt) * un - Bn * uB", "F[4] = (E + pt) * un", pins_mhd,
         "test_linear_magnetosonic_waves_converge", ("fast", "none", 1.9)),
    "MHD: momentum flux without the Maxwell stress":
        ("mhd", "F[1 + k] = rho * un * q[1 + k] - Bn * q[5 + k]", "F[1 + k] = rho * un * q[1 + k]", pins_mhd,
         "test_linear_magnetosonic_waves_converge", ("slow", "none", 1.9)),
    "MHD: induction flux sign":
        ("mhd", "F[5 + k] = un * q[5 + k] - q[1 + k] * Bn", "F[5 + k] = un * q[5 + k] + q[1 + k] * Bn", pins_mhd,
         "test_linear_magnetosonic_waves_converge", ("fast", "none", 1.9)),
    "MHD: GLM face B_n with the psi jump's sign flipped":
        ("mhd", "Bm = 0.5 * (BnL + BnR) - (psiR - psiL) / (2.0 * ch)",
         "Bm = 0.5 * (BnL + BnR) + (psiR - psiL) / (2.0 * ch)", pins_mhd,
         "test_glm_face_characteristic_invariants", ()),
    "MHD: GLM face psi with c_h in place of c_h / 2":
        ("mhd", "pm = 0.5 * (psiL + psiR) - 0.5 * ch * (BnR - BnL)", "pm = 0.5 * (psiL + psiR) - ch * (BnR - BnL)",
         pins_mhd, "test_glm_face_characteristic_invariants", ()),
    "MHD: psi flux c_h B_n in place of c_h^2 B_n":
        ("mhd", "F[8] = ch * ch * Bn              # psi's flux", "F[8] = ch * Bn", pins_mhd,
         "test_hll_consistency_and_upwinding", ()),
    "MHD: normal field flux without psi":
        ("mhd", "F[5 + d] = q[8]                 # the normal field's flux is psi", "F[5 + d] = 0.0 * q[8]",
         pins_mhd, "test_hll_consistency_and_upwinding", ()),
    "MHD: psi damping without c_h":
        ("mhd", "out[8] = out[8] * np.exp(-ALPHA * ch * dt / dx)", "out[8] = out[8] * np.exp(-ALPHA * dt / dx)",
         pins_mhd, "test_uniform_state_unchanged_and_conservation", ()),
    "MHD: c_h without the 1/3 of three axes":
        ("mhd", "return (cfg.cfl / 3.0) * dx / dt", "return cfg.cfl * dx / dt", pins_mhd,
         "test_uniform_state_unchanged_and_conservation", ()),
    "MHD: fast speed discriminant with 2 a^2 b_n^2":
        ("mhd", "s * s - 4.0 * a2 * bn2", "s * s - 2.0 * a2 * bn2", pins_mhd, "test_fast_speed_closed_forms", ()),
    "MHD: HLL S_R ignoring the right state's fast speed":
        ("mhd", "SR = np.maximum(qL[n] + cL, qR[n] + cR)", "SR = np.maximum(qL[n] + cL, qR[n])", pins_mhd,
         "test_mirror_symmetry", ("minmod",)),
    "MHD: HLL average over S_R + S_L":
        ("mhd", "SL * SR * (UR - UL)) / (SR - SL)", "SL * SR * (UR - UL)) / (SR + SL)", pins_mhd,
         "test_hll_consistency_and_upwinding", ()),
    "MHD: predictor advancing the low states backwards":
        ("mhd", "recover(conserved(lo[d], cfg) - h * dF, cfg)", "recover(conserved(lo[d], cfg) + h * dF, cfg)",
         pins_mhd, "test_mirror_symmetry", ("minmod",)),
    "MHD: predictor over a full step":
        ("mhd", "h = 0.5 * dt / dx", "h = dt / dx", pins_mhd, "test_circularly_polarised_alfven_wave_converges",
         ("none", 1.9)),
    "MHD: recovery without the magnetic energy":
        ("mhd", "p = np.maximum((cfg.gamma - 1.0) * ((U[4] - kin) - mag), cfg.p_floor)",
         "p = np.maximum((cfg.gamma - 1.0) * (U[4] - kin), cfg.p_floor)", pins_mhd,
         "test_linear_magnetosonic_waves_converge", ("fast", "none", 1.9)),
    "MHD: conserved energy without the magnetic energy":
        ("mhd", "E = q[4] / (cfg.gamma - 1.0) + kin + mag", "E = q[4] / (cfg.gamma - 1.0) + kin", pins_mhd,
         "test_flux_tensor_symmetries", ()),
    "MHD: CFL from the mean speed":
        ("mhd", "return cfg.cfl * (dx / s.max())", "return cfg.cfl * (dx / s.mean())", pins_mhd,
         "test_cfl_bruteforce", ()),
    # PPM
    "PPM: the two steepening cases exchanged":
        ("ppm", "nL = np.where(ext, q, np.where(lo, 3.0 * q - 2.0 * qR, qL))\n"
                "    nR = np.where(ext, q, np.where(hi, 3.0 * q - 2.0 * qL, qR))",
         "nL = np.where(ext, q, np.where(hi, 3.0 * q - 2.0 * qR, qL))\n"
         "    nR = np.where(ext, q, np.where(lo, 3.0 * q - 2.0 * qL, qR))", pins_ppm,
         "test_edge_properties_on_rough_data", ()),
    "PPM: interface slope correction over 8 in place of 6":
        ("ppm", "(_sh(dq, 1, axis) - dq) / 6.0", "(_sh(dq, 1, axis) - dq) / 8.0", pins_ppm,
         "test_interfaces_exact_for_cubics", ()),
    "PPM: MC bounds 1x in place of 2x the one-sided differences":
        ("ppm", "np.minimum(2.0 * np.abs(dl), 2.0 * np.abs(dr))", "np.minimum(np.abs(dl), np.abs(dr))", pins_ppm,
         "test_interfaces_exact_for_cubics", ()),
    "PPM: extrema not flattened":
        ("ppm", "ext = (qR - q) * (q - qL) <= 0.0", "ext = (qR - q) * (q - qL) < -1e300", pins_ppm,
         "test_edge_properties_on_rough_data", ()),
    "PPM: low-edge steepening never applied":
        ("ppm", "lo = ~ext & (D * Q6 > D * D)", "lo = ~ext & (D * Q6 > 1e300)", pins_ppm,
         "test_edge_properties_on_rough_data", ()),
    "PPM: Q6 with 3 in place of 6":
        ("ppm", "Q6 = 6.0 * (q - 0.5 * (qL + qR))", "Q6 = 3.0 * (q - 0.5 * (qL + qR))", pins_ppm,
         "test_edge_properties_on_rough_data", ()),
    "PPM: low face state from the low edge":
        ("ppm", "qL = qh + (E[d][1] - q) ", "qL = qh + (E[d][0] - q) ", pins_ppm,
         "test_edge_form_with_plm_edges_is_the_plm_step", ("minmod",)),
    "PPM: predictor pressure equation without gamma":
        ("ppm", "out[4] = gamma * q[4] * D[n] + un * D[4]", "out[4] = q[4] * D[n] + un * D[4]", pins_ppm,
         "test_edge_form_with_plm_edges_is_the_plm_step", ("minmod",)),
    # oct bookkeeping
    "octs: y and z bits exchanged in the Morton key":
        ("octs", "key |= ((Y >> b) & 1) << (3 * b + 1)\n        key |= ((Z >> b) & 1) << (3 * b + 2)",
         "key |= ((Y >> b) & 1) << (3 * b + 2)\n        key |= ((Z >> b) & 1) << (3 * b + 1)", pins_octs,
         "test_morton_key_unit_values", ()),
    "octs: SFC order reversed":
        ("octs", 'return np.argsort(key, kind="stable")', 'return np.argsort(-key, kind="stable")', pins_octs,
         "test_sfc_order_is_the_recursive_octant_walk", ()),
    "octs: neighbour slot with x slowest":
        ("octs", "nbr[o, ((dz + 1) * 3 + (dy + 1)) * 3 + (dx + 1)] = where.get(q, -1)",
         "nbr[o, ((dx + 1) * 3 + (dy + 1)) * 3 + (dz + 1)] = where.get(q, -1)", pins_octs,
         "test_neighbour_table_against_pairwise_search", ()),
    "octs: stencil reads the neighbour slot with x slowest":
        ("octs", "n = nbr[o, ((z // 2) * 3 + y // 2) * 3 + x // 2]", "n = nbr[o, ((x // 2) * 3 + y // 2) * 3 + z // 2]",
         pins_octs, "test_table_step_equals_uniform_grid_step", ()),
    "octs: stencil reads the cell with x slowest":
        ("octs", "V[:, n, ((z % 2) * 2 + y % 2) * 2 + x % 2]", "V[:, n, ((x % 2) * 2 + y % 2) * 2 + z % 2]",
         pins_octs, "test_table_step_equals_uniform_grid_step", ()),
    "octs: oct-major copy with the cell axes reversed":
        ("octs", "transpose(0, 1, 3, 5, 2, 4, 6)", "transpose(0, 1, 3, 5, 6, 4, 2)", pins_octs,
         "test_level_oct_round_trip", ()),
    # AMR ghosts and refluxing
    "AMR: child offsets with the wrong sign":
        ("amr", "s = np.where(np.mod(f, 2) == 1, 0.25, -0.25)", "s = np.where(np.mod(f, 2) == 1, -0.25, 0.25)",
         pins_amr, "test_linear_field_reproduced_at_fine_centres", ()),
    "AMR: prolongation MinMod takes the larger difference":
        ("amr", "np.where(np.abs(a) <= np.abs(b), a, b)", "np.where(np.abs(a) <= np.abs(b), b, a)", pins_amr,
         "test_no_new_extrema_and_constant_field", ()),
    "AMR: time weights exchanged":
        ("amr", "w0 = 1.0 - float(theta)", "w0 = float(theta)", pins_amr, "test_time_interpolated_ghosts", ()),
    "AMR: reflux corrections with the wrong signs":
        ("amr", "for side, s in ((0, 1.0), (1, -1.0)):", "for side, s in ((0, -1.0), (1, 1.0)):", pins_amr,
         "test_refluxed_composite_step_conserves_to_round_off", ()),
    "AMR: fine face fluxes summed, not averaged":
        ("amr", "return 0.25 * (F[:, 0::2, 0::2]", "return 1.0 * (F[:, 0::2, 0::2]", pins_amr,
         "test_refluxed_composite_step_conserves_to_round_off", ()),
    "AMR: average-down over four children":
        ("amr", "mean = 0.125 * m.sum(axis=(2, 4, 6))", "mean = 0.25 * m.sum(axis=(2, 4, 6))", pins_amr,
         "test_refluxed_composite_step_conserves_to_round_off", ()),
    "AMR: sibling exchange reads one cell past an interior":
        ("amr", "inside = np.all(rel < dims[b][None, :], axis=1)", "inside = np.all(rel <= dims[b][None, :], axis=1)",
         pins_amr, "test_sibling_exchange_reassembles_a_partitioned_level", ()),
    # exact Riemann solver and Sedov-Taylor constant
    "Riemann: shock relation with gamma - 1 in place of gamma + 1":
        ("riemann_exact", "A = 2.0 / ((g + 1.0) * rho)", "A = 2.0 / ((g - 1.0) * rho)", pins_hydro,
         "test_exact_riemann_matches_toro_table", ()),
    "Riemann: rarefaction relation with the exponent inverted":
        ("riemann_exact", "    r = (p / pk) ** e\n", "    r = (p / pk) ** (1.0 / e)\n", pins_hydro,
         "test_exact_riemann_matches_toro_table", ()),
    "Riemann: star density behind a left shock without the ratio's gm":
        ("riemann_exact", "st = (rl * (ps / pl + gm) / (gm * ps / pl + 1.0), us, ps)",
         "st = (rl * (ps / pl) / (gm * ps / pl + 1.0), us, ps)", pins_hydro,
         "test_exact_riemann_matches_toro_table", ()),
    "Riemann: left fan velocity with the wrong sign of s":
        ("riemann_exact", "u = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + s)",
         "u = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul - s)", pins_hydro,
         "test_sod_converges_to_exact_solution", (1.4,)),
    "Sedov: momentum equation without the 3 phi / 2 source":
        ("sedov", "b = np.array([-2.0 * psi * phi / eta, 1.5 * phi, 3.0])",
         "b = np.array([-2.0 * psi * phi / eta, 0.0 * phi, 3.0])", pins_hydro,
         "test_sedov_constant_matches_tables", ()),
    "Sedov: energy integral without the kinetic 1/2":
        ("sedov", "dI = eta * eta * (0.5 * psi * phi * phi + f / (g - 1.0))",
         "dI = eta * eta * (psi * phi * phi + f / (g - 1.0))", pins_hydro,
         "test_sedov_constant_matches_tables", ()),
}


def _mutant_module(modname, old, new):
    path = os.path.join(ROOT, "oracle", modname + ".py")
    with open(path) as f:
        text = f.read()
    assert text.count(old) == 1, (modname, old)
    m = types.ModuleType("oracle." + modname)
    m.__package__ = "oracle"
    m.__file__ = path
    exec(compile(text.replace(old, new), path, "exec"), m.__dict__)
    return m


@pytest.mark.filterwarnings("ignore::RuntimeWarning")  # overflow and NaN in the planted copies
@pytest.mark.parametrize("name", sorted(PY))
def test_python_oracle_mutant_fails_its_pin(name, monkeypatch):
    modname, old, new, pins, pin, args = PY[name]
    monkeypatch.setattr(pins, modname, _mutant_module(modname, old, new))
    with pytest.raises(AssertionError):
        getattr(pins, pin)(*args)
