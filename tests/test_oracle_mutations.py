"""Planted mistakes: each case builds a copy of the CPU oracle with one plausible mistake in it
(a dropped term, a wrong index, a wrong weight) and checks that the brute-force and invariant
pins of tests/test_oracle.py fail on it.  No GPU is involved; every planted mistake keeps
memory accesses in bounds, so the copies run in this process."""
import os
import subprocess

import pytest

import oracle
import test_oracle as T
from conftest import ROOT

ONE_HOP = [lambda: T.test_one_hop_splits_equally_among_cone_members_and_merges_photon_weighted(s)
           for s in (11, 12, 13)]
UNIFORM_VP = [T.test_virtual_particle_hop_in_a_uniform_medium_is_independent_of_its_position]
CHAIN_VP = [T.test_virtual_particle_shares_absorptions_by_sph_weight_and_neutral_density]
PLACEMENT = [lambda: T.test_virtual_particle_lands_uniformly_in_the_cone_part_of_the_smoothing_sphere(k)
             for k in (8, 32)]
REBIN = [lambda: T.test_rebin_moves_each_held_packet_to_the_new_cone_of_its_direction(n, sh)
         for n, sh in ((8, 0), (32, 0), (8, 1))]
EMISSION = [lambda: T.test_source_emission_is_complete_and_isotropic(e, k)
            for e, k in ((8, 1), (32, 2), (8, 4))]
CONE = [T.test_transmission_cone_solid_angle]
BIN = [T.test_reception_bin_is_nearest_rotated_axis]
RATES = [T.test_recombination_coefficients_match_paper,
         T.test_collisional_ionisation_cooling_removes_the_ionisation_energy]
COLLISIONAL = [T.test_collisional_rates_have_the_atomic_activation_energies,
               T.test_free_free_cooling_has_the_textbook_normalisation]
CHEM = [T.test_chemistry_photon_accounting_and_recombination_photons]
CHAIN = [T.test_beer_lambert_chain]
PHILOX = [T.test_philox_known_answers]
BARRIER = [T.test_barrier_test_is_exact_against_rational_arithmetic]
KNN = [lambda: T.test_knn_grid_equals_brute_force(k) for k in ("uniform", "clustered", "lattice")]
FLOOR = [T.test_subcycle_floor_hits_are_the_subcycles_the_floor_lengthened]
FIELD = [T.test_interior_field_is_the_attenuated_point_source_field]

# name: (text in the oracle, its replacement, the pins expected to catch it)
MUTATIONS = {
    "philox_multiplier": ("uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;",
                          "uint64_t p0 = (uint64_t)0xD2511F55u * (uint64_t)c0;", PHILOX),
    "barrier_crossing_sign": ("+ (__int128)sa * (2 * (b[i1] - a[i1]));",
                              "- (__int128)sa * (2 * (b[i1] - a[i1]));", BARRIER),
    "knn_ties_to_higher_index": ("return da < db || (da == db && ia < ib);",
                                 "return da < db || (da == db && ia > ib);", KNN),
    "knn_distance_without_z": ("return dx * dx + dy * dy + dz * dz;",
                               "return dx * dx + dy * dy + 0 * dz;", KNN),
    "cone_half_the_solid_angle": ("double c = 1.0 - 2.0 / (double)n_tc;",
                                  "double c = 1.0 - 1.0 / (double)n_tc;", CONE),
    "rotation_partly_transposed": ("double e0 = R[0] * d[0] + R[3] * d[1] + R[6] * d[2];",
                                   "double e0 = R[0] * d[0] + R[1] * d[1] + R[2] * d[2];", BIN),
    "case_b_coefficient_off": ("double aB = 2.753e-14 * pow(lam, 1.500)",
                               "double aB = 2.953e-14 * pow(lam, 1.500)", RATES),
    "ionisation_cooling_half_energy": ("double Lci = K_B * T_HI * beta;",
                                       "double Lci = 0.5 * K_B * T_HI * beta;", RATES),
    "free_free_wrong_power": ("double Lff = 1.42e-27 * 1.3 * sqrt(T);",
                              "double Lff = 1.42e-27 * 1.3 * pow(T, 0.45);", RATES),
    "free_free_gaunt_factor_doubled": ("double Lff = 1.42e-27 * 1.3 * sqrt(T);",
                                       "double Lff = 1.42e-27 * 2.6 * sqrt(T);", COLLISIONAL),
    "excitation_to_the_n3_level": ("double Lce = 7.5e-19 * exp(-118348.0 / T)",
                                   "double Lce = 7.5e-19 * exp(-140265.0 / T)", COLLISIONAL),
    "ionisation_boltzmann_factor_halved": ("pow(T, -1.5) * exp(-lam / 2.0)",
                                           "pow(T, -1.5) * exp(-lam / 4.0)", COLLISIONAL),
    "photoionisation_rate_per_atom_not_neutral": ("Gam = phot / (NHI * dt);",
                                                  "Gam = phot / (NH * dt);", CHEM),
    "optical_depth_with_total_density": ("double tau = (sig * s->nHI[j]) * l;",
                                         "double tau = (sig * s->nH[j]) * l;", CHAIN),
    "optical_depth_over_half_the_hop": ("double tau = (sig * s->nHI[j]) * l;",
                                        "double tau = (sig * s->nHI[j]) * (0.5 * l);", FIELD),
    "split_by_k_plus_1": ("double w = N / (double)m;", "double w = N / (double)(m + 1);", ONE_HOP),
    "first_member_only": ("for (int a = 0; a < m; ++a) deliver(",
                          "for (int a = 0; a < 1; ++a) deliver(", ONE_HOP),
    "clock_without_hop": ("s->nx[4][p] += T * (clock + l / C_LIGHT);",
                          "s->nx[4][p] += T * clock;", ONE_HOP),
    "clock_weighted_before_absorption": ("s->nx[4][p] += T * (clock + l / C_LIGHT);",
                                         "s->nx[4][p] += w * (clock + l / C_LIGHT);", ONE_HOP),
    "momentum_weighted_before_absorption": ("s->nx[1][p] += T * d[0];",
                                            "s->nx[1][p] += w * d[0];", ONE_HOP),
    "energy_weighted_before_absorption": ("s->nx[5][p] += T * eps;",
                                          "s->nx[5][p] += w * eps;", ONE_HOP),
    "sph_estimate_unnormalised": ("double nHIv = swn / sw;", "double nHIv = swn / (sw * 1.01);",
                                  UNIFORM_VP),
    "sph_estimate_by_count": ("double nHIv = swn / sw;", "double nHIv = swn / (double)kn;",
                              UNIFORM_VP),
    "virtual_clock_not_advanced": ("v.clock = clock + l / C_LIGHT;", "v.clock = clock;",
                                   UNIFORM_VP),
    "shares_without_neutral_density": ("double Ak = A * ((om[k] * s->nHI[j]) / swn);",
                                       "double Ak = A * (om[k] / sw);", CHAIN_VP),
    "weights_without_kernel": ("om[k] = (s->NH[j] / s->nH[j]) * kernel_w(qk);",
                               "om[k] = (s->NH[j] / s->nH[j]);", CHAIN_VP),
    "volume_as_atom_count": ("om[k] = (s->NH[j] / s->nH[j]) * kernel_w(qk);",
                             "om[k] = s->NH[j] * kernel_w(qk);", CHAIN_VP),
    "kernel_inner_branch": ("if (q <= 0.5) return 1.0 - 6.0 * q * q + 6.0 * q * q * q;",
                            "if (q <= 0.5) return 1.0 - 6.0 * q * q + 5.0 * q * q * q;", CHAIN_VP),
    "identity_not_mixed": ("v.fid = orc_mix64(fid);", "v.fid = fid + 1;", CHAIN_VP),
    "placement_without_cone": ("if (r2 > 0 && r2 <= h2 && orc_in_cone(del, d, n_tc)) found = 1;",
                               "if (r2 > 0 && r2 <= h2) found = 1;", PLACEMENT),
    "placement_sphere_2h": ("if (r2 > 0 && r2 <= h2 && orc_in_cone(del, d, n_tc)) found = 1;",
                            "if (r2 > 0 && r2 <= 4 * h2 && orc_in_cone(del, d, n_tc)) found = 1;",
                            PLACEMENT),
    "placement_fallback_at_h": ("double f = 0.5 * (double)H;", "double f = (double)H;", PLACEMENT),
    "placement_identity_truncated": ("(uint32_t)(fid >> 32)},", "0u},", PLACEMENT),
    "rebin_keeps_clock": ("            s->sl[4][p] += 0.0;\n",
                          "            s->sl[4][p] += tmp[4 * S + sl];\n", REBIN),
    "rebin_keeps_old_slot": ("            long long p = i * S + nu * nrc + b;\n            s->sl[0][p] += N;",
                             "            long long p = i * S + sl; (void)b;\n            s->sl[0][p] += N;",
                             REBIN),
    "rebin_moves_wrong_sum": ("if (s->sg && nu == 0) s->sg[i * nrc + b] += gold[sl];",
                              "if (s->sg && nu == 0) s->sg[i * nrc + b] += gold[b];", REBIN),
    "emission_split_by_n_ec_plus_1": (
        "p.N = s->ndot[j * nfs + nu] * s->cfg.dt_em / (double)nec;",
        "p.N = s->ndot[j * nfs + nu] * s->cfg.dt_em / (double)(nec + 1);", EMISSION),
    "floor_counted_on_the_last_subcycle": ("                if (h < dt - t) ++nfloor;",
                                           "                ++nfloor;", FLOOR),
    "floor_not_counted": ("                if (h < dt - t) ++nfloor;",
                          "                if (h < 0.0) ++nfloor;", FLOOR),
    "single_emission_per_step": (
        "        for (int k = 0; k < s->K; ++k)\n            for (int nu = 0; nu < nfs; ++nu)",
        "        for (int k = 0; k < 1; ++k)\n            for (int nu = 0; nu < nfs; ++nu)", EMISSION),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path, monkeypatch):
    old, new, pins = MUTATIONS[name]
    src = open(os.path.join(ROOT, "oracle", "traphic_oracle.c")).read()
    assert src.count(old) == 1, name
    (tmp_path / "traphic_oracle.c").write_text(src.replace(old, new))
    (tmp_path / "traphic_oracle.h").write_text(
        open(os.path.join(ROOT, "oracle", "traphic_oracle.h")).read())
    so = tmp_path / "liborc_mut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-o", str(so), str(tmp_path / "traphic_oracle.c"),
                           "-lm"])
    monkeypatch.setattr(oracle, "_lib", None)
    monkeypatch.setattr(oracle, "build", lambda force=False: str(so))
    caught = 0
    for pin in pins:
        try:
            pin()
        except AssertionError:
            caught += 1
    assert caught > 0, f"{name}: no pin failed"
