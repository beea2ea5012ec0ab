"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake -- a dropped term, a wrong sign, index or
constant, a transposed operand -- in a private copy of the oracle's C sources,
builds that copy into its own library, and runs the pin meant to catch it
against the planted oracle: the pin must fail.  The planted copies live in a
temporary directory; the oracle under test is never modified.
"""
import concurrent.futures as cf
import importlib
import importlib.util
import os
import shutil
import sys

import pytest

from paper_2605_25963_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_DIR = os.path.join(ROOT, "oracle")
TESTS_DIR = os.path.dirname(os.path.abspath(__file__))


def _tab(o):
    return o.Tables.build(W.MATERIAL_CODES)


def _mesh(o, det):
    return o.Mesh.build(o.Det(**det.as_dict()))


# name, source file, text, planted text, pin (module, function), pin arguments from the planted oracle
MUTANTS = [
    # Philox4x32-10 and the streams
    ("philox_nine_rounds", "orc_rng.c", "round < 10;", "round < 9;",
     ("test_oracle_rng", "test_philox_matches_curand_host_generator"), lambda o: {"seed": 1}),
    ("philox_weyl_constant", "orc_rng.c", "#define PHILOX_W1 0xBB67AE85u", "#define PHILOX_W1 0xBB67AE86u",
     ("test_oracle_rng", "test_philox_matches_curand_host_generator"), lambda o: {"seed": 0xDEADBEEF}),
    ("u01_half_offset_dropped", "orc_rng.c", "(double)(2u * (x >> 9) + 1u)", "(double)(2u * (x >> 9))",
     ("test_oracle_rng", "test_uniform_exact_and_open_interval"), None),
    ("stream_history_words_swapped", "orc_rng.c",
     "uint32_t ctr[4] = { 0u, (uint32_t)hid, (uint32_t)(hid >> 32), inst };",
     "uint32_t ctr[4] = { 0u, (uint32_t)(hid >> 32), (uint32_t)hid, inst };",
     ("test_oracle_rng", "test_stream_layout"), None),
    ("transport_stream_off_layout", "orc_transport.c", "r->ctr[3] = inst;", "r->ctr[3] = inst + 1u;",
     ("test_oracle_transport", "test_point_and_pencil_sources"), None),
    # photon cross sections and tables
    ("kn_total_wrong_term", "orc_xs.c", "double t3 = (1.0 + 3.0 * k) / (a * a);",
     "double t3 = (1.0 + 2.0 * k) / (a * a);",
     ("test_oracle_xs", "test_kn_total_equals_integral_of_differential"), lambda o: {"E": 662.0}),
    ("kn_sin2_sign", "orc_xs.c", "(P + 1.0 / P - s2)", "(P + 1.0 / P + s2)",
     ("test_oracle_xs", "test_kn_thomson_limit"), None),
    ("photoabsorption_energy_power", "orc_xs.c", "pow(ORC_MEC2 / E_keV, 3.5)", "pow(ORC_MEC2 / E_keV, 3.0)",
     ("test_oracle_xs", "test_photoabsorption_model"), None),
    ("pair_threshold_power", "orc_xs.c", "(double)Z * Z * r * r * r;", "(double)Z * Z * r * r;",
     ("test_oracle_xs", "test_pair_model"), None),
    ("water_one_hydrogen", "orc_xs.c", "m->A[0] = 1.008;  m->cnt[0] = 2;", "m->A[0] = 1.008;  m->cnt[0] = 1;",
     ("test_oracle_xs", "test_material_compositions"), None),
    ("table_no_interpolation", "orc_xs.c",
     "out[c] = (1.0 - f) * (double)row[k] + f * (double)row[k + 1];",
     "out[c] = (1.0 - f) * (double)row[k] + f * (double)row[k];",
     ("test_oracle_xs", "test_tables_grid_and_interpolation"), None),
    # charged particles
    ("water_mean_excitation", "orc_xs.c", "case ORC_MAT_WATER: return 75.0;", "case ORC_MAT_WATER: return 85.0;",
     ("test_oracle_electron", "test_water_stopping_power_and_range_match_estar"), lambda o: {"tab": _tab(o)}),
    ("bethe_F_sign", "orc_xs.c", "(2.0 * tau + 1.0) * log(2.0)", "(2.0 * tau - 1.0) * log(2.0)",
     ("test_oracle_electron", "test_water_stopping_power_and_range_match_estar"), lambda o: {"tab": _tab(o)}),
    ("radiative_share_scale", "orc_xs.c", "Zr * (T_keV * 1e-3) / 800.0", "Zr * (T_keV * 1e-3) / 700.0",
     ("test_oracle_electron", "test_stopping_power_shape"), None),
    ("range_simpson_weight", "orc_xs.c", "4.0 * range_integrand(codes[m], 0.5 * (a + b))",
     "2.0 * range_integrand(codes[m], 0.5 * (a + b))",
     ("test_oracle_electron", "test_range_table_and_inversion_against_brute_force"), lambda o: {"tab": _tab(o)}),
    ("range_inversion_direction", "orc_xs.c", "if (orc_e_range(t, m, exp(mid)) < left) lo = mid;",
     "if (orc_e_range(t, m, exp(mid)) > left) lo = mid;",
     ("test_oracle_electron", "test_range_table_and_inversion_against_brute_force"), lambda o: {"tab": _tab(o)}),
    ("track_density_inverted", "orc_transport.c",
     "orc_e_energy_after(cx->xs, mat, T, (t_next - t_cur) * sc)",
     "orc_e_energy_after(cx->xs, mat, T, (t_next - t_cur) / sc)",
     ("test_oracle_electron", "test_track_leaving_through_the_top_face"),
     lambda o: {"tab": _tab(o), "bare": _mesh(o, W.BARE_CYLINDER)}),
    ("track_dead_layer_counted_active", "orc_transport.c", "if (active) *edep += weight * (T - T2);",
     "*edep += weight * (T - T2);",
     ("test_oracle_electron", "test_track_from_active_volume_into_dead_layer"),
     lambda o: {"tab": _tab(o), "coax": _mesh(o, W.COAX_P)}),
    ("compton_electron_momentum_sign", "orc_transport.c", "E * eu[2] - Ep * dir[2]", "E * eu[2] + Ep * dir[2]",
     ("test_oracle_electron", "test_compton_electron_direction_in_a_thin_slab"), None),
    # sampling
    ("kahn_branch_probability", "orc_transport.c", "(1.0 + 2.0 * k) / (9.0 + 2.0 * k)",
     "(1.0 + 2.0 * k) / (8.0 + 2.0 * k)",
     ("test_oracle_transport", "test_kahn_sampler_klein_nishina"), lambda o: {"E": 662.0}),
    ("kahn_acceptance", "orc_transport.c", "r3 <= 0.5 * (c * c + 1.0 / x)", "r3 <= 0.5 * (c * c + 1.0 / (x * x))",
     ("test_oracle_transport", "test_kahn_sampler_klein_nishina"), lambda o: {"E": 662.0}),
    ("isotropic_hemisphere", "orc_transport.c", "double c = 2.0 * rng_u(r) - 1.0;", "double c = rng_u(r);",
     ("test_oracle_transport", "test_point_and_pencil_sources"), None),
    ("disk_radius_not_sqrt", "orc_transport.c", "double rr = src->radius * sqrt(rng_u(r));",
     "double rr = src->radius * rng_u(r);",
     ("test_oracle_transport", "test_source_moments"), None),
    # transport
    ("compton_cosine_sign", "orc_transport.c",
     "double c = 1.0 - (x - 1.0) / k;\n                        double phi",
     "double c = (x - 1.0) / k - 1.0;\n                        double phi",
     ("test_oracle_transport", "test_compton_angle_backscatter_fraction"), lambda o: {"E": 662.0, "alpha": 0.0}),
    ("rotation_frame_sign", "orc_transport.c", "n[2] = d[2] * c - s * r * cp;", "n[2] = d[2] * c + s * r * cp;",
     ("test_oracle_transport", "test_compton_direction_into_a_finite_catcher"), None),
    ("compton_energy_not_deposited", "orc_transport.c", "dep = E - Ep;", "dep = 0.0 * (E - Ep);",
     ("test_oracle_transport", "test_coax_energy_conservation_and_parity"), lambda o: {"E": 59.5}),
    ("process_selection_index", "orc_transport.c", "if (u < mu3[0]) proc = 0;", "if (u < mu3[1]) proc = 0;",
     ("test_oracle_transport", "test_first_interaction_frequencies"), None),
    ("free_flight_half_length", "orc_transport.c", "double lam = -log(rng_u(&r));",
     "double lam = -0.5 * log(rng_u(&r));",
     ("test_oracle_transport", "test_slab_transmission"), None),
    ("boundary_unscaled_attenuation", "orc_transport.c", "lam -= mu * len;", "lam -= mu_unit * len;",
     ("test_oracle_transport", "test_density_scaled_two_slab_transmission"), lambda o: {"s1": 1.7, "s2": 1.0}),
    ("pair_one_rest_mass", "orc_transport.c", "else dep = E - 2.0 * ORC_MEC2;", "else dep = E - ORC_MEC2;",
     ("test_oracle_transport", "test_pair_production_deposits"), None),
    ("escape_not_counted", "orc_transport.c", "esc += E; E = 0.0; alive = 0;", "E = 0.0; alive = 0;",
     ("test_oracle_transport", "test_coax_energy_conservation_and_parity"), lambda o: {"E": 59.5}),
    ("gradient_score_sign", "orc_transport.c", "score[grp] += 1.0 / sc - mu_unit * d_int;",
     "score[grp] += 1.0 / sc + mu_unit * d_int;",
     ("test_oracle_transport", "test_dos_gradient_interaction_term"), None),
    ("gradient_boundary_term_dropped", "orc_transport.c",
     "if (grp >= 0 && grp < o->n_group) score[grp] -= mu_unit * len;", "",
     ("test_oracle_transport", "test_dos_gradient_slab_identity"), None),
    # geometry and localisation
    ("edge_volume_operands_swapped", "orc_transport.c", "cross3(pb, pc, x); double e1",
     "cross3(pc, pb, x); double e1",
     ("test_oracle_transport", "test_black_absorber_solid_angle"), None),
    ("entering_sign", "orc_transport.c", "*entering = dn < 0;", "*entering = dn > 0;",
     ("test_oracle_transport", "test_coax_energy_conservation_and_parity"), lambda o: {"E": 59.5}),
    ("nearest_hit_entering_inverted", "orc_transport.c", "*entering = be;", "*entering = !be;",
     ("test_oracle_mesh", "test_nearest_hit_against_prism_clipping"), None),
    ("nearest_hit_ignores_t_min", "orc_transport.c", "if (th > t_min && th < bt)", "if (th > 0.0 && th < bt)",
     ("test_oracle_mesh", "test_nearest_hit_against_prism_clipping"), None),
    ("parity_any_crossing", "orc_transport.c", "if ((count[i] & 1) && first[i] < bt)",
     "if ((count[i] > 0) && first[i] < bt)",
     ("test_oracle_mesh", "test_parity_rule_locates_known_points"), None),
    # mesh generation
    ("open_edges_always_zero", "orc_mesh.c", "    free(e);\n    return bad;\n}\n\nint orc_mesh_euler",
     "    free(e);\n    return 0 * bad;\n}\n\nint orc_mesh_euler",
     ("test_oracle_mesh", "test_open_edges_detects_holes_and_flips"), None),
    ("side_quad_winding", "orc_mesh.c", "add_tri(b, A1, B0, B1, solid);", "add_tri(b, A1, B1, B0, solid);",
     ("test_oracle_mesh", "test_bare_cylinder_counts_volume_topology"), None),
    ("active_volume_grows", "orc_mesh.c", "add_rounded_g(&b, 4, D[1] - D[3], rch_a,",
     "add_rounded_g(&b, 4, D[1] + D[3], rch_a,",
     ("test_oracle_mesh", "test_coax_solids"), None),
    ("active_rounding_not_shrunk", "orc_mesh.c", "double rch_a = D[2] - D[3] > 0.0 ? D[2] - D[3] : 0.0;",
     "double rch_a = D[2];",
     ("test_oracle_mesh", "test_coax_solids"), None),
    ("bore_vacuum_not_separated", "orc_mesh.c", "z_back + 3.0 * sep, N, nphi, 1);", "z_back + 2.0 * sep, N, nphi, 1);",
     ("test_oracle_mesh", "test_coax_solids"), None),
    ("bore_contact_parent", "orc_mesh.c", "set_solid(m, 5, ORC_MAT_GE, 0, -1, 4);",
     "set_solid(m, 5, ORC_MAT_GE, 0, -1, 3);",
     ("test_oracle_transport", "test_coax_energy_conservation_and_parity"), lambda o: {"E": 1332.0}),
    ("active_flag_dropped", "orc_mesh.c", "set_solid(m, 4, ORC_MAT_GE, 1, 2, 3);", "set_solid(m, 4, ORC_MAT_GE, 0, 2, 3);",
     ("test_oracle_mesh", "test_coax_solids"), None),
    ("rounding_z_sign", "orc_mesh.c", "double zz = z_front - rch * (1.0 - sin(phi));",
     "double zz = z_front - rch * (1.0 - cos(phi));",
     ("test_oracle_mesh", "test_coax_solids"), None),
    ("ring_angle_half_step", "orc_mesh.c",
     "double th = 2.0 * ORC_PI * (double)i / (double)N;\n                add_vertex(b, rho[k]",
     "double th = 2.0 * ORC_PI * ((double)i + 0.5) / (double)N;\n                add_vertex(b, rho[k]",
     ("test_oracle_mesh", "test_bare_cylinder_counts_volume_topology"), None),
    ("disk_ring_spacing", "orc_mesh.c", "const double w = 4.0 * (2.0 * ORC_PI * R / (double)N);",
     "const double w = 3.0 * (2.0 * ORC_PI * R / (double)N);",
     ("test_oracle_mesh", "test_coax_solids"), None),
    ("disk_ring_count_off_by_one", "orc_mesh.c", "long m = lround((double)N * r / R);",
     "long m = lround((double)N * r / R) + 1;",
     ("test_oracle_mesh", "test_coax_solids"), None),
    ("disk_band_winding", "orc_mesh.c", "add_tri(b, a0 + i % na, b0 + j % nb, a0 + (i + 1) % na, solid);",
     "add_tri(b, a0 + i % na, a0 + (i + 1) % na, b0 + j % nb, solid);",
     ("test_oracle_mesh", "test_coax_solids"), None),
]


def _plant(root, name, fname, old, new):
    d = os.path.join(root, name)
    shutil.copytree(ORACLE_DIR, d, ignore=shutil.ignore_patterns("*.so", "*.tmp*", "__pycache__"))
    path = os.path.join(d, fname)
    text = open(path).read()
    assert text.count(old) == 1, (name, "planting site must occur exactly once")
    with open(path, "w") as f:
        f.write(text.replace(old, new))
    spec = importlib.util.spec_from_file_location("oracle_planted_" + name, os.path.join(d, "oracle.py"))
    mod = importlib.util.module_from_spec(spec)
    sys.modules[spec.name] = mod          # dataclasses look their module up there
    spec.loader.exec_module(mod)
    mod.build(force=True)
    return mod


@pytest.fixture(scope="module")
def planted(orc, tmp_path_factory):
    """Every planted oracle, built in parallel (gcc per copy)."""
    root = str(tmp_path_factory.mktemp("planted"))
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        futs = {m[0]: ex.submit(_plant, root, *m[:4]) for m in MUTANTS}
        return {k: f.result() for k, f in futs.items()}


def test_planting_sites_are_unique():
    names = [m[0] for m in MUTANTS]
    assert len(set(names)) == len(names)
    for name, fname, old, new, _, _ in MUTANTS:
        assert open(os.path.join(ORACLE_DIR, fname)).read().count(old) == 1, name
        assert old != new


def test_unplanted_pins_pass(orc):
    """The pins used below pass on the oracle itself with the same arguments."""
    if TESTS_DIR not in sys.path:
        sys.path.insert(0, TESTS_DIR)
    seen = set()
    for _, _, _, _, (mod, fn), args in MUTANTS:
        kw = args(orc) if args else {}
        sig = (mod, fn, tuple(sorted((k, v) for k, v in kw.items() if isinstance(v, float))))
        if sig in seen:
            continue
        seen.add(sig)
        getattr(importlib.import_module(mod), fn)(orc, **kw)


@pytest.mark.parametrize("case", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_catches_planted_mistake(planted, case):
    name, _, _, _, (mod, fn), args = case
    if TESTS_DIR not in sys.path:
        sys.path.insert(0, TESTS_DIR)
    o = planted[name]
    f = getattr(importlib.import_module(mod), fn)
    kw = args(o) if args else {}
    with pytest.raises(AssertionError):
        f(o, **kw)
