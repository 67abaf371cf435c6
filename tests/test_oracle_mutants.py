"""The oracle's pins catch plausible mistakes planted in the oracle.

Each case copies oracle/pyronn_oracle.c, turns one expression into a plausible mistake (a dropped
term, a wrong sign or index, a transposed operand, a half-voxel offset, a wrong normalisation),
compiles the copy with the oracle's own build step into a temporary library, loads a second
instance of the oracle's Python wrapper on it and runs the pins named beside the mistake: every one
of them must fail. A copy without a planted mistake, built and loaded the same way, passes all of
them. The acquisition-artifact references (oracle/artifacts.py) get the same treatment against
their pin, from a copy of the module loaded under another name. The oracle itself is never
modified; everything happens on the CPU.
"""
import importlib.util
import os
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle
import test_oracle_pins as pins

# (mistake, original text, planted text, pins that must fail as (name,) or (name, parameter))
MUTANTS = [
    # forward projector (Sec. 2.1, ray-driven)
    ("hat basis twice as wide", "double a = 1.0 - fabs(s);", "double a = 1.0 - 0.5 * fabs(s);",
     [("test_axis_aligned_rays_are_exact_discrete_line_sums",)]),
    ("FP interpolation with x and y transposed",
     "double w = hat(q[0] - i) * hat(q[1] - j) * hat(q[2] - k);",
     "double w = hat(q[0] - j) * hat(q[1] - i) * hat(q[2] - k);",
     [("test_axis_aligned_3d_rays_trilinear",)]),
    ("FP without the step length dt", "return g->dt * acc;", "return acc;",
     [("test_axis_aligned_rays_are_exact_discrete_line_sums",)]),
    ("samples at k dt instead of (k + 1/2) dt", "double t = (k + 0.5) * g->dt;", "double t = k * g->dt;",
     [("test_brute_force_system_matrix", "parallel")]),
    ("half-voxel shift of the y index", "q[1] = (X[1] - g->oy) / g->sy + 0.5 * (g->ny - 1);",
     "q[1] = (X[1] - g->oy) / g->sy + 0.5 * g->ny;", [("test_brute_force_system_matrix", "parallel")]),
    ("ray reference point on the wrong side", "out->c[i] = a[i] + tau * d[i];", "out->c[i] = a[i] - tau * d[i];",
     [("test_brute_force_system_matrix", "cone")]),
    ("sample range half the volume diagonal", "return (long)ceil(R / g->dt) + 2;",
     "return (long)ceil(0.5 * R / g->dt);", [("test_brute_force_system_matrix", "cone_wide_fan")]),
    ("support box drops the last z slab", "q[2] > -1.0 && q[2] < g->nz;", "q[2] > -1.0 && q[2] < g->nz - 1;",
     [("test_axis_aligned_3d_rays_trilinear",)]),
    ("support box drops the first x slab", "return q[0] > -1.0 && q[0] < g->nx", "return q[0] > 0.0 && q[0] < g->nx",
     [("test_axis_aligned_rays_are_exact_discrete_line_sums",)]),
    ("support box clipped at the voxel edges along y", "q[1] > -1.0 && q[1] < g->ny",
     "q[1] > -0.5 && q[1] < g->ny - 0.5", [("test_fp_is_continuous_in_the_geometry",)]),
    ("FP interpolation clamps to the edge instead of zero padding",
     "                if (i < 0 || i >= g->nx || j < 0 || j >= g->ny || k < 0 || k >= g->nz) continue;\n"
     "                double w = hat(q[0] - i) * hat(q[1] - j) * hat(q[2] - k);\n"
     "                s += w * vol[((size_t)k * g->ny + j) * g->nx + i];",
     "                double w = hat(q[0] - i) * hat(q[1] - j) * hat(q[2] - k);\n"
     "                long ic = i < 0 ? 0 : (i >= g->nx ? g->nx - 1 : i), jc = j < 0 ? 0 : (j >= g->ny ? g->ny - 1 : j);\n"
     "                long kc = k < 0 ? 0 : (k >= g->nz ? g->nz - 1 : k);\n"
     "                s += w * vol[((size_t)kc * g->ny + jc) * g->nx + ic];",
     [("test_axis_aligned_rays_are_exact_discrete_line_sums",), ("test_fp_is_continuous_in_the_geometry",)]),
    ("ray direction with u and v swapped",
     "d[i] = Mi[3 * i + 0] * u + Mi[3 * i + 1] * v + Mi[3 * i + 2];",
     "d[i] = Mi[3 * i + 0] * v + Mi[3 * i + 1] * u + Mi[3 * i + 2];", [("test_brute_force_system_matrix", "cone")]),
    ("ray origin with the wrong sign",
     "a[i] = -(Mi[3 * i + 0] * r[3] + Mi[3 * i + 1] * r[7] + Mi[3 * i + 2] * r[11]);",
     "a[i] = (Mi[3 * i + 0] * r[3] + Mi[3 * i + 1] * r[7] + Mi[3 * i + 2] * r[11]);",
     [("test_brute_force_system_matrix", "cone")]),
    ("ray reference point ignores the volume offset", "double C[3] = {g->ox, g->oy, g->oz};",
     "double C[3] = {0.0, 0.0, 0.0};", [("test_volume_offset_is_a_world_translation",)]),
    ("sample index adds the volume offset", "q[0] = (X[0] - g->ox) / g->sx", "q[0] = (X[0] + g->ox) / g->sx",
     [("test_volume_offset_is_a_world_translation",)]),
    ("sampled rays read one ray further", "for (long i = 0; i < n; ++i) out[i] = fp_one(g, vol, (long)ids[i]);",
     "for (long i = 0; i < n; ++i) out[i] = fp_one(g, vol, (long)ids[i] + 1);",
     [("test_fp_rays_and_bp_voxels_subsets_match_full",)]),
    ("sample count includes samples outside the support box", "total += in_box(g, q);", "total += 1;",
     [("test_constant_volume_axis_ray_and_sample_count",)]),
    ("parallel ray origin with the u offset subtracted",
     "double su = (u - 0.5 * (g->nu - 1)) * g->du + g->ou;", "double su = (u - 0.5 * (g->nu - 1)) * g->du - g->ou;",
     [("test_axis_aligned_rays_are_exact_discrete_line_sums",)]),
    ("parallel ray origin with the v spacing of u",
     "double sv = (v - 0.5 * (g->nv - 1)) * g->dv + g->ov;", "double sv = (v - 0.5 * (g->nv - 1)) * g->du + g->ov;",
     [("test_axis_aligned_3d_rays_trilinear",)]),
    # matched adjoint (Sec. 2.2)
    ("adjoint without dt", "vol[((size_t)kk * g->ny + j) * g->nx + i] += y * g->dt * w;",
     "vol[((size_t)kk * g->ny + j) * g->nx + i] += y * w;", [("test_dot_product_adjoint", "parallel")]),
    ("adjoint with x and y transposed", "double w = hat(q[0] - i) * hat(q[1] - j) * hat(q[2] - kk);",
     "double w = hat(q[0] - j) * hat(q[1] - i) * hat(q[2] - kk);", [("test_dot_product_adjoint", "fan")]),
    # voxel-driven back-projector (Sec. 2.1)
    ("BP projection with u and v swapped", "*u = a / c; *v = b / c; *w = c;", "*u = b / c; *v = a / c; *w = c;",
     [("test_bp_single_pixel_footprint",)]),
    ("BP weight 1 / w instead of 1 / w^2", "1.0 / (w * w) : 1.0;", "1.0 / w : 1.0;",
     [("test_bp_partition_of_unity_and_depth_weights",)]),
    ("BP bilinear taps transposed", "s += q[(size_t)vv * g->nu + uu] * hat(u - uu) * hat(v - vv);",
     "s += q[(size_t)vv * g->nu + uu] * hat(u - vv) * hat(v - uu);", [("test_parallel_bp_constant_along_rays",)]),
    ("BP voxel centre at (N / 2) instead of (N - 1) / 2", "double X[3] = {(i - 0.5 * (g->nx - 1)) * g->sx + g->ox,",
     "double X[3] = {(i - 0.5 * g->nx) * g->sx + g->ox,", [("test_bp_single_pixel_footprint",)]),
    ("BP voxel centre subtracts the z offset", "(k - 0.5 * (g->nz - 1)) * g->sz + g->oz};",
     "(k - 0.5 * (g->nz - 1)) * g->sz - g->oz};", [("test_volume_offset_is_a_world_translation",)]),
    ("BP keeps voxels behind the source", "if (g->kind == 1 && !(w > 0.0)) continue;", "",
     [("test_bp_voxels_behind_the_source_receive_nothing",)]),
    ("parallel BP detector offset with the wrong sign", "- g->ou) / g->du + 0.5 * (g->nu - 1);",
     "+ g->ou) / g->du + 0.5 * (g->nu - 1);", [("test_parallel_bp_detector_offset",)]),
    ("BP detector taps clamp to the edge instead of zero padding",
     "                if (uu < 0 || uu >= g->nu || vv < 0 || vv >= g->nv) continue;\n"
     "                s += q[(size_t)vv * g->nu + uu] * hat(u - uu) * hat(v - vv);",
     "                long uc = uu < 0 ? 0 : (uu >= g->nu ? g->nu - 1 : uu), vc = vv < 0 ? 0 : (vv >= g->nv ? g->nv - 1 : vv);\n"
     "                s += q[(size_t)vc * g->nu + uc] * hat(u - uu) * hat(v - vv);",
     [("test_bp_voxels_behind_the_source_receive_nothing",), ("test_parallel_bp_detector_offset",)]),
    ("sampled voxels read one voxel further",
     "for (long i = 0; i < n; ++i) out[i] = bp_one(g, sino, weight_mode, (long)ids[i]);",
     "for (long i = 0; i < n; ++i) out[i] = bp_one(g, sino, weight_mode, (long)ids[i] + 1);",
     [("test_fp_rays_and_bp_voxels_subsets_match_full",)]),
    # geometry (Sec. 2.4)
    ("pixel (0, 0) half a pixel off along u", "D0[i] = Dc[i] + (ou - 0.5 * (nu - 1) * du) * a[i]",
     "D0[i] = Dc[i] + (ou - 0.5 * nu * du) * a[i]", [("test_listing1_geometry_pins",)]),
    ("pixel (0, 0) v offset with the wrong sign", "(ov - 0.5 * (nv - 1) * dv) * b[i];",
     "(ov + 0.5 * (nv - 1) * dv) * b[i];", [("test_projection_matches_independent_intersection",)]),
    ("source-detector column of M reversed", "M[3 * i + 2] = D0[i] - S[i];", "M[3 * i + 2] = S[i] - D0[i];",
     [("test_listing1_geometry_pins",)]),
    ("3x3 inverse with a cofactor sign flipped", "out[1] = (m[2] * m[7] - m[1] * m[8]) * id;",
     "out[1] = (m[1] * m[8] - m[2] * m[7]) * id;", [("test_projection_matches_independent_intersection",)]),
    ("detector u axis mirrored", "eu[3 * n + 0] = -s;", "eu[3 * n + 0] = s;",
     [("test_projection_matches_independent_intersection",)]),
    ("angular step range / (V - 1)", "double step = angular_range / n_views;",
     "double step = angular_range / (n_views - 1);", [("test_listing1_geometry_pins",)]),
    ("helix not centred on z = 0", "double z = pitch * (n - 0.5 * (n_views - 1)) * step / (2.0 * M_PI);",
     "double z = pitch * n * step / (2.0 * M_PI);", [("test_helical_orbit_advance_and_centring",)]),
    ("normalisation keeps a negative scale", "if (w < 0) kappa = -kappa;", "",
     [("test_positions_equal_circular_and_normalisation",)]),
    # filtered back-projection (Sec. 2.2)
    ("FBP without the cosine pre-weight", "pw[m] = c * row[m];", "pw[m] = row[m];",
     [("test_fdk_cosine_weight_from_independent_geometry",)]),
    ("FBP distance ratio not squared", "pi / g->n_views * ratio * ratio / tau;", "pi / g->n_views * ratio / tau;",
     [("test_fdk_reconstructs_a_ball",)]),
    ("FBP pixel pitch not scaled to the volume centre", "tau = ratio * pu;", "tau = pu;",
     [("test_fdk_reconstructs_a_ball",)]),
    ("FBP source-detector distance inverted", "sdd = 1.0 / nn;", "sdd = nn;",
     [("test_fdk_cosine_weight_from_independent_geometry",)]),
    ("Ram-Lak odd taps with the wrong sign", "return -1.0 / (pi * pi * (double)k * (double)k);",
     "return 1.0 / (pi * pi * (double)k * (double)k);", [("test_ramp_taps_are_the_band_limited_ramp", 0)]),
    ("Shepp-Logan taps with 4 k^2 + 1", "return -2.0 / (pi * pi * (4.0 * (double)k * (double)k - 1.0));",
     "return -2.0 / (pi * pi * (4.0 * (double)k * (double)k + 1.0));",
     [("test_ramp_taps_are_the_band_limited_ramp", 1)]),
    ("FBP angular weight 2 pi / V", "const double scale = pi / g->n_views", "const double scale = 2.0 * pi / g->n_views",
     [("test_ramp_filter_dc_and_nyquist_response", 0)]),
]


# the same for the acquisition-artifact references (oracle/artifacts.py, Sec. 2.4); the pin is
# check_artifact_references
ARTIFACT_MUTANTS = [
    ("row jitter shifts the wrong way", "src = u - int(s[n, v])", "src = u + int(s[n, v])"),
    ("column jitter shifts the wrong way", "src = v - int(s[n, u])", "src = v + int(s[n, u])"),
    ("noise without the mean", "+ mean + std * np.asarray(noise", "+ std * np.asarray(noise"),
    ("noise scaled by the variance", "std * np.asarray(noise, dtype=np.float64)",
     "std * std * np.asarray(noise, dtype=np.float64)"),
    ("ring gain added instead of multiplied", "*= float(gain)", "+= float(gain)"),
    ("ring view range includes its end", "out[view_begin:view_end, :, int(c)]",
     "out[view_begin:view_end + 1, :, int(c)]"),
    ("blur kernel not centred", "t = j - 0.5 * (length - 1)", "t = j - 0.5 * length"),
    ("blur along the mirrored angle", "v + t * sa)", "v - t * sa)"),
    ("blur weight 1 / (L - 1)", "out[n, v, u] = acc / length", "out[n, v, u] = acc / max(length - 1, 1)"),
    ("blur bilinear weights swapped in v", "for dy, wy in ((0, 1.0 - fy), (1, fy)):",
     "for dy, wy in ((0, fy), (1, 1.0 - fy)):"),
]


def _load_copy(name, src_text, tmp):
    """A second instance of the oracle wrapper whose library is built from src_text."""
    init = os.path.join(os.path.dirname(oracle.__file__), "__init__.py")
    spec = importlib.util.spec_from_file_location(name, init)
    mod = importlib.util.module_from_spec(spec)
    sys.modules[name] = mod
    spec.loader.exec_module(mod)
    mod._SRC = os.path.join(tmp, name + ".c")
    mod._LIB_PATH = os.path.join(tmp, "lib" + name + ".so")
    with open(mod._SRC, "w") as f:
        f.write(src_text)
    return mod


@pytest.fixture(scope="module")
def copies(tmp_path_factory):
    tmp = str(tmp_path_factory.mktemp("oracle_mutants"))
    with open(oracle._SRC) as f:
        src = f.read()
    mods = {"control": _load_copy("oracle_control", src, tmp)}
    for i, (label, old, new, _) in enumerate(MUTANTS):
        assert src.count(old) == 1, f"{label}: the original text must occur exactly once"
        mods[label] = _load_copy(f"oracle_mutant_{i}", src.replace(old, new), tmp)
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        list(ex.map(lambda m: m.build(force=True), mods.values()))
    yield mods
    for m in mods.values():
        sys.modules.pop(m.__name__, None)


def _run_pin(pin, mod):
    fn = getattr(pins, pin[0])
    return fn(mod) if len(pin) == 1 else fn(mod, pin[1])


def test_unplanted_copy_passes_every_listed_pin(copies):
    for pin in sorted({p for m in MUTANTS for p in m[3]}, key=str):
        _run_pin(pin, copies["control"])


@pytest.mark.parametrize("label", [m[0] for m in MUTANTS])
def test_planted_mistake_fails_its_pins(copies, label):
    pins_for = next(m[3] for m in MUTANTS if m[0] == label)
    for pin in pins_for:
        with pytest.raises(AssertionError):
            _run_pin(pin, copies[label])


@pytest.mark.parametrize("label", [m[0] for m in ARTIFACT_MUTANTS])
def test_planted_artifact_mistake_fails_its_pin(tmp_path, label):
    from oracle import artifacts
    with open(artifacts.__file__) as f:
        src = f.read()
    i, (_, old, new) = next((i, m) for i, m in enumerate(ARTIFACT_MUTANTS) if m[0] == label)
    assert src.count(old) == 1, f"{label}: the original text must occur exactly once"
    path = tmp_path / f"artifacts_mutant_{i}.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location(f"artifacts_mutant_{i}", str(path))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    with pytest.raises(AssertionError):
        pins.check_artifact_references(mod)
