"""The oracle's pins catch plausible mistakes.

Each case below plants one mistake in a copy of ``oracle/oracle.c`` (on the CPU,
in a temporary directory): a dropped term, a wrong sign, index or constant, a
transposed operand, an off-by-one bound.  The copy is compiled, swapped in for
the oracle's library, and the pins named beside the mistake are run against
it: at least one of them must fail.  None of the pins named here is the
comparison with the NumPy mirror, so each mistake is caught by what the paper
or the mathematics fixes, not by the oracle agreeing with a restatement of
itself.  The unaltered source, built the same way, passes the same pins.
"""
import functools
import os

import pytest

import oracle
import test_oracle_pins as pins

_SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

# pins by name, with the parameters of the parametrised ones bound
PIN = {
    "splitmix": pins.test_splitmix64_published_outputs,
    "nu_band": pins.test_axis_frequencies_uniform_on_band,
    "tiles": pins.test_tile_assignment_exact_including_ties_and_outside,
    "self_sim": pins.test_self_similarity_is_D_and_index_is_2beta_plus_psi,
    "linear": functools.partial(pins.test_bundling_is_linear, "tile"),
    "sinc": pins.test_similarity_is_sinc_kernel,
    "direct": functools.partial(pins.test_memory_form_equals_direct_point_sum, (2, 2), "tile"),
    "direct_global": functools.partial(pins.test_memory_form_equals_direct_point_sum, (1, 1),
                                       "global"),
    "sqrt_d": pins.test_single_point_at_cell_centre_decodes_to_sqrt_D,
    "frames": pins.test_tile_frame_equals_global_frame,
    "born": pins.test_nonlinearity_born_rule,
    "gauss": pins.test_entropy_constant_field_gauss_circle,
    "disk3": functools.partial(pins.test_entropy_equals_disk_correlation_with_zero_padding, 3),
    "delta": pins.test_entropy_delta_field_is_disk_shaped,
    "softmax": pins.test_softmax_psd_identities,
    "threshold": pins.test_classification_threshold_inclusive_in_float32,
}

# (id, source text, planted text, pins expected to catch it).  Every planted
# text keeps all memory accesses of the C code within their buffers.
MUTANTS = [
    ("splitmix_mixer_shift", "z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;",
     "z = (z ^ (z >> 31)) * 0xBF58476D1CE4E5B9ull;", ["splitmix"]),
    ("nu_band_twice_as_wide",
     "nu_x[k] = (float)((2.0 * ux - 1.0) * (0.5 / length_scale));",
     "nu_x[k] = (float)((2.0 * ux - 1.0) * (1.0 / length_scale));", ["nu_band", "sinc"]),
    ("tile_width_from_wrong_axis",
     "return (double)g->W * g->res / (double)g->tiles_x; }",
     "return (double)g->W * g->res / (double)g->tiles_y; }", ["tiles"]),
    ("tile_tie_to_last_minimum", "if (d2 < best_d2) { best_d2 = d2; best = k; }",
     "if (d2 <= best_d2) { best_d2 = d2; best = k; }", ["tiles"]),
    ("encode_conjugated", "omega[(m * nk + q) * 2 + 1] += sin(ph);",
     "omega[(m * nk + q) * 2 + 1] -= sin(ph);", ["direct", "sqrt_d"]),
    ("encode_axes_transposed", "double turns = (double)nu_x[k] * x + (double)nu_y[k] * y;",
     "double turns = (double)nu_x[k] * y + (double)nu_y[k] * x;", ["direct", "sqrt_d"]),
    ("memory_index_class_major", "size_t m = (size_t)(2 * beta[p] + labels[p]);",
     "size_t m = (size_t)(beta[p] + T * labels[p]);", ["self_sim"]),
    ("tile_frame_shift_sign", "                x -= cx;", "                x += cx;",
     ["frames", "direct"]),
    ("norm_without_sqrt", "norms[m] = sqrt(s);", "norms[m] = s;", ["sqrt_d", "direct"]),
    ("decode_without_conj", "acc += wr * cos(ph) + wi * sin(ph);",
     "acc += wr * cos(ph) - wi * sin(ph);", ["direct", "sqrt_d"]),
    ("decode_drops_imaginary_term", "acc += wr * cos(ph) + wi * sin(ph);",
     "acc += wr * cos(ph);", ["direct_global", "direct"]),
    ("cell_corner_not_centre",
     "        double x = g->x_min + ((double)cells[2 * c] + 0.5) * g->res;\n"
     "        double y = g->y_min + ((double)cells[2 * c + 1] + 0.5) * g->res;\n"
     "        int32_t beta = beta_cells",
     "        double x = g->x_min + (double)cells[2 * c] * g->res;\n"
     "        double y = g->y_min + ((double)cells[2 * c + 1] + 0.5) * g->res;\n"
     "        int32_t beta = beta_cells", ["sqrt_d", "direct"]),
    ("phase_in_half_turns", "#define ORC_TWO_PI 6.283185307179586476925286766559",
     "#define ORC_TWO_PI 3.1415926535897932384626433832795", ["sinc"]),
    ("born_rule_without_square", "Phat[c * ncell + q] = v * v;", "Phat[c * ncell + q] = v;",
     ["born"]),
    ("negative_maximum_kept", "double v = m > 0.0 ? P[c * ncell + q] / m : 0.0;",
     "double v = m != 0.0 ? P[c * ncell + q] / m : 0.0;", ["born"]),
    ("disk_radius_exclusive", "if (d2 > (int64_t)r * r) continue;",
     "if (d2 >= (int64_t)r * r) continue;", ["gauss", "disk3"]),
    ("disk_box_one_short", "x1 = x + r > W - 1 ? W - 1 : x + r;",
     "x1 = x + r > W - 1 ? W - 1 : x + r - 1;", ["disk3", "delta"]),
    ("entropy_sign", "if (v > 0.0) s -= v * log(v);", "if (v > 0.0) s += v * log(v);",
     ["gauss"]),
    ("entropy_log_base_2", "if (v > 0.0) s -= v * log(v);", "if (v > 0.0) s -= v * log2(v);",
     ["gauss", "disk3"]),
    ("softmax_classes_swapped", "pr1[q] = e1 / (e0 + e1);", "pr1[q] = e0 / (e0 + e1);",
     ["softmax"]),
    ("psd_sign", "ogm[q] = pr1[q] - pr0[q];", "ogm[q] = pr0[q] - pr1[q];", ["softmax"]),
    ("threshold_strict", "cls[q] = (uint8_t)(ogm[q] >= rho ? 1 : 0);",
     "cls[q] = (uint8_t)(ogm[q] > rho ? 1 : 0);", ["threshold"]),
]


def _build(tmp_path, name, find=None, plant=None):
    with open(_SRC) as f:
        src = f.read()
    if find is not None:
        assert src.count(find) == 1, f"{name}: the source text must occur exactly once"
        src = src.replace(find, plant)
    path = tmp_path / f"{name}.c"
    path.write_text(src)
    return oracle.bind(oracle.compile_source(str(path), str(tmp_path / f"lib{name}.so")))


def _failing(monkeypatch, lib, names):
    failed = []
    with monkeypatch.context() as mp:
        mp.setattr(oracle, "_lib", lib)
        for n in names:
            try:
                PIN[n]()
            except (AssertionError, ValueError):
                failed.append(n)
    return failed


def test_unaltered_source_passes_the_pins(tmp_path, monkeypatch):
    lib = _build(tmp_path, "unaltered")
    assert _failing(monkeypatch, lib, list(PIN)) == []


@pytest.mark.parametrize("name,find,plant,names", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, monkeypatch, name, find, plant, names):
    lib = _build(tmp_path, name, find, plant)
    failed = _failing(monkeypatch, lib, names)
    assert failed, f"{name}: none of {names} caught the planted mistake"
