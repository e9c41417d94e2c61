"""The pins catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of the oracle's C source (a flipped sign, a wrong
index or time level, a dropped factor, the wrong adjoint operator, a broken sponge or
fold), builds it, and runs the pins against it: at least one must fail.  Nothing here
touches the real oracle library or a GPU.
"""
import os

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "fwi_oracle.c")

MUTATIONS = {
    "coefficient sign": ("double sgn = (k % 2 == 1) ? 1.0 : -1.0;",
                         "double sgn = (k % 2 == 1) ? -1.0 : 1.0;"),
    "stencil index on x": ("og_at(g, u, iz, iy, ix - k))", "og_at(g, u, iz, iy, ix - k + 1))"),
    "stencil drops z": ("double lap = sz * iz2 + sx * ix2;", "double lap = sx * ix2;"),
    "update sign of u^{n-1}": ("2.0 * ucur[i] + g->W[i] * lap[i] - g->am[i] * uprev[i]",
                               "2.0 * ucur[i] + g->W[i] * lap[i] + g->am[i] * uprev[i]"),
    "source without dt^2": ("og_step(&g, b, a, c, lap, &q.src, s, dt * dt * w);",
                            "og_step(&g, b, a, c, lap, &q.src, s, dt * w);"),
    "trace one step early": ("og_sample(&q.rec, (int64_t)s * nrec + r, c);",
                             "og_sample(&q.rec, (int64_t)s * nrec + r, b);"),
    "adjoint applies L before W": ("for (int64_t i = 0; i < g->ncell; ++i) tmp[i] = g->W[i] * n1[i];",
                                   "for (int64_t i = 0; i < g->ncell; ++i) tmp[i] = n1[i];"),
    "imaging with u^{m-1}": ("og_laplacian(g, hist + (size_t)(m - a) * g->ncell, lap);",
                             "og_laplacian(g, hist + (size_t)(m - a - 1) * g->ncell, lap);"),
    "gradient fold drops 2": ("+= 2.0 * g.vc[i] * dt * dt * gW[i];", "+= g.vc[i] * dt * dt * gW[i];"),
    "sponge a- sign": ("g->am[i] = 1.0 - eta * dt / 2.0;", "g->am[i] = 1.0 + eta * dt / 2.0;"),
    "misfit not squared": ("phi += r * r;", "phi += fabs(r);"),
    "bf16 rounding truncates": ("x += 0x7fffu + lsb;", "x += 0u * lsb;"),
    "off-grid window dropped": ("const double win = fabs(r) <= 1.0 ? og_i0(OG_KB * sqrt(1.0 - r * r)) / norm : 0.0;",
                                "const double win = fabs(r) <= 1.0 ? 1.0 : 0.0;"),
    "off-grid taps shifted": ("*first = i0 - OG_HW + 1;", "*first = i0 - OG_HW;"),
}

# the pins run against each mutant (fast ones; each is a plain function of the module)
PINS = [
    pins.test_coefficients_8th_order_known_values,
    lambda: pins.test_coefficients_match_exact_moment_solution(4),
    lambda: pins.test_laplacian_modified_wavenumber(3, 4),
    lambda: pins.test_closed_box_energy_is_conserved(2, 4),
    pins.test_sponge_dissipates_energy,
    pins.test_sponge_reflection_is_small,
    lambda: pins.test_homogeneous_greens_function(2),
    lambda: pins.test_source_dot_product(2, 4),
    lambda: pins.test_gradient_directional_finite_difference(2),
    pins.test_gradient_pointwise_including_sponge_edge,
]


def _offgrid_pin():
    import test_offgrid_pins as offgrid
    offgrid.test_weights_interpolate_sampled_cosines((30, 40))


def _codec_pin():
    import test_oracle_codec as codec
    codec.test_bf16_conversion_is_nearest_even()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_a_pin_catches_the_mutation(name, tmp_path):
    old, new = MUTATIONS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"pattern for '{name}' not found exactly once"
    lib = oracle.compile_source(text.replace(old, new), str(tmp_path / "mutant.so"))
    caught = []
    with oracle.use_library(lib):
        for pin in PINS + [_codec_pin, _offgrid_pin]:
            try:
                pin()
            except (AssertionError, RuntimeError, FloatingPointError, ValueError):
                caught.append(getattr(pin, "__name__", "pin"))
                break
    assert caught, f"no pin caught the mutation '{name}'"
