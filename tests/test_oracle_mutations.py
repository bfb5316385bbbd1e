"""Planted mistakes in the oracle fail its pins (CPU).

Each case below changes tnlm_oracle.c in one plausible way -- a sign, an
index, a dropped factor or term, a misread step order -- compiles the
changed copy with the oracle's own flags, and runs the oracle's pin tests
(projector, weights, solvers, outer-loop step order, Eq. 1's terms, FBP)
against it in a fresh
pytest process (TNLM_ORACLE_LIB points the oracle package at the copy).
At least one pin must fail for every case; the unchanged source, compiled
the same way, must pass them all.  The network oracle (unet_oracle.py) is
treated the same way: each changed copy is loaded as a module and its pins
(correlation, identity, adjoint pairs, finite-difference gradients, BF16
rounding) run against it.  The mistakes are planted in the oracle, on the
CPU; no GPU code is involved.
"""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "tnlm_oracle.c")
PINS = [os.path.join(HERE, f) for f in ("test_oracle_projector.py", "test_oracle_weights.py",
                                        "test_oracle_solvers.py", "test_oracle_outer_loop.py",
                                        "test_oracle_objective.py", "test_oracle_fbp.py")]

# name -> list of (text, replacement, which occurrence)
MUTATIONS = {
    "fan_angle_sign": [("double ux = cx * cos(gam) - cy * sin(gam);",
                        "double ux = cx * cos(gam) + cy * sin(gam);", 0),
                       ("double uy = cx * sin(gam) + cy * cos(gam);",
                        "double uy = -cx * sin(gam) + cy * cos(gam);", 0)],
    "segment_pixel_from_its_start": [("double am = 0.5 * (a_lo + a_hi);", "double am = a_lo;", 0)],
    "segment_length_without_ray_length": [("len[n] = (a_hi - a_lo) * d12;",
                                           "len[n] = (a_hi - a_lo);", 0)],
    "transpose_reads_phase_0": [("long r = (long)i * rays_per_phase + rr;", "long r = rr;", 0)],
    "weighted_residual_w_not_sqrt_w": [("r[k] = sqrt(w[k]) * (y[k] - t[k]);",
                                        "r[k] = w[k] * (y[k] - t[k]);", 0)],
    "cgls_b_inverted": [("double b = gnew / gam[i];", "double b = gam[i] / gnew;", 0)],
    "patch_one_column_short": [("for (int px = -r; px <= r; ++px)", "for (int px = -r; px < r; ++px)", 0)],
    "patch_l1_distance": [("            s += e * e;", "            s += fabs(e);", 0)],
    "h_not_squared": [("exp(-(dl[k] - dmin) / (h * h))", "exp(-(dl[k] - dmin) / h)", 0)],
    "weights_window_axes_swapped": [("int x1 = x + sx, y1 = yy + sy;", "int x1 = x + sy, y1 = yy + sx;", 0)],
    "weights_neighbours_swapped": [("int j = dir == 0 ? (i + 1) % N : (i + N - 1) % N;",
                                    "int j = dir == 0 ? (i + N - 1) % N : (i + 1) % N;", 0)],
    "jacobi_coefficient": [("mu_hat / (2.0 * mu_hat + 2.0)", "mu_hat / (mu_hat + 2.0)", 0)],
    "jacobi_forward_weights_for_both": [("sp += up[(long)y1 * nx + x1] * wp[k];",
                                         "sp += up[(long)y1 * nx + x1] * wn[k];", 0)],
    "weights_from_the_previous_iterate": [("orc_weights(NPH, NX, NY, g, d, W, h, wn, wp, NULL);",
                                           "orc_weights(NPH, NX, NY, f, d, W, h, wn, wp, NULL);", 0)],
    "jacobi_from_the_previous_iterate": [("orc_gj(NPH, NX, NY, W, g, use_n, use_p, mu_hat, m2, fn);",
                                          "orc_gj(NPH, NX, NY, W, f, use_n, use_p, mu_hat, m2, fn);", 0)],
    "no_positivity_step": [("if (fn[q] < 0.0) fn[q] = 0.0;", "if (fn[q] < -1e300) fn[q] = 0.0;", 0)],
    "gradient_step_sign": [("g[k] = f[k] - g[k] / beta;", "g[k] = f[k] + g[k] / beta;", 0)],
    "cgls_a_inverted": [("else a[i] = gam[i] / den;", "else a[i] = den / gam[i];", 0)],
    "cgls_residual_not_updated": [("r[i * nsg + k] -= a[i] * t[i * nsg + k];",
                                   "r[i * nsg + k] -= 0.0 * t[i * nsg + k];", 0)],
    "tnlm_term_neighbours_swapped": [("const int j = dir == 0 ? (i + N - 1) % N : (i + 1) % N;",
                                      "const int j = dir == 0 ? (i + 1) % N : (i + N - 1) % N;", 0)],
    "tnlm_term_unsquared": [("J += dv * dv * w[", "J += fabs(dv) * w[", 0)],
    "data_term_sqrt_w": [("data += w[k] * (t[k] - y[k]) * (t[k] - y[k]);",
                          "data += sqrt(w[k]) * (t[k] - y[k]) * (t[k] - y[k]);", 1)],
    "fbp_angular_step_halved": [("const double dbeta = 2.0 * ORC_PI / (double)M;",
                                 "const double dbeta = ORC_PI / (double)M;", 0)],
    "fbp_no_cosine_weight": [("acc += y[v * B + k] * SID * cos(gk) * c[n - k + B - 1];",
                              "acc += y[v * B + k] * SID * c[n - k + B - 1];", 0)],
}


def replace_nth(text, old, new, n):
    starts, i = [], text.find(old)
    while i >= 0:
        starts.append(i)
        i = text.find(old, i + 1)
    assert len(starts) > n, f"'{old}' not found in the oracle source"
    k = starts[n]
    return text[:k] + new + text[k + len(old):]


def run_pins(tmp_path, source_text, tag):
    import oracle
    src = tmp_path / f"{tag}.c"
    src.write_text(source_text)
    lib = str(tmp_path / f"lib{tag}.so")
    oracle.compile_source(str(src), lib)
    env = dict(os.environ, TNLM_ORACLE_LIB=lib, OMP_NUM_THREADS="4")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] + PINS,
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r


@pytest.fixture(scope="module")
def source():
    return open(SRC).read()


def test_unchanged_source_passes_the_pins(tmp_path, source):
    r = run_pins(tmp_path, source, "unchanged")
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_planted_mistake_fails_a_pin(tmp_path, source, name):
    text = source
    for old, new, n in MUTATIONS[name]:
        text = replace_nth(text, old, new, n)
    assert text != source
    r = run_pins(tmp_path, text, name)
    assert r.returncode == 1, f"no pin caught '{name}':\n{r.stdout[-2000:]}"


# ---------------------------------------------------------------- network oracle
UNET_SRC = os.path.join(ROOT, "oracle", "unet_oracle.py")
UNET_MUTATIONS = {
    "convolution_instead_of_correlation": [
        ('out += np.einsum("bchw,oc->bohw", xp[:, :, ky:ky + H, kx:kx + W], w[:, :, ky, kx])',
         'out += np.einsum("bchw,oc->bohw", xp[:, :, ky:ky + H, kx:kx + W], w[:, :, 2 - ky, 2 - kx])', 0)],
    "weight_gradient_taps_transposed": [("gw[:, :, ky, kx] = ", "gw[:, :, kx, ky] = ", 0)],
    "relu_mask_dropped_in_the_decoder": [("g2 = g * (a2 > 0)", "g2 = g", 0)],
    "upsampling_adjoint_averages": [("return g.reshape(B, C, H // 2, 2, W // 2, 2).sum(axis=(3, 5))",
                                     "return g.reshape(B, C, H // 2, 2, W // 2, 2).mean(axis=(3, 5))", 0)],
    "bf16_truncates": [("r = ((u + 0x7FFF + lsb) >> 16) << 16", "r = (u >> 16) << 16", 0)],
    "no_residual_input": [("out = xin + np.einsum(", "out = 0.0 * xin + np.einsum(", 0)],
    "loss_gradient_halved": [("g_out = 2.0 * (out - target) / n", "g_out = (out - target) / n", 0)],
}


def load_module(text, name):
    import types
    mod = types.ModuleType(name)
    exec(compile(text, name, "exec"), mod.__dict__)
    return mod


def unet_pins():
    import test_oracle_unet as t
    return [t.test_conv3_is_a_padded_correlation, t.test_zero_final_layer_gives_the_identity,
            t.test_pool_and_upsample_adjoint_pairs, t.test_gradients_match_finite_differences,
            t.test_bf16_rounding_is_nearest_even]


def test_unchanged_network_oracle_passes_its_pins():
    pytest.importorskip("scipy.signal")
    mod = load_module(open(UNET_SRC).read(), "unet_unchanged")
    for pin in unet_pins():
        pin(mod)


@pytest.mark.parametrize("name", list(UNET_MUTATIONS))
def test_planted_network_mistake_fails_a_pin(name):
    pytest.importorskip("scipy.signal")
    source = open(UNET_SRC).read()
    text = source
    for old, new, n in UNET_MUTATIONS[name]:
        text = replace_nth(text, old, new, n)
    assert text != source
    mod = load_module(text, "unet_" + name)
    failed = []
    for pin in unet_pins():
        try:
            pin(mod)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"no pin caught '{name}'"
