"""Plant plausible mistakes in copies of the CNN oracle (oracle/cnn.py) and
check that the pins catch every one (the pins run fastest first and a
mutant counts as caught at the first that fails).

Each mutant is a one-expression edit of the module's source: an index or
axis swapped, a term or factor dropped, a wrong constant or branch."""
import importlib.util
import os

import pytest

from oracle import cnn
from cnn_pins import ALL_CNN_PINS

SRC = cnn.__file__

MUTANTS = [
    ("morton_axes_swapped", "q |= ((x >> i) & 1) << (2 * i) | ((y >> i) & 1) << (2 * i + 1)",
     "q |= ((y >> i) & 1) << (2 * i) | ((x >> i) & 1) << (2 * i + 1)"),
    ("flatten_transposed", "f[:, FLAT[y, x], :] = h3[:, y, x, :]", "f[:, FLAT[x, y], :] = h3[:, y, x, :]"),
    ("encode_mask_not_applied", "np.asarray(v, np.float64) / V_SCALE * m", "np.asarray(v, np.float64) / V_SCALE"),
    ("encode_scales_swapped", "V_SCALE, S_SCALE = 200.0, 100.0", "V_SCALE, S_SCALE = 100.0, 200.0"),
    ("conv_channel_major_kernel", "    Wr = W.reshape(Cout, p, p, Cin)\n    out",
     "    Wr = W.reshape(Cout, Cin, p, p).transpose(0, 2, 3, 1)\n    out"),
    ("conv_offsets_swapped", "out += np.einsum(\"nyxc,oc->nyxo\", x[:, dy::p, dx::p, :], Wr[:, dy, dx, :])",
     "out += np.einsum(\"nyxc,oc->nyxo\", x[:, dx::p, dy::p, :], Wr[:, dy, dx, :])"),
    ("conv_bias_dropped", "out = np.zeros((x.shape[0], x.shape[1] // p, x.shape[2] // p, Cout)) + b",
     "out = np.zeros((x.shape[0], x.shape[1] // p, x.shape[2] // p, Cout))"),
    ("loss_mean_over_samples_only", "loss = float(np.sum(d * d) / (n * N_T))", "loss = float(np.sum(d * d) / n)"),
    ("gradient_factor_two_dropped", "dy = q(2.0 * d / (n * N_T))", "dy = q(d / (n * N_T))"),
    ("dense_relu_mask_dropped", "dz5 = q((dy @ L[5][0]) * (h5 > 0))", "dz5 = q(dy @ L[5][0])"),
    ("conv_relu_mask_dropped", "dz = q(dh * (hs[l] > 0))", "dz = q(dh)"),
    ("bias_gradient_halved", "return dW.reshape(Cout, -1), dz.sum(axis=(0, 1, 2)), dx_",
     "return dW.reshape(Cout, -1), 0.5 * dz.sum(axis=(0, 1, 2)), dx_"),
    ("input_gradient_offsets_swapped", "dx_[:, dy::p, dx::p, :] = np.einsum(\"nyxo,oc->nyxc\", dz, Wr[:, dy, dx, :])",
     "dx_[:, dx::p, dy::p, :] = np.einsum(\"nyxo,oc->nyxc\", dz, Wr[:, dy, dx, :])"),
    ("targets_cos_sin_swapped", "np.cos(pa), np.sin(pa)", "np.sin(pa), np.cos(pa)"),
    ("adam_bias_correction_dropped", "P = P - lr * (m / (1 - b1 ** step)) / (np.sqrt(v / (1 - b2 ** step)) + eps)",
     "P = P - lr * m / (np.sqrt(v / (1 - b2 ** step)) + eps)"),
    ("adam_eps_inside_sqrt", "(np.sqrt(v / (1 - b2 ** step)) + eps)", "np.sqrt(v / (1 - b2 ** step) + eps)"),
    ("splitmix_first_shift", "z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64",
     "z = ((z ^ (z >> 31)) * 0xBF58476D1CE4E5B9) & M64"),
    ("box_muller_sine_branch", "return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)",
     "return math.sqrt(-2.0 * math.log(u1)) * math.sin(2.0 * math.pi * u2)"),
    ("synth_same_normal_for_v_and_s", "s = m2 + math.sqrt(2.0) * noise_v * sm_normal(seed, 2 * i + 1)",
     "s = m2 + math.sqrt(2.0) * noise_v * sm_normal(seed, 2 * i)"),
    ("synth_sigma_noise_not_scaled", "s = m2 + math.sqrt(2.0) * noise_v * sm_normal(seed, 2 * i + 1)",
     "s = m2 + noise_v * sm_normal(seed, 2 * i + 1)"),
    ("synth_dead_test_inverted", "dead = sm_uniform(seed ^ 0xD1B54A32D192ED03, i) < dead_frac",
     "dead = sm_uniform(seed ^ 0xD1B54A32D192ED03, i) > dead_frac"),
    ("bf16_seven_bits", "return np.ldexp(np.rint(np.ldexp(m, 8)), e - 8)", "return np.ldexp(np.rint(np.ldexp(m, 7)), e - 7)"),
    ("bf16_truncates", "return np.ldexp(np.rint(np.ldexp(m, 8)), e - 8)", "return np.ldexp(np.trunc(np.ldexp(m, 8)), e - 8)"),
    ("bf16_encode_unrounded", "return np.stack([bf16(sv) * m, bf16(ss) * m, m, np.zeros_like(m)], axis=-1)",
     "return np.stack([sv * m, ss * m, m, np.zeros_like(m)], axis=-1)"),
    ("bf16_activations_before_relu", "hs.append(q(np.maximum(conv(hs[-1], *L[l], P_SIZE[l]), 0.0)))",
     "hs.append(np.maximum(q(conv(hs[-1], *L[l], P_SIZE[l])) - 1e-3, 0.0))"),
    ("init_std_halved", "sd = math.sqrt((1.0 if l == NL - 1 else 2.0) / K[l])",
     "sd = math.sqrt((1.0 if l == NL - 1 else 1.0) / K[l])"),
]


def _load(name, old, new, tmp_path):
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    path = os.path.join(str(tmp_path), "cnn_%s.py" % name)
    with open(path, "w") as f:
        f.write(src.replace(old, new, 1))
    spec = importlib.util.spec_from_file_location("cnn_" + name, path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_the_mutant(name, old, new, tmp_path):
    mod = _load(name, old, new, tmp_path)
    for pin in ALL_CNN_PINS:
        try:
            pin(mod)
        except (AssertionError, ValueError, IndexError, FloatingPointError):
            return
    pytest.fail("no pin catches the mutant %s" % name)
