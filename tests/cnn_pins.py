"""Pins of the CNN oracle (oracle/cnn.py) as functions of the module under
test, so that the same pins check the oracle and the mistakes planted in
copies of it.  They test it against things it does not compute itself:
direct convolution loops, finite differences of its own loss, the bit
structure of the Morton order, PyTorch's BF16 conversion, the sequential SplitMix64 generator (in
oracle/fit.py), the He-normal statistics of its initial weights, and closed
forms of the target map and of Adam's first step."""
import math

import numpy as np
import pytest

from oracle import fit


def pin_conv_equals_direct_loops(cnn):
    rng = np.random.default_rng(1)
    for p, H, cin, cout in ((4, 8, 3, 5), (2, 6, 4, 3)):
        x = rng.normal(size=(2, H, H, cin))
        W = rng.normal(size=(cout, p * p * cin))
        b = rng.normal(size=cout)
        got = cnn.conv(x, W, b, p)
        ref = np.zeros_like(got)
        for n in range(2):
            for Y in range(H // p):
                for X in range(H // p):
                    for o in range(cout):
                        acc = b[o]
                        for dy in range(p):
                            for dx in range(p):
                                for c in range(cin):
                                    acc += W[o, (dy * p + dx) * cin + c] * x[n, p * Y + dy, p * X + dx, c]
                        ref[n, Y, X, o] = acc
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def pin_morton_structure(cnn):
    q = np.array([[cnn.morton(y, x, 5) for x in range(32)] for y in range(32)])
    assert sorted(q.ravel().tolist()) == list(range(1024))           # a bijection
    for y in range(32):
        for x in range(32):
            # the 2 x 2 block of (y, x) is the run q >> 2, its position in the block q & 3
            assert q[y, x] >> 2 == cnn.morton(y >> 1, x >> 1, 4)
            assert q[y, x] & 3 == (y & 1) * 2 + (x & 1)
    f = np.random.default_rng(2).normal(size=(3, 4, 4, 256))
    np.testing.assert_array_equal(cnn.unflatten(cnn.flatten(f)), f)


def _small_problem(cnn, seed=3, n=2):
    rng = np.random.default_rng(seed)
    P = np.zeros(cnn.param_count())
    off = cnn.param_offsets()
    for l in range(cnn.NL):
        blk = rng.normal(size=(cnn.C[l], cnn.K[l] + 1)) * math.sqrt(2.0 / cnn.K[l])
        blk[:, -1] = rng.normal(size=cnn.C[l]) * 0.1
        P[off[l]:off[l + 1]] = blk.ravel()
    v = rng.normal(0, 100, size=(n, 64, 64))
    s = rng.uniform(20, 80, size=(n, 64, 64))
    mask = (rng.uniform(size=(n, 64, 64)) > 0.1).astype(np.uint8)
    t = rng.normal(size=(n, 10))
    return P, cnn.encode(v, s, mask), t


def pin_gradient_matches_finite_differences(cnn):
    P, x, t = _small_problem(cnn)
    loss, g = cnn.loss_and_grad(P, x, t)
    off = cnn.param_offsets()
    rng = np.random.default_rng(4)
    checked = 0
    for l in range(cnn.NL):
        idx = list(rng.choice(np.arange(off[l], off[l + 1]), size=8, replace=False))
        idx.append(off[l] + cnn.K[l])  # a bias
        for i in idx:
            # central differences; a step that crosses a ReLU kink shows as a
            # step-dependent error, so a miss is re-measured with a smaller step
            ok = False
            for h in (1e-6, 1e-7):
                Pp, Pm = P.copy(), P.copy()
                Pp[i] += h
                Pm[i] -= h
                fd = (cnn.loss_and_grad(Pp, x, t)[0] - cnn.loss_and_grad(Pm, x, t)[0]) / (2 * h)
                scale = max(abs(fd), abs(g[i]), 1e-8)
                if abs(fd - g[i]) <= 1e-5 * scale + 1e-9:
                    ok = True
                    break
            assert ok, (l, i, fd, g[i])
            checked += 1
    assert checked == 9 * cnn.NL


def pin_loss_definition(cnn):
    P, x, t = _small_problem(cnn, n=3)
    y, _ = cnn.forward(P, x)
    loss, _ = cnn.loss_and_grad(P, x, t)
    assert loss == pytest.approx(float(np.mean((y[:, :10] - t) ** 2)), rel=1e-12)


def pin_encode_masks_and_scales(cnn):
    v = np.full((1, 64, 64), 100.0)
    s = np.full((1, 64, 64), 50.0)
    m = np.ones((1, 64, 64), np.uint8)
    m[0, 3, 5] = 0
    x = cnn.encode(v, s, m)
    assert x[0, 0, 0].tolist() == [0.5, 0.5, 1.0, 0.0]
    assert x[0, 3, 5].tolist() == [0.0, 0.0, 0.0, 0.0]


def pin_targets_decode_round_trip(cnn):
    rng = np.random.default_rng(5)
    p = np.stack([rng.uniform(25, 38, 50), rng.uniform(25, 38, 50), rng.uniform(0, 360, 50), rng.uniform(20, 80, 50),
                  rng.uniform(-30, 30, 50), rng.uniform(50, 300, 50), rng.uniform(1, 8, 50), rng.uniform(10, 80, 50),
                  np.ones(50), rng.uniform(4, 10, 50)], axis=1)
    t = cnn.targets(p)
    y = np.zeros((50, 16))
    y[:, :10] = t
    q = cnn.decode(y)
    np.testing.assert_allclose(q, p, rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(t[:, 2] ** 2 + t[:, 3] ** 2, 1.0, rtol=1e-12)


def pin_counter_splitmix_equals_sequential(cnn):
    for seed in (0, 12345, (1 << 63) + 7):
        r = fit.SplitMix64(seed)
        seq = [r.next() for _ in range(12)]
        assert [cnn.sm_output(seed, k) for k in range(1, 13)] == seq
        # normal j = Box-Muller (cosine) of outputs 2j+1, 2j+2 (u1 shifted into (0, 1])
        for j in range(5):
            u1 = ((seq[2 * j] >> 11) + 1) / 9007199254740992.0
            u2 = (seq[2 * j + 1] >> 11) / 9007199254740992.0
            assert cnn.sm_normal(seed, j) == pytest.approx(math.sqrt(-2 * math.log(u1)) * math.cos(2 * math.pi * u2),
                                                           rel=1e-15)


def pin_normal_stream_statistics(cnn):
    z = np.array([cnn.sm_normal(99, j) for j in range(20000)])
    assert abs(z.mean()) < 4 / math.sqrt(20000)
    assert abs(z.std() - 1.0) < 0.02


def pin_adam_first_step(cnn):
    g = np.array([1e-3, -2.0, 5e-2, 0.0])
    P = np.zeros(4)
    P1, m, v = cnn.adam(P, np.zeros(4), np.zeros(4), g, 1, 1e-2)
    # bias-corrected first step: -lr g / (|g| + eps)
    np.testing.assert_allclose(P1, -1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def pin_init_statistics(cnn):
    """He-normal weights: standard deviation sqrt(2 / K) (sqrt(1 / K) for the
    last layer) within sampling error, biases zero."""
    P = cnn.init(7)
    off = cnn.param_offsets()
    for l in range(cnn.NL):
        blk = P[off[l]:off[l + 1]].reshape(cnn.C[l], cnn.K[l] + 1)
        w, b = blk[:, :-1].ravel(), blk[:, -1]
        sd = math.sqrt((1.0 if l == cnn.NL - 1 else 2.0) / cnn.K[l])
        assert np.all(b == 0.0)
        assert abs(w.std() / sd - 1.0) < 6.0 / math.sqrt(2.0 * w.size), (l, w.std(), sd)
        assert abs(w.mean()) < 6.0 * sd / math.sqrt(w.size)


def pin_synthetic_observations(cnn):
    """synth_obs on one 64 x 64 map: with no noise and no dead fibres it
    returns the model maps (masked where m0 = 0); with every fibre dead it
    masks everything; with noise, (v - m1) / noise and (s - m2) / (sqrt 2
    noise) are standard normal and uncorrelated (distinct numbers of the
    stream), and the dead fraction is the one asked for."""
    rng = np.random.default_rng(8)
    maps = np.stack([rng.uniform(0.0, 1.0, (64, 64)), rng.normal(0, 100, (64, 64)),
                     rng.uniform(10, 80, (64, 64))])[None]
    maps[0, 0, :3, :] = 0.0  # three rows without light
    out = np.array(cnn.synth_obs(maps, 5, 0.0, 0.0))
    np.testing.assert_array_equal(out[:, 0], maps[0, 1].ravel())
    np.testing.assert_array_equal(out[:, 1], maps[0, 2].ravel())
    np.testing.assert_array_equal(out[:, 2], (maps[0, 0].ravel() > 0).astype(float))
    assert np.all(np.array(cnn.synth_obs(maps, 5, 0.0, 1.0))[:, 2] == 0)
    out = np.array(cnn.synth_obs(maps, 5, 5.0, 0.02))
    zv = (out[:, 0] - maps[0, 1].ravel()) / 5.0
    zs = (out[:, 1] - maps[0, 2].ravel()) / (5.0 * math.sqrt(2.0))
    n = zv.size
    for z in (zv, zs):
        assert abs(z.mean()) < 5.0 / math.sqrt(n) and abs(z.std() - 1.0) < 0.05
    assert abs(np.corrcoef(zv, zs)[0, 1]) < 5.0 / math.sqrt(n)
    lit = maps[0, 0].ravel() > 0
    dead = np.mean(out[lit, 2] == 0)
    assert abs(dead - 0.02) < 5.0 * math.sqrt(0.02 * 0.98 / lit.sum()), dead


def pin_bf16_rounding_matches_the_library(cnn):
    """bf16() is round-to-nearest-even to 8 significant bits: on FP32 values
    (random, and exact ties, halfway between two BF16 neighbours) it equals
    PyTorch's float32 -> bfloat16 conversion."""
    import torch
    rng = np.random.default_rng(21)
    x = (rng.normal(size=4000) * 10.0 ** rng.uniform(-6, 6, size=4000)).astype(np.float32)
    bits = x.view(np.uint32)
    ties = ((bits & np.uint32(0xFFFF0000)) | np.uint32(0x8000)).view(np.float32)  # halfway cases
    for v in (x, ties, np.array([0.0, -0.0, 1.0, -3.0, 2.0 ** -120], np.float32)):
        ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
        np.testing.assert_array_equal(cnn.bf16(v.astype(np.float64)), ref)


def pin_bf16_form_rounds_where_stated(cnn):
    """The BF16 form reads BF16 values only: its encoded input, every hidden
    activation and the flattened features are BF16 numbers (bf16(h) == h) and
    non-negative after the ReLU; it stays within BF16 rounding (relative
    2^-9 per value, compounded over six layers) of the FP64 network; and
    with no rounding it is the FP64 network itself."""
    rng = np.random.default_rng(22)
    n = 2
    P = np.zeros(cnn.param_count())
    off = cnn.param_offsets()
    for l in range(cnn.NL):
        blk = rng.normal(size=(cnn.C[l], cnn.K[l] + 1)) * math.sqrt(2.0 / cnn.K[l])
        blk[:, -1] = 0.05 * rng.normal(size=cnn.C[l])
        P[off[l]:off[l + 1]] = blk.ravel()
    v = rng.normal(0, 100, size=(n, 64, 64)).astype(np.float32)
    s = rng.uniform(20, 80, size=(n, 64, 64)).astype(np.float32)
    m = (rng.uniform(size=(n, 64, 64)) > 0.1).astype(np.uint8)
    xb = cnn.encode(v, s, m, rounding="bf16")
    np.testing.assert_array_equal(cnn.bf16(xb), xb)
    assert np.all(xb[..., 2] == (m != 0)) and np.all(xb[..., 3] == 0) and np.all(xb[m == 0] == 0)
    yb, (hs, f, h5) = cnn.forward(P, xb, rounding="bf16")
    for h in hs[1:] + [f, h5]:
        np.testing.assert_array_equal(cnn.bf16(h), h)
        assert h.min() >= 0.0
    x = cnn.encode(v, s, m)
    y, _ = cnn.forward(P, x)
    assert np.linalg.norm(yb - y) <= 2e-2 * np.linalg.norm(y), np.linalg.norm(yb - y) / np.linalg.norm(y)
    np.testing.assert_array_equal(cnn.forward(P, x, rounding=None)[0], y)


# fastest first: a mutant test stops at the first pin that fails
ALL_CNN_PINS = [pin_morton_structure, pin_encode_masks_and_scales, pin_bf16_rounding_matches_the_library,
                pin_conv_equals_direct_loops, pin_bf16_form_rounds_where_stated,
                pin_targets_decode_round_trip, pin_adam_first_step, pin_counter_splitmix_equals_sequential,
                pin_normal_stream_statistics, pin_synthetic_observations, pin_init_statistics, pin_loss_definition,
                pin_gradient_matches_finite_differences]
