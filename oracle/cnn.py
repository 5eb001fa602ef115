"""FP64 oracle of the CNN seed (TEST INFRASTRUCTURE: only tests/, the smoke
check and the bench's CPU leg use it).

The network maps observed velocity and dispersion maps (64 x 64) to the
parameters the optimisers of Sec. 2.3 start from, replacing the heuristic
initial guess of Sec. 2.1.9.  It is defined as:
  input  x[n][64][64][4] = (v / 200, sigma / 100, mask, 0), 0 where masked
  conv   2 x 2 stride 2 -> 32 x 32 x 32,  ReLU
  conv   2 x 2 stride 2 -> 16 x 16 x 64,  ReLU
  conv   2 x 2 stride 2 ->  8 x  8 x 128, ReLU
  conv   2 x 2 stride 2 ->  4 x  4 x 256, ReLU
  dense  flatten f[morton(y, x) * 256 + c] -> 256, ReLU
  dense  256 -> 16 (outputs 0..9 used)
with W_l[o][k], k = (dy * p + dx) * C_in + c for the convolutions, and the
parameter vector holding each layer as [C_l][K_l + 1] (bias last).  The loss
is the mean over samples and the 10 used outputs of (y - t)^2.  Everything
here is FP64 and follows that definition directly (convolutions as sums
over kernel offsets), with the backward pass derived by hand and pinned by
finite differences in the tests.
"""
import math

import numpy as np

MAP = 64
C = (32, 64, 128, 256, 256, 16)
K = (16, 128, 256, 512, 4096, 256)
P_SIZE = (2, 2, 2, 2)       # conv kernel = stride of the four convolutions
NL = len(C)
N_OUT, N_T = 16, 10
V_SCALE, S_SCALE = 200.0, 100.0
GOLDEN = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1


def param_offsets():
    off = [0]
    for c, k in zip(C, K):
        off.append(off[-1] + c * (k + 1))
    return off


def param_count():
    return param_offsets()[-1]


def unpack(P):
    """[(W_l [C_l][K_l], b_l [C_l])] from the parameter vector."""
    off = param_offsets()
    out = []
    for l in range(NL):
        blk = np.asarray(P[off[l]:off[l + 1]], dtype=np.float64).reshape(C[l], K[l] + 1)
        out.append((blk[:, :K[l]], blk[:, K[l]]))
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W, b[:, None]], axis=1).ravel() for W, b in layers])


def morton(y, x, bits):
    """Bit interleave: x bit i -> bit 2i, y bit i -> bit 2i + 1."""
    q = 0
    for i in range(bits):
        q |= ((x >> i) & 1) << (2 * i) | ((y >> i) & 1) << (2 * i + 1)
    return q


def bf16(x):
    """Round to the nearest BF16 value (8 significant bits, ties to even),
    returned in FP64.  For the BF16 form of the network below; the values
    met there are normal numbers of FP32's exponent range, and 0."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)  # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(np.ldexp(m, 8)), e - 8)


def encode(v, s, mask, rounding=None):
    """x [n][64][64][4] from maps [n][64][64] (the fourth channel is zero).
    rounding="bf16": the BF16 input of the low-precision form (the scaled
    values taken in FP32, then rounded to BF16)."""
    m = (np.asarray(mask) != 0).astype(np.float64)
    if rounding == "bf16":
        sv = (np.asarray(v, np.float32) / np.float32(V_SCALE)).astype(np.float64)
        ss = (np.asarray(s, np.float32) / np.float32(S_SCALE)).astype(np.float64)
        return np.stack([bf16(sv) * m, bf16(ss) * m, m, np.zeros_like(m)], axis=-1)
    return np.stack([np.asarray(v, np.float64) / V_SCALE * m, np.asarray(s, np.float64) / S_SCALE * m, m,
                     np.zeros_like(m)], axis=-1)


def conv(x, W, b, p):
    """Stride-p convolution with a p x p kernel: out[n][Y][X][o] = b[o] +
    sum_{dy,dx,c} W[o][(dy p + dx) Cin + c] x[n][p Y + dy][p X + dx][c]."""
    Cout, Cin = W.shape[0], x.shape[-1]
    Wr = W.reshape(Cout, p, p, Cin)
    out = np.zeros((x.shape[0], x.shape[1] // p, x.shape[2] // p, Cout)) + b
    for dy in range(p):
        for dx in range(p):
            out += np.einsum("nyxc,oc->nyxo", x[:, dy::p, dx::p, :], Wr[:, dy, dx, :])
    return out


def conv_backward(x, W, dz, p):
    """Gradients of conv() with respect to W, b and x."""
    Cout, Cin = W.shape[0], x.shape[-1]
    Wr = W.reshape(Cout, p, p, Cin)
    dW = np.zeros_like(Wr)
    dx_ = np.zeros_like(x)
    for dy in range(p):
        for dx in range(p):
            xs = x[:, dy::p, dx::p, :]
            dW[:, dy, dx, :] = np.einsum("nyxo,nyxc->oc", dz, xs)
            dx_[:, dy::p, dx::p, :] = np.einsum("nyxo,oc->nyxc", dz, Wr[:, dy, dx, :])
    return dW.reshape(Cout, -1), dz.sum(axis=(0, 1, 2)), dx_


FLAT = np.array([[morton(y, x, 2) for x in range(4)] for y in range(4)])  # 4 x 4 -> flatten slot


def flatten(h3):
    n = h3.shape[0]
    f = np.zeros((n, 16, 256))
    for y in range(4):
        for x in range(4):
            f[:, FLAT[y, x], :] = h3[:, y, x, :]
    return f.reshape(n, 4096)


def unflatten(f):
    n = f.shape[0]
    f = f.reshape(n, 16, 256)
    h = np.zeros((n, 4, 4, 256))
    for y in range(4):
        for x in range(4):
            h[:, y, x, :] = f[:, FLAT[y, x], :]
    return h


def _rounder(rounding):
    if rounding is None:
        return lambda a: a
    if rounding == "bf16":
        return bf16
    raise ValueError("rounding must be None or 'bf16'")


def forward(P, x, rounding=None):
    """Outputs [n][16] and the activations needed by backward().

    rounding=None: the network in FP64.  rounding="bf16": its low-precision
    form, the values the products read rounded to BF16 -- the weights (the
    biases stay as given), and each hidden layer's output after the ReLU --
    with every sum still exact in FP64; x is then expected from
    encode(..., rounding="bf16")."""
    q = _rounder(rounding)
    L = [(q(W), b) for W, b in unpack(P)]
    hs = [x]
    for l in range(4):
        hs.append(q(np.maximum(conv(hs[-1], *L[l], P_SIZE[l]), 0.0)))
    f = flatten(hs[-1])
    h5 = q(np.maximum(f @ L[4][0].T + L[4][1], 0.0))
    y = h5 @ L[5][0].T + L[5][1]
    return y, (hs, f, h5)


def loss_and_grad(P, x, t, rounding=None):
    """Mean squared error over the 10 used outputs and its gradient.
    rounding="bf16" (see forward): also the output gradient dL/dy and each
    back-propagated gradient (after its ReLU mask) are rounded to BF16
    before the products that read them; the parameter gradients are exact
    sums of those products."""
    q = _rounder(rounding)
    L = [(q(W), b) for W, b in unpack(P)]
    y, (hs, f, h5) = forward(P, x, rounding)
    n = x.shape[0]
    d = np.zeros_like(y)
    d[:, :N_T] = y[:, :N_T] - t
    loss = float(np.sum(d * d) / (n * N_T))
    dy = q(2.0 * d / (n * N_T))
    g6 = (dy.T @ h5, dy.sum(0))
    dz5 = q((dy @ L[5][0]) * (h5 > 0))
    g5 = (dz5.T @ f, dz5.sum(0))
    dz = q(unflatten(dz5 @ L[4][0]) * (hs[4] > 0))
    grads = []
    for l in range(3, -1, -1):
        W, b, dh = conv_backward(hs[l], L[l][0], dz, P_SIZE[l])
        grads.insert(0, (W, b))
        if l > 0:
            dz = q(dh * (hs[l] > 0))
    return loss, pack(grads + [g5, g6])


def targets(params):
    p = np.asarray(params, np.float64).reshape(-1, 10)
    pa = np.radians(p[:, 2])
    return np.stack([(p[:, 0] - 31.5) / 8.0, (p[:, 1] - 31.5) / 8.0, np.cos(pa), np.sin(pa),
                     (p[:, 3] - 50.0) / 20.0, p[:, 4] / 30.0, (p[:, 5] - 175.0) / 75.0, (p[:, 6] - 4.5) / 2.5,
                     (p[:, 7] - 45.0) / 25.0, (p[:, 9] - 7.0) / 3.0], axis=1)


def decode(y):
    y = np.asarray(y, np.float64)
    pa = np.degrees(np.arctan2(y[:, 3], y[:, 2])) % 360.0
    return np.stack([31.5 + 8.0 * y[:, 0], 31.5 + 8.0 * y[:, 1], pa, 50.0 + 20.0 * y[:, 4], 30.0 * y[:, 5],
                     175.0 + 75.0 * y[:, 6], 4.5 + 2.5 * y[:, 7], 45.0 + 25.0 * y[:, 8], np.ones(len(y)),
                     7.0 + 3.0 * y[:, 9]], axis=1)


def adam(P, m, v, g, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    P = P - lr * (m / (1 - b1 ** step)) / (np.sqrt(v / (1 - b2 ** step)) + eps)
    return P, m, v


# ---------------------------------------------------------------------------
# Counter-based access to SplitMix64 (Steele, Lea & Flood 2014): output k of
# the stream seeded with s is mix(s + k * golden).
def sm_mix(z):
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def sm_output(seed, k):
    return sm_mix(seed + k * GOLDEN)


def sm_normal(seed, j):
    """Normal number j: Box-Muller (cosine branch) of outputs 2j+1, 2j+2."""
    u1 = ((sm_output(seed, 2 * j + 1) >> 11) + 1) * (1.0 / 9007199254740992.0)
    u2 = (sm_output(seed, 2 * j + 2) >> 11) * (1.0 / 9007199254740992.0)
    return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


def sm_uniform(seed, i):
    return (sm_output(seed, i + 1) >> 11) * (1.0 / 9007199254740992.0)


def init(seed):
    """He-normal weights (std sqrt(2 / K), last layer sqrt(1 / K)), zero biases;
    parameter i uses normal number i of the stream."""
    off = param_offsets()
    P = np.zeros(off[-1])
    for l in range(NL):
        sd = math.sqrt((1.0 if l == NL - 1 else 2.0) / K[l])
        for j in range(C[l] * (K[l] + 1)):
            if j % (K[l] + 1) != K[l]:
                P[off[l] + j] = sd * sm_normal(seed, off[l] + j)
    return P


def synth_obs(maps, seed, noise_v, dead_frac, pixels=None):
    """Observed (v, sigma, mask) from model maps [n][3][64][64]; `pixels`
    restricts the work to a list of flat indices (returns those only)."""
    maps = np.asarray(maps, np.float64)
    n = maps.shape[0]
    npix = MAP * MAP
    flat = range(n * npix) if pixels is None else pixels
    out = []
    for i in flat:
        i = int(i)
        b, pix = divmod(i, npix)
        m0, m1, m2 = maps[b, 0].ravel()[pix], maps[b, 1].ravel()[pix], maps[b, 2].ravel()[pix]
        v = m1 + noise_v * sm_normal(seed, 2 * i)
        s = m2 + math.sqrt(2.0) * noise_v * sm_normal(seed, 2 * i + 1)
        dead = sm_uniform(seed ^ 0xD1B54A32D192ED03, i) < dead_frac
        out.append((v, s, 0 if (dead or not m0 > 0) else 1))
    return out
