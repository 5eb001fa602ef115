"""Pins of the FP64 oracle against facts the paper and mathematics fix.

Each pin is a function of the oracle module; it raises AssertionError when the
oracle disagrees.  ``test_oracle_pins.py`` runs them against the oracle, and
``test_oracle_mutants.py`` runs them against deliberately broken copies of the
oracle to show that a plausible mistake anywhere in it fails at least one pin.

None of the pins re-types the oracle's formulas for a generic input: they use
closed forms of special cases (face-on disc, the major and minor axes, a line
far from the band edges), invariants (rotations, reflections, flux
conservation), brute force on tiny inputs, and hand-checked numbers.
"""
import math

import numpy as np

PAR = dict(x0=0, y0=1, pa=2, incl=3, vsys=4, vmax=5, rt=6, sig0=7, i0=8, h=9)
# A Gaussian's FWHM is 2 sqrt(2 ln 2) sigma.
FWHM_PER_SIGMA = math.sqrt(8.0 * math.log(2.0))


def P(x0=10.3, y0=9.7, pa=30.0, incl=50.0, vsys=12.0, vmax=180.0, rt=2.5,
      sig0=30.0, i0=1.0, h=3.0):
    return np.array([x0, y0, pa, incl, vsys, vmax, rt, sig0, i0, h], dtype=np.float64)


def _grid(n=9, span=6.0, c=(10.3, 9.7)):
    s = np.linspace(-span, span, n)
    return np.meshgrid(c[0] + s, c[1] + s)


# --------------------------------------------------------------------------
# Geometry and kinematics (Sec. 2.1, Eqs. 1-8)

def pin_los_face_on(og):
    """i = 0: the disc has no line-of-sight rotation; v = Vsys everywhere and
    the brightness is circularly symmetric: I = I0 exp(-d/h) with d the sky
    distance."""
    p = P(incl=0.0)
    x, y = _grid()
    v, b = og.los(p, x, y)
    np.testing.assert_allclose(v, 12.0, rtol=0, atol=1e-12)
    d = np.hypot(x - p[0], y - p[1])
    np.testing.assert_allclose(b, np.exp(-d / 3.0), rtol=1e-13)


def pin_los_pa_flip(og):
    """PA -> PA + 180 deg reverses the projected rotation: v - Vsys flips."""
    x, y = _grid()
    v1, b1 = og.los(P(pa=30.0), x, y)
    v2, b2 = og.los(P(pa=210.0), x, y)
    np.testing.assert_allclose(v2 - 12.0, -(v1 - 12.0), rtol=0, atol=1e-9)
    np.testing.assert_allclose(b2, b1, rtol=1e-12)


def pin_los_major_axis(og):
    """Along the projected major axis (y_e = 0) the field is the rotation
    curve of Eq. 6 times sin i.  With PA = 0 the major axis is the line
    x = x0 (points (x0, y0+s)); with PA = 90 deg it is y = y0 and points
    (x0+s, y0) have x_e = -s."""
    s = np.array([-7.0, -3.0, -0.5, 0.25, 1.0, 4.0, 9.0])
    vmax, rt, incl = 180.0, 2.5, math.radians(50.0)
    curve = (2.0 / np.pi) * vmax * np.arctan(np.abs(s) / rt) * np.sin(incl)
    v, b = og.los(P(pa=0.0), 10.3 + 0 * s, 9.7 + s)
    np.testing.assert_allclose(v - 12.0, np.sign(s) * curve, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(b, np.exp(-np.abs(s) / 3.0), rtol=1e-12)
    v, b = og.los(P(pa=90.0), 10.3 + s, 9.7 + 0 * s)
    np.testing.assert_allclose(v - 12.0, -np.sign(s) * curve, rtol=1e-12, atol=1e-9)


def pin_los_minor_axis(og):
    """Along the projected minor axis (x_e = 0) there is no line-of-sight
    rotation, and the deprojected radius is |s| / cos i (Eq. 3)."""
    s = np.array([-6.0, -2.0, -0.3, 0.7, 3.0, 8.0])
    v, b = og.los(P(pa=0.0), 10.3 + s, 9.7 + 0 * s)
    np.testing.assert_allclose(v, 12.0, rtol=0, atol=1e-12)
    r = np.abs(s) / math.cos(math.radians(50.0))
    np.testing.assert_allclose(b, np.exp(-r / 3.0), rtol=1e-12)


def pin_los_centre(og):
    """At the centre (r = 0) v = Vsys and I = I0."""
    v, b = og.los(P(i0=2.5), np.array([10.3]), np.array([9.7]))
    assert abs(v[0] - 12.0) < 1e-12 and abs(b[0] - 2.5) < 1e-12


def pin_los_rotation_equivariance(og):
    """Rotating a sky point about the centre by alpha and adding alpha to PA
    leaves x_e and y_e, hence v and I, unchanged (Eqs. 1-2 are a rotation)."""
    x, y = _grid(7, 5.0)
    p = P(pa=20.0)
    v0, b0 = og.los(p, x, y)
    for alpha in (37.0, 90.0, 145.0, 300.0):
        a = math.radians(alpha)
        dx, dy = x - p[0], y - p[1]
        xr = p[0] + dx * math.cos(a) - dy * math.sin(a)
        yr = p[1] + dx * math.sin(a) + dy * math.cos(a)
        v1, b1 = og.los(P(pa=20.0 + alpha), xr, yr)
        np.testing.assert_allclose(v1, v0, rtol=0, atol=1e-9)
        np.testing.assert_allclose(b1, b0, rtol=1e-10)


def pin_los_worked_example(og):
    """Hand-worked point.  x0 = y0 = 0, PA = 90 deg, i = 60 deg, Vsys = 10,
    Vmax = 100, rt = 2, I0 = 2, h = 4, at (x, y) = (-1, 2*sqrt(3)):
      x_e = -x sin PA + y cos PA = 1
      y_e = -x cos PA - y sin PA = -2 sqrt(3);  y_e / cos i = -4 sqrt(3)
      r = sqrt(1 + 48) = 7;  cos(theta) = 1/7
      Vrot(7) = (200/pi) atan(3.5);  v = 10 + Vrot(7) (sqrt(3)/2) / 7
      I = 2 exp(-7/4)."""
    p = np.array([0.0, 0.0, 90.0, 60.0, 10.0, 100.0, 2.0, 30.0, 2.0, 4.0])
    v, b = og.los(p, np.array([-1.0]), np.array([2.0 * math.sqrt(3.0)]))
    vrot7 = (200.0 / math.pi) * math.atan(3.5)
    assert abs(v[0] - (10.0 + vrot7 * (math.sqrt(3.0) / 2.0) / 7.0)) < 1e-9, v
    assert abs(b[0] - 2.0 * math.exp(-1.75)) < 1e-12, b


# --------------------------------------------------------------------------
# Kernel taps (Eq. 9 sampled per axis)

def pin_taps(og):
    """R = ceil(4 sigma); taps sum to one, are symmetric and follow the
    Gaussian ratio w_j / w_0 = exp(-j^2 / (2 sigma^2))."""
    for sigma, R in ((1.0616, 5), (0.637, 3), (1.274, 6), (0.25, 1), (2.0, 8)):
        assert og.radius(sigma, 4.0) == R, (sigma, og.radius(sigma, 4.0))
        w = og.taps(sigma, R)
        assert abs(w.sum() - 1.0) < 1e-14
        np.testing.assert_allclose(w, w[::-1], rtol=1e-15)
        j = np.arange(-R, R + 1)
        np.testing.assert_allclose(w / w[R], np.exp(-j * j / (2 * sigma * sigma)), rtol=1e-12)
    assert og.radius(0.0, 4.0) == 0
    np.testing.assert_array_equal(og.taps(0.0, 0), [1.0])


# --------------------------------------------------------------------------
# Convolution (Sec. 2.2.3, valid linear convolution with the product kernel)

def pin_conv_delta(og):
    """A unit voxel at the centre of the extended cube produces the product
    kernel wz (x) wy (x) wx, centred on the corresponding output voxel."""
    wx, wy, wz = og.taps(1.1, 4), og.taps(0.8, 3), og.taps(0.6, 2)
    ext = np.zeros((2 * 2 + 9, 2 * 3 + 11, 2 * 4 + 13))
    ext[2 + 4, 3 + 5, 4 + 6] = 1.0
    out = og.conv3d(ext, wx, wy, wz)
    exp = np.zeros((9, 11, 13))
    exp[4 - 2:4 + 3, 5 - 3:5 + 4, 6 - 4:6 + 5] = wz[:, None, None] * wy[None, :, None] * wx[None, None, :]
    np.testing.assert_allclose(out, exp, rtol=0, atol=1e-15)


def pin_conv_alignment(og):
    """With a one-hot kernel the valid convolution is a pure shift: a tap at
    offset +a along x reads ext[..., i + R + a]."""
    rng = np.random.default_rng(11)
    ext = rng.uniform(size=(5, 6, 12))
    wx = np.zeros(7); wx[3 + 2] = 1.0
    out = og.conv3d(ext, wx, np.ones(1), np.ones(1))
    np.testing.assert_array_equal(out, ext[:, :, 3 + 2:3 + 2 + 6])


def pin_conv_flux(og):
    """Flux conservation: with a zero border at least 2R wide, the valid
    output holds the full linear convolution, whose sum equals the input's
    (unit-sum taps)."""
    rng = np.random.default_rng(12)
    wx, wz = og.taps(1.3, 6), og.taps(0.9, 4)
    inner = rng.uniform(size=(6, 7, 8))
    ext = np.zeros((6 + 16, 7 + 24, 8 + 24))
    ext[8:14, 12:19, 12:20] = inner
    out = og.conv3d(ext, wx, wx, wz)
    assert abs(out.sum() - inner.sum()) < 1e-12 * inner.sum()


def pin_conv_separable(og):
    """Brute force: three 1-D passes equal the direct 3-D sum (distinct
    kernels on the three axes)."""
    rng = np.random.default_rng(13)
    ext = rng.normal(size=(11, 10, 9))
    wx, wy, wz = og.taps(0.9, 3), og.taps(0.7, 2), og.taps(1.2, 4)
    a = og.conv3d(ext, wx, wy, wz)
    b = og.conv3d(ext, wx, wy, wz, separable=True)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-14)


# --------------------------------------------------------------------------
# Moments (Sec. 2.2.5) and down-sampling (Sec. 2.2.4)

def pin_moments_closed_forms(og):
    """Constant spectrum: mean = band centre, std = dv sqrt((n^2-1)/12).
    Two channels with weights a, b at v1, v2: mean (a v1 + b v2)/(a+b),
    std |v2 - v1| sqrt(a b)/(a + b)."""
    nz, dv, vc = 40, 12.5, 30.0
    m = og.moments(np.full((nz, 2, 3), 0.7), dv, vc)
    np.testing.assert_allclose(m[0], 0.7 * nz, rtol=1e-14)
    np.testing.assert_allclose(m[1], vc, rtol=0, atol=1e-12)
    np.testing.assert_allclose(m[2], dv * math.sqrt((nz * nz - 1) / 12.0), rtol=1e-13)
    cube = np.zeros((nz, 1, 1))
    cube[5, 0, 0], cube[17, 0, 0] = 2.0, 3.0
    v5, v17 = vc + (5 - 19.5) * dv, vc + (17 - 19.5) * dv
    m = og.moments(cube, dv, vc)
    assert abs(m[1, 0, 0] - (2 * v5 + 3 * v17) / 5.0) < 1e-12
    assert abs(m[2, 0, 0] - abs(v17 - v5) * math.sqrt(6.0) / 5.0) < 1e-12


def pin_moments_invalid(og):
    """A spectrum whose total is at most 1e-20 of the scale is invalid:
    (0, fallback velocity, 0)."""
    cube = np.zeros((10, 1, 2))
    cube[3, 0, 1] = 1.0
    cube[4, 0, 0] = 5e-21
    m = og.moments(cube, 10.0, 0.0, scale=1.0, v_invalid=-7.0)
    assert m[0, 0, 0] == 0.0 and m[1, 0, 0] == -7.0 and m[2, 0, 0] == 0.0
    assert m[0, 0, 1] == 1.0 and abs(m[1, 0, 1] - (3 - 4.5) * 10.0) < 1e-12


def pin_downsample(og):
    """u = 1 is the identity; a constant cube stays constant; the mean of the
    cube is preserved; a block's value is its mean (brute force)."""
    rng = np.random.default_rng(14)
    c = rng.uniform(size=(4, 5, 6))
    np.testing.assert_array_equal(og.downsample(c, 1), c)
    np.testing.assert_allclose(og.downsample(np.full((6, 6, 6), 3.0), 2), 3.0, rtol=1e-15)
    f = rng.uniform(size=(6, 8, 10))
    d = og.downsample(f, 2)
    assert abs(d.mean() - f.mean()) < 1e-14
    assert abs(d[1, 2, 3] - f[2:4, 4:6, 6:8].mean()) < 1e-15


# --------------------------------------------------------------------------
# The whole model (Sec. 2.2.2 - 2.2.5)

def pin_unconvolved_moments(og):
    """Without PSF/LSF, each spectrum is a sampled Gaussian of width sigma0 at
    v_los.  For sigma0 >= dv and a line far from the band edges the Poisson
    summation formula makes its discrete sum, mean and variance equal the
    continuous ones to exp(-2 pi^2 sigma^2 / dv^2): m0 = I(r), m1 = v_los,
    m2 = sigma0.  (v_los and I(r) are pinned above.)"""
    G = og.Geom(12, 10, 160, 10.0, 0.0, 0.0, 0.0, 0)
    p = P(x0=5.3, y0=4.6, pa=70.0, incl=40.0, vsys=15.0, vmax=150.0, sig0=25.0)
    maps = og.evaluate(G, p)
    yy, xx = np.mgrid[0:10, 0:12]
    v, b = og.los(p, xx.astype(float), yy.astype(float))
    np.testing.assert_allclose(maps[0], b, rtol=1e-10)
    np.testing.assert_allclose(maps[1], v, rtol=0, atol=1e-8)
    np.testing.assert_allclose(maps[2], 25.0, rtol=1e-9)


def pin_mode_b_width(og):
    """LSF mode 1 folds the LSF into the line width in quadrature: without a
    PSF, m2 = sqrt(sigma0^2 + sigma_LSF^2)."""
    G = og.Geom(6, 5, 160, 10.0, 0.0, 0.0, 40.0, 1)
    p = P(x0=2.2, y0=2.1, sig0=25.0, vmax=120.0)
    maps = og.evaluate(G, p)
    sl = 40.0 / FWHM_PER_SIGMA
    np.testing.assert_allclose(maps[2], math.hypot(25.0, sl), rtol=1e-9)


def pin_lsf_variance(og):
    """LSF mode 0 without a PSF: the symmetric unit-sum LSF taps add their
    discrete variance, m2^2 = sigma0^2 + dv^2 sum_j j^2 w_j, and leave m1 and
    m0 unchanged (line far from the band edges)."""
    G = og.Geom(6, 5, 160, 10.0, 0.0, 0.0, 45.0, 0)
    p = P(x0=2.2, y0=2.1, sig0=25.0, vmax=120.0)
    maps = og.evaluate(G, p)
    sz = 45.0 / FWHM_PER_SIGMA / 10.0
    R = int(math.ceil(4 * sz))
    j = np.arange(-R, R + 1)
    w = np.exp(-j * j / (2 * sz * sz)); w /= w.sum()
    var = float((w * j * j).sum()) * 100.0
    np.testing.assert_allclose(maps[2], math.sqrt(25.0 ** 2 + var), rtol=1e-9)
    G0 = og.Geom(6, 5, 160, 10.0, 0.0, 0.0, 0.0, 0)
    m_0 = og.evaluate(G0, p)
    np.testing.assert_allclose(maps[1], m_0[1], rtol=0, atol=1e-8)
    np.testing.assert_allclose(maps[0], m_0[0], rtol=1e-10)


def pin_face_on_convolved(og):
    """Face-on disc with PSF and LSF: every spectrum is the same Gaussian at
    Vsys, so after convolution m1 = Vsys and m2^2 = sigma0^2 + LSF variance
    everywhere."""
    G = og.Geom(14, 13, 120, 10.0, 12.0, 3.0, 30.0, 0)
    p = P(x0=6.4, y0=6.2, incl=0.0, vsys=12.0, sig0=30.0)
    maps = og.evaluate(G, p)
    sz = 30.0 / FWHM_PER_SIGMA / 10.0
    R = int(math.ceil(4 * sz))
    j = np.arange(-R, R + 1)
    w = np.exp(-j * j / (2 * sz * sz)); w /= w.sum()
    m2 = math.sqrt(900.0 + 100.0 * float((w * j * j).sum()))
    np.testing.assert_allclose(maps[1], 12.0, rtol=0, atol=1e-9)
    np.testing.assert_allclose(maps[2], m2, rtol=1e-10)


def _symmetry_case(og, u):
    nx, ny = 15, 17
    G = og.Geom(nx, ny, 64, 20.0, 0.0, 2.5, 30.0, 0, u)
    p = P(x0=(nx - 1) / 2.0, y0=(ny - 1) / 2.0, pa=0.0, incl=55.0, vsys=0.0, vmax=200.0,
          rt=3.0, sig0=40.0, h=4.0)
    return og.evaluate(G, p)


def pin_reflection_symmetry(og):
    """PA = 0 puts the major axis along y.  Reflecting y about y0 (across the
    minor axis) reverses the rotation: m1 flips sign, m0 and m2 are kept.
    Reflecting x about x0 (across the major axis) keeps all three maps.  The
    PSF/LSF convolution, the down-sampling (u = 2) and the channel grid are
    symmetric, so the convolved maps obey the same symmetry."""
    for u in (1, 2):
        m = _symmetry_case(og, u)
        np.testing.assert_allclose(m[1][::-1, :], -m[1], rtol=0, atol=1e-9)
        np.testing.assert_allclose(m[0][::-1, :], m[0], rtol=1e-11)
        np.testing.assert_allclose(m[2][::-1, :], m[2], rtol=1e-11)
        np.testing.assert_allclose(m[1][:, ::-1], m[1], rtol=0, atol=1e-9)
        np.testing.assert_allclose(m[2][:, ::-1], m[2], rtol=1e-11)
        assert np.abs(m[1]).max() > 50.0


def pin_beam_smearing_linear_field(og):
    """Beam smearing of a linear velocity field: with r_t much larger than the
    field the rotation curve is solid-body, v = Vsys + k (y - y0) for PA = 0
    with k = (2/pi) (Vmax/r_t) sin i, and with h >> field the brightness is
    flat.  The PSF then mixes Gaussians of width sigma0 centred on the
    neighbours' velocities, so m1 = v and m2^2 = sigma0^2 + k^2 Var_y, where
    Var_y = sum_j j^2 w_j is the variance of the PSF taps for
    sigma_PSF = FWHM / (2 sqrt(2 ln 2))."""
    G = og.Geom(9, 11, 200, 5.0, 0.0, 3.0, 0.0, 0)
    vmax, rt, incl = 1.8e5, 1.0e4, 60.0
    p = P(x0=4.0, y0=5.0, pa=0.0, incl=incl, vsys=0.0, vmax=vmax, rt=rt, sig0=30.0, h=1e7)
    maps = og.evaluate(G, p)
    k = (2.0 / math.pi) * (vmax / rt) * math.sin(math.radians(incl))
    s = 3.0 / FWHM_PER_SIGMA
    R = int(math.ceil(4 * s))
    j = np.arange(-R, R + 1)
    w = np.exp(-j * j / (2 * s * s)); w /= w.sum()
    var_y = float((w * j * j).sum())
    yy = np.arange(11.0)[:, None] * np.ones((1, 9))
    np.testing.assert_allclose(maps[1], k * (yy - 5.0), rtol=0, atol=2e-3)
    np.testing.assert_allclose(maps[2] ** 2, 900.0 + k * k * var_y, rtol=1e-4)


def pin_mode_a_close_to_b(og):
    """LSF as a z convolution (mode 0) and folded into the width (mode 1)
    describe the same observation; they agree to the discretisation of the
    LSF taps (about 1e-2 km/s here)."""
    a = og.evaluate(og.Geom(16, 16, 64, 20.0, 0.0, 2.5, 30.0, 0), P(x0=7.6, y0=7.4))
    b = og.evaluate(og.Geom(16, 16, 64, 20.0, 0.0, 2.5, 30.0, 1), P(x0=7.6, y0=7.4))
    np.testing.assert_allclose(a[1], b[1], rtol=0, atol=0.05)
    np.testing.assert_allclose(a[2], b[2], rtol=2e-3)


def pin_upsampling_converges(og):
    """u = 2 and u = 1 describe the same sky; for a smooth model they agree
    to a small fraction of the velocity scale."""
    G1 = og.Geom(12, 12, 48, 20.0, 0.0, 3.0, 30.0, 0, 1)
    G2 = og.Geom(12, 12, 48, 20.0, 0.0, 3.0, 30.0, 0, 2)
    p = P(x0=5.4, y0=5.7, rt=4.0, h=5.0, sig0=50.0)
    a, b = og.evaluate(G1, p), og.evaluate(G2, p)
    assert np.abs(a[1] - b[1]).max() < 3.0
    assert np.abs(a[2] - b[2]).max() < 3.0


# --------------------------------------------------------------------------
# Goodness of fit (Sec. 2.2.6, Eq. 11)

def pin_chi2_hand(og):
    """2x2 hand-computed case: one masked spaxel, one invalid spaxel.
      spaxel 0: (2 (101 - 100))^2 + (0.5 (22 - 20))^2 = 4 + 1 = 5
      spaxel 1: masked; spaxel 2: m0 = 0 (invalid)
      spaxel 3: (1 (-3 - 0))^2 + (0.25 (10 - 14))^2 = 9 + 1 = 10."""
    maps = np.array([[[1.0, 1.0], [0.0, 2.0]],
                     [[101.0, 50.0], [0.0, -3.0]],
                     [[22.0, 5.0], [0.0, 10.0]]])
    obs = og.Obs(v=np.array([[100.0, 0.0], [7.0, 0.0]]), s=np.array([[20.0, 0.0], [9.0, 14.0]]),
                 w_v=np.array([[2.0, 1.0], [1.0, 1.0]]), w_s=np.array([[0.5, 1.0], [1.0, 0.25]]),
                 mask=np.array([[1, 0], [1, 1]]))
    c, r = og.chi2_maps(maps, obs, want_resid=True)
    assert abs(c - 15.0) < 1e-12, c
    np.testing.assert_allclose(r[0], [[2.0, 0.0], [0.0, -3.0]], atol=1e-12)
    np.testing.assert_allclose(r[1], [[1.0, 0.0], [0.0, -1.0]], atol=1e-12)


def pin_chi2_noiseless(og):
    """Observed maps made from the true parameters give chi2 = 0 (up to the
    FP32 storage of the observed maps)."""
    G = og.Geom(10, 9, 40, 20.0, 0.0, 2.0, 30.0, 0)
    p = P(x0=4.6, y0=4.3)
    m = og.evaluate(G, p)
    wv = np.full((9, 10), 0.2); ws = np.full((9, 10), 0.2 / math.sqrt(2))
    obs = og.Obs(m[1], m[2], wv, ws, np.ones((9, 10)))
    c = og.chi2_batch(G, p[None], obs)[0]
    assert c < 1e-9, c


def pin_parameter_domain(og):
    """Where the model is undefined -- i = 90 (Eq. 3 divides by cos i), r_t
    = 0 (Eq. 6 divides by r_t), sigma0 = 0 (a zero-width Gaussian), h = 0
    (Eq. 5), I0 <= 0 (no light), a non-finite value -- maps and chi2 are NaN,
    and so are the residuals of unmasked spaxels (masked ones stay 0); just
    inside (i = 89.9, i = 0) they are finite.  A velocity field needs only
    the kinematic values (sigma0 = 0 is a valid constant dispersion)."""
    G = og.Geom(8, 7, 24, 20.0, 0.0, 2.0, 30.0, 0)
    ok = P(x0=3.6, y0=3.3)
    m = np.ones((7, 8))
    m[2, 3] = 0
    obs = og.Obs(np.zeros((7, 8)), np.full((7, 8), 30.0), np.full((7, 8), 0.2), np.full((7, 8), 0.1), m)
    for k, v in ((PAR["incl"], 90.0), (PAR["incl"], 95.0), (PAR["rt"], 0.0), (PAR["sig0"], 0.0),
                 (PAR["h"], 0.0), (PAR["i0"], 0.0), (PAR["x0"], float("nan")), (PAR["vmax"], float("inf"))):
        q = ok.copy()
        q[k] = v
        assert np.all(np.isnan(og.evaluate(G, q))), (k, v)
        c, r = og.chi2_batch(G, q[None], obs, want_resid=True)
        assert np.isnan(c[0]) and np.all(np.isnan(r[0][:, m != 0])) and np.all(r[0][:, m == 0] == 0.0), (k, v)
    for incl in (0.0, 89.9):
        q = ok.copy()
        q[PAR["incl"]] = incl
        assert np.all(np.isfinite(og.evaluate(G, q))) and np.isfinite(og.chi2_batch(G, q[None], obs)[0]), incl
    for model in (1, 2):
        V = og.Geom(8, 7, 1, 20.0, 0.0, 0.0, 0.0, model=model)
        q = ok.copy()
        q[PAR["sig0"]] = 0.0
        q[PAR["i0"]], q[PAR["h"]] = 1.5, 0.8  # the Epinat slopes
        assert np.all(np.isfinite(og.evaluate(V, q))), model
        q[PAR["incl"]] = 90.0
        assert np.all(np.isnan(og.evaluate(V, q))), model


def pin_chi2_statistics(og):
    """At the true parameters with Gaussian noise of standard deviation E on
    both maps and weights 1/E, chi2 follows a chi-squared distribution with
    2N degrees of freedom: its mean over 100 seeds is 2N within 4 standard
    errors sqrt(2 * 2N / 100)."""
    G = og.Geom(8, 8, 40, 20.0, 0.0, 2.0, 30.0, 0)
    p = P(x0=3.6, y0=3.3)
    m = og.evaluate(G, p)
    N = 64
    vals = []
    for seed in range(100):
        rng = np.random.default_rng(1000 + seed)
        obs = og.Obs(m[1] + rng.normal(0, 5.0, (8, 8)), m[2] + rng.normal(0, 7.0, (8, 8)),
                     np.full((8, 8), 0.2), np.full((8, 8), 1 / 7.0), np.ones((8, 8)))
        vals.append(og.chi2_maps(m, obs))
    mean = float(np.mean(vals))
    assert abs(mean - 2 * N) < 4 * math.sqrt(2 * 2 * N / 100.0), mean


# --------------------------------------------------------------------------
# Velocity-field strategy (Sec. 2.2.1): Eq. 8 per pixel, arctan (Eq. 6) or
# Epinat (Eq. 7) rotation curve; slots 8, 9 hold the Epinat slopes a, g.

def _vf(og, model, nx=21, ny=17):
    return og.Geom(nx, ny, 1, 10.0, 0.0, 0.0, 0.0, 0, model=model)


def pin_vfield_face_on(og):
    """i = 0: the field is Vsys everywhere, for both curves; m0 = 1 (every
    pixel valid) and m2 = sigma_model."""
    for model in (1, 2):
        p = P(incl=0.0, sig0=37.0, i0=1.5, h=0.8)
        m = og.evaluate(_vf(og, model), p)
        np.testing.assert_allclose(m[1], 12.0, rtol=0, atol=1e-12)
        np.testing.assert_array_equal(m[0], 1.0)
        np.testing.assert_array_equal(m[2], 37.0)


def pin_vfield_pa_flip(og):
    """PA -> PA + 180 deg reverses the rotation: v - Vsys changes sign."""
    for model in (1, 2):
        p = P(pa=35.0, i0=2.0, h=1.3)
        q = P(pa=215.0, i0=2.0, h=1.3)
        a = og.evaluate(_vf(og, model), p)[1] - 12.0
        b = og.evaluate(_vf(og, model), q)[1] - 12.0
        np.testing.assert_allclose(b, -a, rtol=0, atol=1e-9)
        assert np.max(np.abs(a)) > 10.0


def pin_vfield_major_axis_values(og):
    """PA = 90 deg puts the major axis on the row y = y0 with x_e = -(x - x0),
    so v = Vsys - sign(x - x0) Vrot(|x - x0|) sin i.  Hand values at
    r_t = 2 px, V_t = 200 km/s, i = 30 deg (sin i = 1/2):
      arctan: Vrot(r_t) = V_t / 2 = 100; Vrot(sqrt(3) r_t) is off the grid,
              Vrot(2 r_t) = (2/pi) V_t atan 2 = 140.9666...;
      Epinat a = g = 1: Vrot(r_t) = V_t / 2, Vrot(2 r_t) = 2 V_t / 3;
      Epinat a = 2, g = 1 (declining): Vrot(r_t) = V_t / 2, Vrot(2 r_t) = 2 V_t / 5;
      Epinat a = 1, g = 2 (rising):    Vrot(2 r_t) = 4 V_t / 3."""
    x0, y0 = 10.0, 8.0
    cases = [(1, 1.0, 1.0, 100.0, 200.0 * 2.0 / math.pi * math.atan(2.0)),
             (2, 1.0, 1.0, 100.0, 400.0 / 3.0),
             (2, 2.0, 1.0, 100.0, 80.0),
             (2, 1.0, 2.0, 100.0, 800.0 / 3.0)]
    for model, a, g, v_rt, v_2rt in cases:
        p = P(x0=x0, y0=y0, pa=90.0, incl=30.0, vsys=12.0, vmax=200.0, rt=2.0, i0=a, h=g)
        m = og.evaluate(_vf(og, model), p)
        row = m[1][int(y0)]
        for dx, vr in ((2, v_rt), (4, v_2rt)):
            assert abs(row[int(x0) + dx] - (12.0 - 0.5 * vr)) < 1e-9, (model, a, g, dx)
            assert abs(row[int(x0) - dx] - (12.0 + 0.5 * vr)) < 1e-9, (model, a, g, -dx)


def pin_vfield_minor_axis_and_centre(og):
    """On the minor axis (x_e = 0: the column x = x0 at PA = 90 deg) and at the
    centre itself the field is Vsys, for both curves and any slopes."""
    for model, a, g in ((1, 1.0, 1.0), (2, 1.0, 0.5), (2, 3.0, 0.2)):
        p = P(x0=10.0, y0=8.0, pa=90.0, incl=60.0, vsys=-7.0, vmax=250.0, rt=3.0, i0=a, h=g)
        col = og.evaluate(_vf(og, model), p)[1][:, 10]
        np.testing.assert_allclose(col, -7.0, rtol=0, atol=1e-9)


def pin_vfield_equals_unconvolved_cube(og):
    """The two strategies share Eq. 8: the arctan velocity field equals m1 of
    an unconvolved cube whose lines sit far from the band edges (Poisson
    summation makes the discrete mean exact to ~exp(-2 pi^2 sigma^2/dv^2))."""
    p = P(x0=5.3, y0=4.6, pa=70.0, incl=40.0, vsys=15.0, vmax=150.0, sig0=25.0)
    cube = og.evaluate(og.Geom(12, 10, 160, 10.0, 0.0, 0.0, 0.0, 0), p)
    vf = og.evaluate(og.Geom(12, 10, 1, 10.0, 0.0, 0.0, 0.0, 0, model=1), p)
    np.testing.assert_allclose(vf[1], cube[1], rtol=0, atol=1e-8)


ALL_PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]
