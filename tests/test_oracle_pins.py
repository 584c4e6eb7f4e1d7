"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, a special case that reduces to a textbook result, a library routine, a
brute-force evaluation, or an invariant.  They are chosen so that a dropped
term, a wrong sign or index, or a transposed operand in any oracle step fails
at least one of them.  No GPU is needed.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_21381_gb300 import scenes

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def one_particle(**kw):
    p = dict(cx=32.0, cy=32.0, theta=0.0, a=5.0, b=5.0, T=1.0, dn=0.03, mu=0.0, kind=0.0)
    p.update(kw)
    return np.array([[p[f]] for f in scenes.FIELDS], dtype=np.float32)


# ------------------------------------------------------------------ geometry
def test_sphere_opd_closed_form():
    """Sec. III.B, Eq. 2: a sphere of radius R (um) has OPD 2 dn sqrt(R^2 - r^2)."""
    dx, R_um, dn = 0.5, 3.0, 0.04
    soa = one_particle(cx=31.3, cy=30.6, a=R_um / dx, b=R_um / dx, T=2 * R_um, dn=dn,
                       theta=0.7)
    H, W = 64, 80
    opd, att = oracle.opd_att(soa, 1, H, W, dx=dx)
    y, x = np.mgrid[0:H, 0:W] + 0.5
    r2 = ((x - np.float32(31.3)) ** 2 + (y - np.float32(30.6)) ** 2) * dx * dx
    want = 2 * dn * np.sqrt(np.maximum(0.0, R_um ** 2 - r2))
    want = np.float32(dn).astype(np.float64) / dn * want  # dn is stored as fp32
    assert np.abs(opd - want).max() < 1e-12
    assert np.all(att == 0.0)
    assert opd.max() > 0.2


def sphere_chord_um(H, W, cx, cy, R_um, dx):
    """Closed-form chord 2 sqrt(R^2 - r^2) (um) of a sphere through every
    pixel centre; centre coordinates are the fp32 values the oracle reads."""
    y, x = np.mgrid[0:H, 0:W] + 0.5
    r2 = ((x - np.float32(cx)) ** 2 + (y - np.float32(cy)) ** 2) * dx * dx
    return 2 * np.sqrt(np.maximum(0.0, R_um ** 2 - r2))


def test_sphere_absorption_closed_form():
    """Eq. 4 (Beer-Lambert amplitude) composed like Eq. 2's integral: an
    absorbing sphere of radius R has absorption exponent ATT = mu * 2
    sqrt(R^2 - r^2), independent of its dn and orientation."""
    dx, R_um = 0.5, 2.5
    H, W = 48, 56
    for mu, dn, th in ((0.013, 0.02, 0.0), (0.2, 0.0, 1.9), (-0.05, 0.04, 0.4)):
        soa = one_particle(cx=27.4, cy=22.9, a=R_um / dx, b=R_um / dx, T=2 * R_um, dn=dn,
                           mu=mu, theta=th)
        opd, att = oracle.opd_att(soa, 1, H, W, dx=dx)
        want = np.float64(np.float32(mu)) * sphere_chord_um(H, W, 27.4, 22.9, R_um, dx)
        assert np.abs(att - want).max() < 1e-12
        assert np.abs(att).max() > 0.5 * abs(mu) * 2 * R_um
        # the same chord carries the OPD: ATT / OPD = mu / dn wherever dn != 0
        if dn:
            want_opd = np.float64(np.float32(dn)) * sphere_chord_um(H, W, 27.4, 22.9, R_um, dx)
            assert np.abs(opd - want_opd).max() < 1e-12


def test_beer_lambert_intensity_through_an_all_pass_pupil():
    """Eq. 2 with the amplitude of Eq. 4 imaged through a pupil that passes
    every grid frequency with unit modulus (NA beyond the grid's corner
    frequency, dz = 0): I = |E|^2 = exp(-2 ATT) at every pixel, whatever the
    phase.  ATT is taken from the closed form of two disjoint absorbing
    spheres, not from the oracle's own map."""
    dx, H, W = 0.5, 64, 64
    spheres = ((20.3, 18.6, 3.0, 0.03, 0.011), (41.8, 44.2, 2.25, 0.05, 0.07))  # fp32-exact radii
    soa = np.concatenate([one_particle(cx=cx, cy=cy, a=R / dx, b=R / dx, T=2 * R, dn=dn, mu=mu)
                          for cx, cy, R, dn, mu in spheres], axis=1)
    att = sum(np.float64(np.float32(mu)) * sphere_chord_um(H, W, cx, cy, R, dx)
              for cx, cy, R, dn, mu in spheres)
    # corner frequency sqrt(2) / (2 dx) = 1.41 cycles/um < NA / lambda = 1.82
    o = oracle.make_optics(H, W, dx=dx, lambda_um=0.55, NA=1.0, n_medium=1.5, defocus=0.0,
                           modes=1)
    I = oracle.render(soa, 2, o)["images"][0]
    assert np.abs(I - np.exp(-2 * att)).max() < 1e-12
    assert I.min() < 0.7  # the absorption did act


def test_ellipse_orientation_convention():
    """theta turns the first semi-axis from +x toward +y."""
    th = math.pi / 6
    soa = one_particle(cx=40.0, cy=40.0, a=10.0, b=2.0, theta=th)
    opd, _ = oracle.opd_att(soa, 1, 80, 80)
    on = (40 + 8 * math.cos(th), 40 + 8 * math.sin(th))
    off = (40 + 8 * math.cos(th), 40 - 8 * math.sin(th))
    assert opd[int(on[1]), int(on[0])] > 0.0
    assert opd[int(off[1]), int(off[0])] == 0.0


def test_ellipse_rotation_invariance_for_circles():
    a = one_particle(a=6.0, b=6.0, theta=0.0)
    b = one_particle(a=6.0, b=6.0, theta=1.234)
    oa, _ = oracle.opd_att(a, 1, 64, 64)
    ob, _ = oracle.opd_att(b, 1, 64, 64)
    assert np.abs(oa - ob).max() < 1e-12


def test_prism_closed_form_plateau_and_ramp():
    """Bevelled prism: chord = clamp(2 s_b d, 0, T), d the in-plane distance
    to the nearest side wall (um); plateau dn T, linear ramp at the edges."""
    dx, T, dn, sb = 0.5, 2.0, 0.05, 1.0
    for th in (0.0, 0.3, 1.1, 2.5):
        soa = one_particle(cx=40.2, cy=39.7, a=11.0, b=6.5, T=T, dn=dn, kind=1.0, theta=th)
        H = W = 80
        opd, _ = oracle.opd_att(soa, 1, H, W, dx=dx, bevel_slope=sb)
        y, x = np.mgrid[0:H, 0:W] + 0.5
        c, s = math.cos(np.float32(th)), math.sin(np.float32(th))
        ex, ey = x - np.float32(40.2), y - np.float32(39.7)
        u, v = c * ex + s * ey, -s * ex + c * ey
        d = dx * np.minimum(11.0 - np.abs(u), 6.5 - np.abs(v))
        want = np.float64(np.float32(dn)) * np.clip(2 * sb * d, 0.0, T)
        assert np.abs(opd - want).max() < 1e-12
        assert abs(opd.max() - np.float64(np.float32(dn)) * T) < 1e-12


def test_prism_bevel_slope_scales_ramp():
    """A steeper chamfer shortens the ramp: width of the ramp = T / (2 s_b)."""
    for sb in (0.5, 2.0):
        soa = one_particle(cx=40.0, cy=40.0, a=14.0, b=14.0, T=1.0, dn=1.0, kind=1.0)
        opd, _ = oracle.opd_att(soa, 1, 80, 80, dx=0.5, bevel_slope=sb)
        row = opd[40]  # y = 40.5, through the middle; x = j + 0.5
        j = np.arange(80) + 0.5
        d = 0.5 * (14.0 - np.abs(j - 40.0))
        assert np.abs(row - np.clip(2 * sb * d, 0, 1.0)).max() < 1e-12


def test_halfspace_chord_cube_and_outside():
    """Eq. 1 with a unit cube's 6 half-spaces: chord 1 inside, 0 outside."""
    A = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    b = np.full(6, 0.5)
    assert oracle.halfspace_chord(A, b, 0.1, -0.2) == pytest.approx(1.0)
    assert oracle.halfspace_chord(A, b, 0.6, 0.0) == 0.0
    # a tilted top plane z <= 0.5 - 0.5 u shortens the chord linearly
    A2 = np.vstack([A, [0.5, 0, 1]])
    b2 = np.append(b, 0.5)
    assert oracle.halfspace_chord(A2, b2, 0.4, 0.0) == pytest.approx(1.0 - 0.2)


def test_superposition_and_window():
    """Eq. 7 accumulate=True: overlaps add.  The scene map equals the sum of
    single-particle maps, and the per-particle window loses nothing."""
    rng = np.random.default_rng(5)
    soa = scenes.draw_particles(rng, 12, 48, 40, mu=(0.0, 0.03), size_scale=1.5)
    opd, att = oracle.opd_att(soa, 12, 48, 40)
    so = np.zeros_like(opd)
    sa = np.zeros_like(att)
    for p in range(12):
        o1, a1 = oracle.opd_att(np.ascontiguousarray(soa[:, p:p + 1]), 1, 48, 40,
                                full_canvas=True)
        so += o1
        sa += a1
    assert np.abs(opd - so).max() < 1e-14
    assert np.abs(att - sa).max() < 1e-14
    fo, fa = oracle.opd_att(soa, 12, 48, 40, full_canvas=True)
    assert np.array_equal(fo, opd) and np.array_equal(fa, att)
    pix = rng.integers(0, 48 * 40, 200)
    po, pa = oracle.opd_at(soa, 12, 40, pix)
    assert np.abs(po - opd.ravel()[pix]).max() < 1e-14
    assert np.abs(pa - att.ravel()[pix]).max() < 1e-14


def test_off_canvas_particles_are_clipped():
    soa = one_particle(cx=-3.0, cy=10.0, a=6.0, b=6.0)
    opd, _ = oracle.opd_att(soa, 1, 32, 32)
    assert opd[:, :3].max() > 0 and opd[:, 4:].max() == 0.0
    far = one_particle(cx=500.0, cy=10.0)
    opd2, _ = oracle.opd_att(far, 1, 32, 32)
    assert opd2.max() == 0.0


# ------------------------------------------------------------------ field
def test_field_special_values():
    """Eq. 2 with Beer-Lambert amplitude (Eq. 4): OPD = lambda/4 gives a
    quarter-wave phase i, lambda/2 gives -1, ATT = ln 2 halves the amplitude."""
    lam = 0.55
    opd = np.array([0.0, lam / 4, lam / 2, 0.0])
    att = np.array([0.0, 0.0, 0.0, math.log(2.0)])
    E = oracle.field(opd, att, lam)
    assert np.allclose(E, [1, 1j, -1, 0.5], atol=1e-15)


# ------------------------------------------------------------------ Fourier
def test_fft_matches_bruteforce_dft_32x32():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((32, 32)) + 1j * rng.standard_normal((32, 32))
    for sign in (-1, 1):
        a = oracle.fft2(x, sign)
        b = oracle.dft2_brute(x, sign)
        assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()


def test_fft_nonsquare_matches_numpy():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((64, 256)) + 1j * rng.standard_normal((64, 256))
    a = oracle.fft2(x, -1)
    assert np.abs(a - np.fft.fft2(x)).max() < 1e-11 * np.abs(a).max()
    b = oracle.fft2(x, +1)
    assert np.abs(b - np.fft.ifft2(x) * x.size).max() < 1e-11 * np.abs(b).max()


def test_parseval_all_pass_pupil():
    """A pupil of modulus one (circle larger than every grid frequency, pure
    defocus phase) conserves energy: sum I = sum |E|^2."""
    rng = np.random.default_rng(3)
    E = np.exp(1j * rng.uniform(0, 6, (64, 32))) * rng.uniform(0.5, 1.0, (64, 32))
    o = oracle.make_optics(64, 32, NA=20.0, n_medium=40.0, defocus=1.7, modes=1)
    I = oracle.images_from_field(o, E)[0]
    assert abs(I.sum() - (np.abs(E) ** 2).sum()) < 1e-10 * I.sum()
    assert np.abs(I - np.abs(E) ** 2).max() > 1e-3  # the phase did act


def test_empty_field_uniform_background():
    """No particles: brightfield and oblique (|k_ill| < k_NA) image 1, DIC
    images 4 sin^2(theta_b) (Eq. 5 with U = 1)."""
    o = oracle.make_optics(64, 64, modes=7, defocus=1.3, bias_phase=0.6)
    I = oracle.render(np.zeros((9, 1), np.float32), 0, o)["images"]
    assert np.abs(I[0] - 1).max() < 1e-12
    assert np.abs(I[1] - 1).max() < 1e-12
    assert np.abs(I[2] - 4 * math.sin(0.6) ** 2).max() < 1e-12


def test_airy_first_zero():
    """Coherent point response of the circ pupil (Eq. 3 at dz = 0):
    |h|^2 has its first zero at 0.61 lambda / NA."""
    N, dx, lam, NA = 512, 0.05, 0.55, 0.4
    E = np.zeros((N, N), complex)
    E[N // 2, N // 2] = 1.0
    o = oracle.make_optics(N, N, dx=dx, lambda_um=lam, NA=NA, modes=1)
    I = oracle.images_from_field(o, E)[0]
    row = I[N // 2, N // 2:N // 2 + 40]
    k = int(np.argmin(row[5:30])) + 5
    a, b, c = row[k - 1], row[k], row[k + 1]
    x0 = k + 0.5 * (a - c) / (a - 2 * b + c)
    want = 0.6098 * lam / NA / dx  # first zero of J1(x)/x at x = 3.8317
    assert abs(x0 - want) < 0.02 * want
    assert b < 1e-3 * row[0]


def test_weak_phase_defocus_transfer():
    """Weak phase object E = exp(i eps phi) through a centred circ + defocus
    pupil: the intensity spectrum is -2 eps sin(chi(k)) phi_hat(k) inside the
    aperture to O(eps^2), with chi = dz (sqrt(k0^2 - k^2) - k0); at dz = 0 the
    linear phase contrast vanishes."""
    H, W = 64, 128
    rng = np.random.default_rng(4)
    phi = rng.standard_normal((H, W))
    eps = 1e-5
    for dz in (1.5, -2.0, 0.0):
        o = oracle.make_optics(H, W, dx=0.25, NA=0.5, defocus=dz, modes=1)
        I = oracle.images_from_field(o, np.exp(1j * eps * phi))[0]
        spec = np.fft.fft2(I - 1.0)
        kx = 2 * np.pi * np.fft.fftfreq(W, 0.25)[None, :]
        ky = 2 * np.pi * np.fft.fftfreq(H, 0.25)[:, None]
        k2 = kx ** 2 + ky ** 2
        kna, k0 = 2 * np.pi * 0.5 / 0.55, 2 * np.pi / 0.55
        inside = k2 <= kna ** 2
        chi = dz * (np.sqrt(np.maximum(k0 ** 2 - k2, 0)) - k0)
        want = -2 * eps * np.sin(chi) * np.fft.fft2(phi)
        err = np.abs(spec - want)[inside].max()
        assert err < 50 * eps ** 2 * H * W
        if dz == 0.0:
            assert np.abs(spec[inside]).max() < 50 * eps ** 2 * H * W
        else:
            assert np.abs(want[inside]).max() > 1e3 * err


def plane_wave(H, W, fx, fy):
    y, x = np.mgrid[0:H, 0:W]
    return np.exp(2j * np.pi * (fx * x / W + fy * y / H))


def test_dic_plane_wave_uniform_intensity():
    """Eq. 5 for a plane wave exp(i k.r): U(r + ds) e^{i theta} -
    U(r - ds) e^{-i theta} has uniform modulus^2 4 sin^2(k.ds + theta)."""
    H, W, dx = 64, 64, 0.5
    for (fx, fy, bias, ang) in [(3, 1, math.pi / 4, math.pi / 4), (-5, 2, 0.3, 1.0),
                                (0, -4, 1.2, 0.0)]:
        o = oracle.make_optics(H, W, dx=dx, NA=0.5, modes=4, bias_phase=bias,
                               shear_px=1.0, shear_angle=ang)
        I = oracle.images_from_field(o, plane_wave(H, W, fx, fy))[0]
        kx, ky = 2 * np.pi * fx / (W * dx), 2 * np.pi * fy / (H * dx)
        ds = 0.5 * 1.0 * dx
        want = 4 * math.sin(kx * ds * math.cos(ang) + ky * ds * math.sin(ang) + bias) ** 2
        assert np.abs(I - want).max() < 1e-12


def test_oblique_offset_direction():
    """Tilted illumination shifts the pupil: a plane wave at k passes iff
    |k + k_ill| <= k_NA (k_ill = 0.3 k_NA along +x here)."""
    H = W = 64
    dx, lam, NA = 0.5, 0.55, 0.4
    kna = 2 * np.pi * NA / lam
    o = oracle.make_optics(H, W, dx=dx, lambda_um=lam, NA=NA, modes=2,
                           oblique_frac=0.3, oblique_angle=0.0)
    step = 2 * np.pi / (W * dx)
    f_pass = int(-0.9 * kna / step)   # |k + k_ill| ~ 0.6 k_NA: passes
    f_block = int(0.85 * kna / step)  # |k + k_ill| ~ 1.15 k_NA: blocked
    assert abs(f_block * step) < kna and abs(f_pass * step) < kna
    Ip = oracle.images_from_field(o, plane_wave(H, W, f_pass, 0))[0]
    Ib = oracle.images_from_field(o, plane_wave(H, W, f_block, 0))[0]
    assert np.abs(Ip - 1).max() < 1e-12
    assert np.abs(Ib).max() < 1e-20


def test_pupil_circle_is_closed():
    """The circ pupil includes its rim: a plane wave exactly at |k| = k_NA
    passes (grid chosen so the rim falls exactly on a sample)."""
    H = W = 64
    o = oracle.make_optics(H, W, dx=0.5, lambda_um=0.5, NA=0.125, modes=1)
    assert np.abs(oracle.images_from_field(o, plane_wave(H, W, 8, 0))[0] - 1).max() < 1e-12
    assert np.abs(oracle.images_from_field(o, plane_wave(H, W, 9, 0))[0]).max() < 1e-20
    Ht = oracle.transfer(o, 1)
    assert Ht[0, 8] == 1.0 and Ht[8, 0] == 1.0 and Ht[0, 9] == 0.0


def test_transfer_axes_not_transposed():
    """On a non-square grid the pupil's k_x runs along columns (W) and k_y
    along rows (H): count samples inside the circle per axis."""
    o = oracle.make_optics(32, 128, dx=0.5, NA=0.4, modes=1)
    Ht = oracle.transfer(o, 1)
    kna = 2 * np.pi * 0.4 / 0.55
    nx = np.sum(np.abs(2 * np.pi * np.fft.fftfreq(128, 0.5)) <= kna)
    ny = np.sum(np.abs(2 * np.pi * np.fft.fftfreq(32, 0.5)) <= kna)
    assert np.count_nonzero(Ht[0]) == nx
    assert np.count_nonzero(Ht[:, 0]) == ny


def test_render_c0_background_and_finiteness():
    soa, o = scenes.plain_256()
    out = oracle.render(soa, soa.shape[1], o)
    assert out["images"].shape == (2, 256, 256)
    assert np.all(np.isfinite(out["images"]))
    assert abs(np.median(out["images"][0]) - 1.0) < 0.05
    assert out["opd"].max() > 0.01
