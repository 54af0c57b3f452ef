"""Pins for the oracle's backprojection sum (Sec. II-A: Eq. 1 inverted per pixel)."""
import numpy as np
import pytest

import oracle
from oracle import brute

SIG = oracle.Signal(fc=100e3, fs=40e3, c=1500.0, t0=0.025, n_samples=512)


def _scene(P=6, C=2, seed=0, attitude=True):
    rng = np.random.default_rng(seed)
    pos = np.stack([np.arange(P) * 0.1, rng.normal(0, 0.02, P), -10.0 + rng.normal(0, 0.02, P)], 1)
    att = rng.uniform(-0.05, 0.05, size=(P, 3)) if attitude else np.zeros((P, 3))
    txl = np.array([0.01, -0.02, 0.03])
    rxl = np.stack([(np.arange(C) - 0.5 * (C - 1)) * 0.025, np.full(C, 0.01), np.zeros(C)], 1)
    return pos, att, txl, rxl


def _random_echo(P, C, Ns, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(P, C, Ns)) + 1j * rng.normal(size=(P, C, Ns))


def _pixels(nx=12, ny=10, x0=0.1, y0=16.0, d=0.02):
    return oracle.grid_points(x0, y0, 0.0, d, d, 0.0, nx, ny, 1)


@pytest.mark.parametrize("taps,beta", [(8, 4.0), (32, 10.0)])
def test_matches_numpy_brute_force(taps, beta):
    pos, att, txl, rxl = _scene(P=8, C=2, seed=1)
    tx, rx = oracle.sensor_positions(pos, att, txl, rxl)
    txb, rxb = brute.sensor_positions(pos, att, txl, rxl)
    e = _random_echo(8, 2, SIG.n_samples, 2)
    pix = _pixels(16, 16)
    a = oracle.backproject(tx, rx, SIG, e, taps, beta, pix)
    b = brute.backproject(txb, rxb, SIG.fc, SIG.fs, SIG.c, SIG.t0, e, taps, beta, pix)
    assert oracle.rel_l2(a, b) < 1e-10


def test_edges_read_zero_outside_the_row():
    """Pixels whose tap windows straddle sample 0 or Ns-1 see zeros there
    (checked against the brute force, which masks explicitly)."""
    pos, att, txl, rxl = _scene(P=3, C=2, seed=3)
    tx, rx = oracle.sensor_positions(pos, att, txl, rxl)
    e = _random_echo(3, 2, SIG.n_samples, 4)
    r0 = SIG.t0 * SIG.c / 2.0
    r1 = (SIG.t0 + SIG.n_samples / SIG.fs) * SIG.c / 2.0
    ys = np.concatenate([np.linspace(np.sqrt(r0 ** 2 - 100) - 0.3, np.sqrt(r0 ** 2 - 100) + 0.3, 30),
                         np.linspace(np.sqrt(r1 ** 2 - 100) - 0.3, np.sqrt(r1 ** 2 - 100) + 0.3, 30)])
    pix = np.stack([np.full(60, 0.1), ys, np.zeros(60)], 1)
    a = oracle.backproject(tx, rx, SIG, e, 8, 4.0, pix)
    b = brute.backproject(tx, rx, SIG.fc, SIG.fs, SIG.c, SIG.t0, e, 8, 4.0, pix)
    assert oracle.rel_l2(a, b) < 1e-10
    assert np.abs(a[:5]).max() == 0.0 and np.abs(a[-5:]).max() == 0.0


def test_linearity_in_echo():
    pos, att, txl, rxl = _scene(seed=5)
    tx, rx = oracle.sensor_positions(pos, att, txl, rxl)
    e1, e2 = _random_echo(6, 2, SIG.n_samples, 6), _random_echo(6, 2, SIG.n_samples, 7)
    a, b = 0.7 - 0.2j, -1.3 + 0.4j
    pix = _pixels()
    lhs = oracle.backproject(tx, rx, SIG, a * e1 + b * e2, 8, 4.0, pix)
    rhs = a * oracle.backproject(tx, rx, SIG, e1, 8, 4.0, pix) + b * oracle.backproject(tx, rx, SIG, e2, 8, 4.0, pix)
    assert oracle.rel_l2(lhs, rhs) < 1e-13


def test_translation_invariance():
    pos, att, txl, rxl = _scene(seed=8)
    tx, rx = oracle.sensor_positions(pos, att, txl, rxl)
    e = _random_echo(6, 2, SIG.n_samples, 9)
    pix = _pixels()
    v = np.array([3.1, -2.7, 0.9])
    a = oracle.backproject(tx, rx, SIG, e, 8, 4.0, pix)
    b = oracle.backproject(tx + v, rx + v, SIG, e, 8, 4.0, pix + v)
    assert oracle.rel_l2(a, b) < 1e-9


@pytest.mark.parametrize("taps,beta,tol", [(32, 10.0, 1e-4), (8, 4.0, 2e-2)])
def test_point_scatterer_closed_form(taps, beta, tol):
    """One noiseless point of complex amplitude A on a pixel, ideal compressed
    pulse sinc(B t): the image peaks at that pixel with I = A P C (the echo's
    carrier term exp(-j 2 pi fc tau) is undone exactly; the only error is the
    interpolator's).  Sensor positions are written out here (zero attitude,
    position + lever arm) rather than taken from the oracle's geometry."""
    P, C = 16, 3
    pos = np.stack([np.arange(P) * 0.1, np.zeros(P), np.full(P, -10.0)], 1)
    txl = np.array([0.0, 0.0, 0.0])
    rxl = np.stack([(np.arange(C) - 1) * 0.025, np.zeros(C), np.zeros(C)], 1)
    tx = pos + txl
    rx = pos[:, None, :] + rxl[None]
    d = 0.02
    nx, ny = 15, 15
    x0, y0 = 0.6, 18.0
    ixs, iys = 7, 6
    A = 0.8 * np.exp(1j * 0.9)
    xs = np.array([x0 + ixs * d, y0 + iys * d, 0.0])
    sig = oracle.Signal(100e3, 40e3, 1500.0, 0.02, 1024)
    echo = oracle.simulate_points(tx, rx, sig, 20e3, 0.0, [[*xs, A.real, A.imag]])
    pix = oracle.grid_points(x0, y0, 0.0, d, d, 0.0, nx, ny, 1)
    img = oracle.backproject(tx, rx, sig, echo, taps, beta, pix).reshape(ny, nx)
    iy, ix = np.unravel_index(np.argmax(np.abs(img)), img.shape)
    assert (ix, iy) == (ixs, iys)
    peak = img[iys, ixs]
    assert abs(peak - A * P * C) <= tol * abs(A) * P * C


def test_adjoint_dot_product():
    """<B e, I> = <e, B^H I> with <a, b> = sum conj(a) b."""
    pos, att, txl, rxl = _scene(P=5, C=2, seed=10)
    tx, rx = oracle.sensor_positions(pos, att, txl, rxl)
    e = _random_echo(5, 2, SIG.n_samples, 11)
    pix = _pixels(9, 7)
    rng = np.random.default_rng(12)
    img = rng.normal(size=pix.shape[0]) + 1j * rng.normal(size=pix.shape[0])
    Be = oracle.backproject(tx, rx, SIG, e, 8, 4.0, pix)
    BhI = oracle.backproject_adjoint(tx, rx, SIG, img, 8, 4.0, pix)
    lhs = np.vdot(Be, img)
    rhs = np.vdot(e, BhI)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_sharpness_special_cases():
    img = np.zeros(10, dtype=complex)
    img[3] = 2.0 - 1.0j
    assert abs(oracle.sharpness(img)[0] - 1.0) < 1e-15
    u = np.exp(1j * np.linspace(0, 3, 25)) * 1.7
    assert abs(oracle.sharpness(u)[0] - 1.0 / 25) < 1e-15
    rng = np.random.default_rng(13)
    z = rng.normal(size=40) + 1j * rng.normal(size=40)
    assert abs(oracle.sharpness(z)[0] - oracle.sharpness(3.3j * z)[0]) < 1e-14


def test_sharpness_gradient_central_difference():
    rng = np.random.default_rng(14)
    z = rng.normal(size=30) + 1j * rng.normal(size=30)
    (_, _, _), g = oracle.sharpness(z, want_grad=True)
    h = 1e-7
    for p in range(0, 30, 7):
        for dirn in (1.0, 1j):
            zp, zm = z.copy(), z.copy()
            zp[p] += h * dirn
            zm[p] -= h * dirn
            fd = (oracle.sharpness(zp)[0] - oracle.sharpness(zm)[0]) / (2 * h)
            # dS/dtheta = 2 Re(conj(g) dI/dtheta)
            an = 2.0 * np.real(np.conj(g[p]) * dirn)
            assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * np.abs(g).max())


def test_offset_gradient_central_difference():
    """Analytic dS/d(dp) against central differences of S through the full
    pipeline (positions from offsets, backprojection, sharpness)."""
    P, C = 6, 2
    pos, att, txl, rxl = _scene(P=P, C=C, seed=15)
    sig = oracle.Signal(100e3, 40e3, 1500.0, 0.02, 512)
    tx0, rx0 = oracle.sensor_positions(pos, att, txl, rxl)
    scat = [[0.3, 16.1, 0.0, 0.9, 0.2], [0.2, 16.05, 0.0, -0.3, 0.6]]
    echo = oracle.simulate_points(tx0, rx0, sig, 20e3, 5e-3, scat)
    echo += 0.05 * _random_echo(P, C, sig.n_samples, 16)
    pix = oracle.grid_points(0.15, 15.95, 0.0, 0.02, 0.02, 0.0, 12, 12, 1)
    rng = np.random.default_rng(17)
    off = rng.normal(0, 0.003, size=(P, 3))

    def S(o):
        tx, rx = oracle.sensor_positions(pos, att, txl, rxl, o)
        return oracle.sharpness(oracle.backproject(tx, rx, sig, echo, 8, 4.0, pix))[0]

    tx, rx = oracle.sensor_positions(pos, att, txl, rxl, off)
    img = oracle.backproject(tx, rx, sig, echo, 8, 4.0, pix)
    _, g = oracle.sharpness(img, want_grad=True)
    grad = oracle.vjp_offsets(tx, rx, sig, echo, 8, 4.0, pix, g)
    h = 1e-6
    fd = np.zeros((P, 3))
    for i in range(P):
        for a in range(3):
            op, om = off.copy(), off.copy()
            op[i, a] += h
            om[i, a] -= h
            fd[i, a] = (S(op) - S(om)) / (2 * h)
    assert oracle.rel_l2(grad, fd) < 1e-6


def test_complex64_echo_read_in_place():
    """A complex64 echo gives the same image as its exact complex128 widening."""
    pos, att, txl, rxl = _scene(P=4, C=2, seed=20)
    tx, rx = oracle.sensor_positions(pos, att, txl, rxl)
    e = _random_echo(4, 2, SIG.n_samples, 21).astype(np.complex64)
    pix = _pixels(8, 8)
    a = oracle.backproject(tx, rx, SIG, e, 8, 4.0, pix)
    b = oracle.backproject(tx, rx, SIG, e.astype(np.complex128), 8, 4.0, pix)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("side", [1, -1])
def test_beam_mask_matches_brute_force(side):
    """Beam field of view: the C tangent-form test against the NumPy arctan2
    restatement, with attitude, on pixels both inside and outside the beam."""
    P, C = 10, 2
    pos, att, txl, rxl = _scene(P=P, C=C, seed=30)
    att[:, 2] += 0.05                         # some yaw so the beam edge moves with the ping
    tx, rx = oracle.sensor_positions(pos, att, txl, rxl)
    e = _random_echo(P, C, SIG.n_samples, 31)
    y0 = 16.0 * side
    pix = oracle.grid_points(-6.0, y0, 0.0, 0.5, 0.05, 0.0, 28, 12, 1)   # spans far forward / aft of the track
    width = np.deg2rad(40.0)
    a = oracle.backproject(tx, rx, SIG, e, 8, 4.0, pix, att=att, beam_width=width, side=side)
    m = brute.beam_mask(att, tx, rx, pix, width, side)
    assert 0.1 < m.mean() < 0.9
    b = brute.backproject(tx, rx, SIG.fc, SIG.fs, SIG.c, SIG.t0, e, 8, 4.0, pix, mask=m)
    assert oracle.rel_l2(a, b) < 1e-10


def test_beam_off_is_unmasked_and_wrong_side_is_empty():
    pos, att, txl, rxl = _scene(P=6, C=2, seed=32)
    tx, rx = oracle.sensor_positions(pos, att, txl, rxl)
    e = _random_echo(6, 2, SIG.n_samples, 33)
    pix = _pixels()
    full = oracle.backproject(tx, rx, SIG, e, 8, 4.0, pix)
    assert np.array_equal(full, oracle.backproject(tx, rx, SIG, e, 8, 4.0, pix, att=att, beam_width=0.0))
    wide = oracle.backproject(tx, rx, SIG, e, 8, 4.0, pix, att=att, beam_width=np.deg2rad(179.0), side=1)
    assert oracle.rel_l2(wide, full) < 1e-12          # the scene is broadside to starboard
    assert np.abs(oracle.backproject(tx, rx, SIG, e, 8, 4.0, pix, att=att, beam_width=np.deg2rad(179.0),
                                     side=-1)).max() == 0.0


def test_beam_adjoint_dot_product_and_gradient():
    """With the beam on, the masked adjoint stays the exact adjoint of the
    masked sum, and the masked offset gradient matches central differences."""
    P, C = 6, 2
    pos, att, txl, rxl = _scene(P=P, C=C, seed=34)
    width = np.deg2rad(30.0)
    tx, rx = oracle.sensor_positions(pos, att, txl, rxl)
    e = _random_echo(P, C, SIG.n_samples, 35)
    pix = oracle.grid_points(-7.0, 16.0, 0.0, 1.0, 0.05, 0.0, 14, 8, 1)   # beam edges at about x = -4, +4.8
    rng = np.random.default_rng(36)
    img = rng.normal(size=pix.shape[0]) + 1j * rng.normal(size=pix.shape[0])
    kw = dict(att=att, beam_width=width, side=1)
    Be = oracle.backproject(tx, rx, SIG, e, 8, 4.0, pix, **kw)
    BhI = oracle.backproject_adjoint(tx, rx, SIG, img, 8, 4.0, pix, **kw)
    m = brute.beam_mask(att, tx, rx, pix, width, 1)
    assert 0.1 < m.mean() < 0.9                       # the beam edge crosses the pixels
    lhs, rhs = np.vdot(Be, img), np.vdot(e, BhI)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # gradient of S through the masked sum (the mask moves with the offsets,
    # but central differences of size h rarely cross its edge)
    off = rng.normal(0, 0.002, size=(P, 3))

    def S(o):
        t, r = oracle.sensor_positions(pos, att, txl, rxl, o)
        return oracle.sharpness(oracle.backproject(t, r, SIG, e, 8, 4.0, pix, **kw))[0]

    t, r = oracle.sensor_positions(pos, att, txl, rxl, off)
    _, g = oracle.sharpness(oracle.backproject(t, r, SIG, e, 8, 4.0, pix, **kw), want_grad=True)
    grad = oracle.vjp_offsets(t, r, SIG, e, 8, 4.0, pix, g, **kw)
    h = 1e-7
    fd = np.zeros((P, 3))
    for i in range(P):
        for a in range(3):
            op, om = off.copy(), off.copy()
            op[i, a] += h
            om[i, a] -= h
            fd[i, a] = (S(op) - S(om)) / (2 * h)
    assert oracle.rel_l2(grad, fd) < 1e-5


def test_beam_split_bounds_every_nearby_decision():
    """Margin split of the beam-limited sum: eps -> 0 gives the plain sum with
    no ambiguous terms; beam widths perturbed by a relative +-eps (each moves
    the decision margins by well under eps) change the image only through
    ambiguous terms, so |I_perturbed - sure| <= amb pixel by pixel, and they do
    change it; the ambiguous sum grows with eps."""
    P, C = 10, 2
    pos, att, txl, rxl = _scene(P=P, C=C, seed=37)
    att[:, 2] += 0.05
    tx, rx = oracle.sensor_positions(pos, att, txl, rxl)
    e = _random_echo(P, C, SIG.n_samples, 38)
    pix = oracle.grid_points(-6.0, 16.0, 0.0, 0.5, 0.05, 0.0, 28, 12, 1)
    width = np.deg2rad(40.0)
    kw = dict(att=att, side=1)
    plain = oracle.backproject(tx, rx, SIG, e, 8, 4.0, pix, beam_width=width, **kw)
    sure0, amb0 = oracle.backproject_beam_split(tx, rx, SIG, e, 8, 4.0, pix, att, width, 1, eps=1e-15)
    assert amb0.max() == 0.0 and oracle.rel_l2(sure0, plain) < 1e-14
    eps = 1e-2
    sure, amb = oracle.backproject_beam_split(tx, rx, SIG, e, 8, 4.0, pix, att, width, 1, eps=eps)
    assert np.count_nonzero(amb) > 0
    changed = 0
    for f in (1.0 - eps, 1.0 + eps):
        pert = oracle.backproject(tx, rx, SIG, e, 8, 4.0, pix, beam_width=width * f, **kw)
        assert np.all(np.abs(pert - sure) <= amb + 1e-9)
        changed += np.count_nonzero(np.abs(pert - plain) > 1e-9)
    assert changed > 0
    _, amb_small = oracle.backproject_beam_split(tx, rx, SIG, e, 8, 4.0, pix, att, width, 1, eps=eps / 10)
    assert np.all(amb_small <= amb + 1e-12) and amb_small.sum() < amb.sum()
