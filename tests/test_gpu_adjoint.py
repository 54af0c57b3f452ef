"""GPU parity of the adjoints: the linear adjoint (image -> echo), the
gradient with respect to per-ping position offsets, and the autofocus loop
built on it."""
import numpy as np
import pytest

import oracle
import paper_2101_05888_gb300 as sas
from paper_2101_05888_gb300 import synth

from _scene import grid_pixels, in_band, lib_signal, oracle_positions, oracle_signal, point_echo

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BETA = 4.0
# The adjoint scatters each pixel through the interpolator's taps, so its echo
# output carries the Farrow form's weight error (4.2e-4 at most per tap, most
# of it at |nu| > 1/4) at every frequency; inside the echoes' band (|nu| <= 1/4,
# what any band-limited echo is compared on) it is held to the FP32 tolerance.
ADJ_FULL_BAND = 1e-3


def _small(name="small_2d", **kw):
    w = synth.workload(name)
    return synth.scaled(w, **kw)


@pytest.mark.parametrize("dim3", [False, True])
def test_linear_adjoint_matches_oracle(dim3):
    if dim3:
        g = synth.Grid(0.5, 0.7, 0.0, 0.02, 0.02, 0.02, 20, 30, 9)
        w = synth.workload("volume_3d", grid=g, n_pings=16, n_rx=4, n_samples=2048, lattice=4, lattice_pitch=0.4)
    else:
        w = _small(n_pings=13, n_rx=3, nx=60, ny=70, n_samples=1024)
    nav = synth.nav(w)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    img = synth.random_image((w.grid.nz, w.grid.ny, w.grid.nx), seed=3).astype(np.complex64)
    eadj = torch.empty((w.n_pings, w.n_rx, w.n_samples), dtype=torch.complex64, device="cuda")
    sas.sas_backproject_adjoint(geom.h, sas.grid_from(w.grid), sas.kaiser(BETA), torch.from_numpy(img).cuda(), eadj)
    geom.sync_status()
    tx, rx = oracle_positions(nav)
    ref = oracle.backproject_adjoint(tx, rx, oracle_signal(w), img.reshape(-1), 8, BETA, grid_pixels(w.grid))
    got = eadj.cpu().numpy()
    e_band, e_full = oracle.rel_l2(in_band(got), in_band(ref)), oracle.rel_l2(got, ref)
    print("linear adjoint vs oracle: in band %.3g, full band %.3g" % (e_band, e_full))
    assert e_band < 1e-4
    assert e_full < ADJ_FULL_BAND
    geom.close()


def test_gpu_dot_product():
    """<B e, I> = <e, B^H I> with both operators on the GPU (FP32)."""
    w = _small(n_pings=64, n_rx=4, nx=256, ny=128, n_samples=2048)
    nav = synth.nav(w)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    e = synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=4)
    geom.upload_echo(e)
    Be = geom.backproject(sas.grid_from(w.grid), sas.kaiser(BETA)).cpu().numpy().astype(np.complex128)
    I = synth.random_image(Be.shape, seed=5).astype(np.complex64)
    eadj = torch.empty((w.n_pings, w.n_rx, w.n_samples), dtype=torch.complex64, device="cuda")
    sas.sas_backproject_adjoint(geom.h, sas.grid_from(w.grid), sas.kaiser(BETA), torch.from_numpy(I).cuda(), eadj)
    geom.sync_status()
    lhs = np.vdot(Be.reshape(-1), I.reshape(-1).astype(np.complex128))
    rhs = np.vdot(e.reshape(-1).astype(np.complex128), eadj.cpu().numpy().reshape(-1).astype(np.complex128))
    # FP32 rounding in both operators moves <B e, I> by ~1e-6 of a random
    # inner product's size |B e| |I| / sqrt(n); a wrong term or sign in the
    # adjoint would move it by O(1) of that size
    assert abs(lhs - rhs) <= 2e-5 * np.linalg.norm(Be) * np.linalg.norm(I) / np.sqrt(I.size)
    geom.close()


def _grad_case(P=24, C=4, n=64, seed=6):
    base = synth.workload("autofocus_2d")
    g = synth.Grid(base.grid.x0 + 10.0, base.grid.y0 + 5.0, 0.0, 0.015, 0.015, 0.0, n, n, 1)
    w = synth.workload("autofocus_2d", grid=g, n_pings=P, n_rx=C, n_samples=4096, t0=0.04,
                       ping_spacing=0.1)
    nav = synth.nav(w)
    # place the track so the small grid sits broadside to it
    nav["pos"][:, 0] += g.x0 - 0.5 * P * 0.1
    nav["true_pos"][:, 0] += g.x0 - 0.5 * P * 0.1
    return w, nav


def test_offset_gradient_matches_oracle():
    w, nav = _grad_case()
    echo = synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=7)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    geom.upload_echo(echo)
    G = synth.random_image((1, w.grid.ny, w.grid.nx), seed=8).astype(np.complex64)
    grad = torch.empty((w.n_pings, 3), dtype=torch.float64, device="cuda")
    sas.sas_backproject_adjoint(geom.h, sas.grid_from(w.grid), sas.kaiser(BETA), torch.from_numpy(G).cuda(),
                                None, grad)
    geom.sync_status()
    tx, rx = oracle_positions(nav)
    ref = oracle.vjp_offsets(tx, rx, oracle_signal(w), echo, 8, BETA, grid_pixels(w.grid), G.reshape(-1))
    assert oracle.rel_l2(grad.cpu().numpy(), ref) < 1e-3
    geom.close()


def test_offset_gradient_of_sharpness_central_differences():
    """dS/d(dp) from the adjoint kernel against central differences of S
    computed with the GPU forward pass, along random directions."""
    from paper_2101_05888_gb300 import autofocus as af

    w, nav = _grad_case(P=16, C=4, n=64)
    scat = np.array([[w.grid.x0 + 20 * w.grid.dx, w.grid.y0 + 30 * w.grid.dy, 0.0, 0.9, 0.3],
                     [w.grid.x0 + 40 * w.grid.dx, w.grid.y0 + 21 * w.grid.dy, 0.0, -0.5, 0.6]])
    echo = point_echo(w, nav, scat, noise=True).astype(np.complex64)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    geom.upload_echo(echo)
    grid, interp = sas.grid_from(w.grid), sas.kaiser(BETA)
    dp0 = torch.from_numpy(np.random.default_rng(9).normal(0, 0.002, (w.n_pings, 3))).cuda()
    _, grad = af.offset_gradient(geom, grid, interp, dp0)
    rng = np.random.default_rng(10)
    # Richardson-extrapolated central difference: truncation O((k h)^4) with
    # k = 4 pi / lambda, so a step large enough to keep the FP32 rounding noise
    # of the GPU sharpness small
    h = 2e-4
    an, fd = [], []

    def S(x):
        return af.offset_gradient(geom, grid, interp, x)[0][0].item()

    for _ in range(6):
        v = torch.from_numpy(rng.normal(size=(w.n_pings, 3))).cuda()
        v /= torch.linalg.norm(v)
        d1 = (S(dp0 + h * v) - S(dp0 - h * v)) / (2 * h)
        d2 = (S(dp0 + 2 * h * v) - S(dp0 - 2 * h * v)) / (4 * h)
        fd.append((4 * d1 - d2) / 3)
        an.append(float((grad * v).sum().item()))
    geom.sync_status()
    err = oracle.rel_l2(np.array(an), np.array(fd))
    print("offset gradient vs Richardson central differences of the GPU sharpness: %.3g" % err)
    assert err < 1e-3
    geom.close()


def test_offset_gradient_vs_fp64_central_differences():
    """dS/d(dp) from the GPU (forward image, sharpness gradient, offset VJP)
    along random directions against Richardson-extrapolated central
    differences of the sharpness the FP64 oracle computes from its own
    backprojection with the offsets applied (Sec. II-D: the motion is
    estimated from the data by this gradient).  FP64 differences leave
    truncation O((k h)^4), k = 4 pi / lambda, and no rounding noise."""
    from paper_2101_05888_gb300 import autofocus as af

    w, nav = _grad_case(P=16, C=4, n=64)
    scat = np.array([[w.grid.x0 + 20 * w.grid.dx, w.grid.y0 + 30 * w.grid.dy, 0.0, 0.9, 0.3],
                     [w.grid.x0 + 40 * w.grid.dx, w.grid.y0 + 21 * w.grid.dy, 0.0, -0.5, 0.6]])
    echo = point_echo(w, nav, scat, noise=True).astype(np.complex64)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    geom.upload_echo(echo)
    grid, interp = sas.grid_from(w.grid), sas.kaiser(BETA)
    dp0 = np.random.default_rng(9).normal(0, 0.002, (w.n_pings, 3))
    _, grad = af.offset_gradient(geom, grid, interp, torch.from_numpy(dp0).cuda())
    geom.sync_status()
    grad = grad.cpu().numpy()
    geom.close()
    sig, pix = oracle_signal(w), grid_pixels(w.grid)

    def S(dp):
        tx, rx = oracle_positions(nav, offsets=dp)
        return oracle.sharpness(oracle.backproject(tx, rx, sig, echo, 8, BETA, pix))[0]

    rng = np.random.default_rng(10)
    h = 1e-5
    an, fd = [], []
    for _ in range(6):
        v = rng.normal(size=(w.n_pings, 3))
        v /= np.linalg.norm(v)
        d1 = (S(dp0 + h * v) - S(dp0 - h * v)) / (2 * h)
        d2 = (S(dp0 + 2 * h * v) - S(dp0 - 2 * h * v)) / (4 * h)
        fd.append((4 * d1 - d2) / 3)
        an.append(float((grad * v).sum()))
    err = oracle.rel_l2(np.array(an), np.array(fd))
    print("GPU offset gradient vs FP64 central differences of the oracle's sharpness: %.3g" % err)
    assert err < 1e-3


def test_autograd_function_backward():
    """torch autograd through BackprojectOffsets for L = sum |I|^2 equals the
    oracle's gradient with dL/dI* = I."""
    from paper_2101_05888_gb300 import autofocus as af

    w, nav = _grad_case(P=12, C=2, n=48)
    echo = synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=11)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    geom.upload_echo(echo)
    dp = torch.zeros((w.n_pings, 3), dtype=torch.float64, device="cuda", requires_grad=True)
    img = af.backproject_offsets(dp, geom, sas.grid_from(w.grid), sas.kaiser(BETA))
    loss = (img.abs() ** 2).sum()
    loss.backward()
    tx, rx = oracle_positions(nav)
    pix = grid_pixels(w.grid)
    I = oracle.backproject(tx, rx, oracle_signal(w), echo, 8, BETA, pix)
    ref = oracle.vjp_offsets(tx, rx, oracle_signal(w), echo, 8, BETA, pix, I)
    assert oracle.rel_l2(dp.grad.cpu().numpy(), ref) < 1e-3
    geom.close()


def test_autofocus_full_size():
    """Autofocus workload: 1024 pings x 16 RX x 8192 samples, 2048^2 pixels at
    1.5 cm, navigation error N(0, 2 cm) per axis.  The offset gradient on a
    64^2 sub-grid matches the oracle, and 20 sharpness-ascent steps on the
    full image raise the sharpness."""
    from paper_2101_05888_gb300 import autofocus as af

    w = synth.workload("autofocus_2d")
    nav = synth.nav(w)
    scat = synth.scatterers(w)
    echo = point_echo(w, nav, scat, half_width=160).astype(np.complex64)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    geom.upload_echo(echo)
    interp = sas.kaiser(BETA)
    # gradient on a 64^2 sub-grid around the first scatterer vs the oracle
    ij = synth.scatterer_indices(w, scat)[0]
    g = w.grid
    sub = synth.Grid(g.x0 + (ij[0] - 32) * g.dx, g.y0 + (ij[1] - 32) * g.dy, 0.0, g.dx, g.dy, 0.0, 64, 64, 1)
    img = geom.backproject(sas.grid_from(sub), interp)
    out, G = af.sharpness_and_grad(img)
    grad = torch.empty((w.n_pings, 3), dtype=torch.float64, device="cuda")
    sas.sas_backproject_adjoint(geom.h, sas.grid_from(sub), interp, G, None, grad)
    geom.sync_status()
    tx, rx = oracle_positions(nav)
    ref = oracle.vjp_offsets(tx, rx, oracle_signal(w), echo, 8, BETA, grid_pixels(sub), G.cpu().numpy().reshape(-1))
    assert oracle.rel_l2(grad.cpu().numpy(), ref) < 1e-3
    # 20 ascent steps on the full image
    dp, hist = af.autofocus(geom, sas.grid_from(w.grid), steps=20, step_m=1e-3, interp=interp)
    geom.sync_status()
    print("autofocus sharpness:", " ".join("%.4g" % s for s in hist))
    assert len(hist) == 21 and all(b >= a for a, b in zip(hist, hist[1:]))
    assert hist[-1] > 2.0 * hist[0]
    geom.close()
