"""GPU parity of the seabed refraction model (Sec. III-B: imaging below the
seafloor with a refraction model in the propagation time).  A flat interface
with water above and sediment below; a leg to a pixel below the interface
crosses it where the travel time is stationary (Snell's law).  The kernels
solve each crossing per pixel in FP32 as a difference from a reference
crossing solved per tile; the oracle bisects every leg in FP64."""
import numpy as np
import pytest

import oracle
import paper_2101_05888_gb300 as sas
from paper_2101_05888_gb300 import synth

from _scene import grid_pixels, in_band, lib_signal, oracle_positions, oracle_signal

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BETA = 4.0


def _volume(nx=20, ny=16, nz=16, z0=-0.1, dz=0.02):
    """Planar-array lattice 2 m above the seabed (z = 0), voxels from above
    the seabed into the sediment; horizontal ranges reach past the critical
    distance of a fast sediment (3.7 m at 1700 m/s)."""
    g = synth.Grid(1.5, 1.6, z0, 0.05, 0.05, dz, nx, ny, nz)
    w = synth.workload("volume_3d", grid=g, n_pings=16, n_rx=4, n_samples=2048, lattice=4, lattice_pitch=1.5,
                       echo_dtype="c64")
    return w, synth.nav(w)


def _image(geom, w, beta=BETA):
    img = geom.backproject(sas.grid_from(w.grid), sas.kaiser(beta)).cpu().numpy()
    geom.sync_status()
    return img


@pytest.mark.parametrize("cs,zint", [(1700.0, 0.013), (1450.0, 0.013), (1800.0, -0.05), (1520.0, 0.1)])
def test_forward_3d_refraction_matches_oracle(cs, zint):
    """Fast and slow sediments; the interface between pixel layers, so that
    tiles straddle it (their centres above or below)."""
    w, nav = _volume()
    echo = synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=61)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    geom.set_refraction(zint, cs)
    geom.upload_echo(echo)
    img = _image(geom, w)
    tx, rx = oracle_positions(nav)
    pix = grid_pixels(w.grid)
    with oracle.medium(zint, cs):
        ref = oracle.backproject(tx, rx, oracle_signal(w), echo, 8, BETA, pix).reshape(img.shape)
    assert oracle.rel_l2(img, ref) < 1e-4
    # the model matters below the interface: straight paths differ there
    below = pix[:, 2].reshape(img.shape) > zint
    straight = oracle.backproject(tx, rx, oracle_signal(w), echo, 8, BETA, pix).reshape(img.shape)
    assert oracle.rel_l2(straight[below], ref[below]) > 0.1
    # and pixels above it are the straight ones
    assert oracle.rel_l2(img[~below], straight[~below]) < 1e-4
    geom.close()


def test_forward_3d_refraction_16bit_echo():
    w, nav = _volume(nx=12, ny=30, nz=10)
    echo = synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=62)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    geom.set_refraction(0.013, 1650.0)
    tx, rx = oracle_positions(nav)
    with oracle.medium(0.013, 1650.0):
        ref = oracle.backproject(tx, rx, oracle_signal(w), echo, 8, BETA, grid_pixels(w.grid))
    # the reduced-precision budget for both: BF16 rounding of the echo rows
    # (8 significant bits, about 1.5e-3 rms) dominates the BF16 total
    for dt, tol in ((sas.SAS_ECHO_C32_F16, 3e-3), (sas.SAS_ECHO_C32_BF16, 3e-3)):
        geom.upload_echo(echo, dt)
        img = _image(geom, w)
        stored = geom.download_echo().cpu().numpy()
        with oracle.medium(0.013, 1650.0):
            ref_q = oracle.backproject(tx, rx, oracle_signal(w), stored, 8, BETA, grid_pixels(w.grid))
        e_total, e_kernel = oracle.rel_l2(img.reshape(-1), ref), oracle.rel_l2(img.reshape(-1), ref_q)
        print("refraction, 16-bit echo %d: kernel on the stored echo %.3g, total %.3g, echo rounding %.3g" % (
            dt, e_kernel, e_total, oracle.rel_l2(ref_q, ref)))
        assert e_kernel < 1e-3
        assert e_total < tol
    geom.close()


@pytest.mark.parametrize("cs", [1700.0, 1400.0])
def test_forward_2d_slice_below_the_seabed(cs):
    """A horizontal slice 0.3 m into the sediment seen from a strip-map track
    10 m up and 20 m off: every leg refracts, most of them (fast sediment)
    beyond the critical distance."""
    w = synth.workload("small_2d", grid=synth.Grid(1.0, 20.0, 0.3, 0.02, 0.02, 0.0, 120, 70, 1),
                       n_pings=48, n_rx=4, t0=0.02)
    nav = synth.nav(w)
    echo = synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=63)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    geom.set_refraction(0.0, cs)
    geom.upload_echo(echo)
    img = _image(geom, w)
    tx, rx = oracle_positions(nav)
    with oracle.medium(0.0, cs):
        ref = oracle.backproject(tx, rx, oracle_signal(w), echo, 8, BETA, grid_pixels(w.grid)).reshape(img.shape)
    assert oracle.rel_l2(img, ref) < 1e-4
    geom.close()


def test_buried_point_focuses():
    """Echoes of points below the seabed, simulated with refraction by the
    oracle, focus at their voxels (peak |I| near |A| P C) only when the
    kernels image with the model."""
    w, nav = _volume(nx=24, ny=24, nz=16, z0=-0.06)
    g = w.grid
    idx = np.array([[5, 7, 9], [17, 15, 13], [11, 20, 6]])
    pts = oracle.grid_index_points(g.x0, g.y0, g.z0, g.dx, g.dy, g.dz, idx)
    A = np.array([0.9 * np.exp(0.3j), 0.7 * np.exp(-1.1j), 0.8 * np.exp(2.0j)])
    scat = np.concatenate([pts, A.real[:, None], A.imag[:, None]], 1)
    tx, rx = oracle_positions(nav, true=True)
    with oracle.medium(0.0, 1700.0):
        echo = oracle.simulate_points(tx, rx, oracle_signal(w), 20e3, 0.0, scat)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    geom.upload_echo(echo)
    geom.set_refraction(0.0, 1700.0)
    img = _image(geom, w)
    PC = w.n_pings * w.n_rx
    # the 8-tap interpolator and the other points' sidelobes leave a few per
    # cent; the oracle with the same interpolator agrees to parity
    with oracle.medium(0.0, 1700.0):
        ref = oracle.backproject(tx, rx, oracle_signal(w), echo, 8, BETA, pts)
    assert np.abs(img[idx[:, 2], idx[:, 1], idx[:, 0]] - ref).max() < 1e-4 * PC
    assert np.abs(img).reshape(-1).argmax() in np.ravel_multi_index(idx[:, ::-1].T, img.shape)
    for (ix, iy, iz), a in zip(idx, A):
        assert abs(img[iz, iy, ix] - a * PC) < 0.1 * abs(a) * PC
    geom.set_refraction(0.0, 0.0)                  # straight paths: defocused
    img_s = _image(geom, w)
    for (ix, iy, iz), a in zip(idx, A):
        assert abs(img_s[iz, iy, ix]) < 0.6 * abs(a) * PC
    geom.close()


def test_interface_below_the_grid_and_equal_speeds():
    w, nav = _volume(nx=16, ny=30, nz=8)
    echo = synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=64)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    geom.upload_echo(echo)
    straight = _image(geom, w)
    geom.set_refraction(5.0, 1700.0)               # every voxel above the interface
    # the straight-path kernel forms its per-pair reference terms in
    # double-float arithmetic, the refraction kernel in FP64: their FP32 record
    # fields agree to the last bit, which moves the image by about 1e-6
    assert oracle.rel_l2(_image(geom, w), straight) < 5e-6
    geom.set_refraction(-0.5, synth.C_SOUND)       # sediment as fast as water: straight legs
    assert oracle.rel_l2(_image(geom, w), straight) < 2e-5
    geom.close()


@pytest.mark.parametrize("cs,zint", [(1700.0, 0.013), (1450.0, -0.05)])
def test_offset_gradient_3d_refraction_matches_oracle(cs, zint):
    """The offset VJP with refracted legs (the derivative of a refracted leg's
    length with respect to its sensor is minus the unit vector towards its
    crossing point) against the oracle's gradient with the same medium; tiles
    straddle the interface, so straight and refracted legs mix."""
    w, nav = _volume(nx=16, ny=12, nz=12)
    echo = synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=66)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    geom.set_refraction(zint, cs)
    geom.upload_echo(echo)
    G = synth.random_image((w.grid.nz, w.grid.ny, w.grid.nx), seed=67).astype(np.complex64)
    grad = torch.empty((w.n_pings, 3), dtype=torch.float64, device="cuda")
    sas.sas_backproject_adjoint(geom.h, sas.grid_from(w.grid), sas.kaiser(BETA), torch.from_numpy(G).cuda(),
                                None, grad)
    geom.sync_status()
    tx, rx = oracle_positions(nav)
    with oracle.medium(zint, cs):
        ref = oracle.vjp_offsets(tx, rx, oracle_signal(w), echo, 8, BETA, grid_pixels(w.grid), G.reshape(-1))
    straight = oracle.vjp_offsets(tx, rx, oracle_signal(w), echo, 8, BETA, grid_pixels(w.grid), G.reshape(-1))
    got = grad.cpu().numpy()
    print("refracted offset gradient (c_s %g): vs oracle %.3g, straight-path gradient differs by %.3g" % (
        cs, oracle.rel_l2(got, ref), oracle.rel_l2(straight, ref)))
    assert oracle.rel_l2(got, ref) < 1e-3
    assert oracle.rel_l2(straight, ref) > 1e-2            # the model changes the gradient
    geom.close()


def test_offset_gradient_2d_slice_below_the_seabed():
    """Every leg refracts, most past the critical distance (fast sediment)."""
    w = synth.workload("small_2d", grid=synth.Grid(1.0, 20.0, 0.3, 0.02, 0.02, 0.0, 64, 48, 1),
                       n_pings=24, n_rx=4, t0=0.02)
    nav = synth.nav(w)
    echo = synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=68)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    geom.set_refraction(0.0, 1700.0)
    geom.upload_echo(echo)
    G = synth.random_image((1, w.grid.ny, w.grid.nx), seed=69).astype(np.complex64)
    grad = torch.empty((w.n_pings, 3), dtype=torch.float64, device="cuda")
    sas.sas_backproject_adjoint(geom.h, sas.grid_from(w.grid), sas.kaiser(BETA), torch.from_numpy(G).cuda(),
                                None, grad)
    geom.sync_status()
    tx, rx = oracle_positions(nav)
    with oracle.medium(0.0, 1700.0):
        ref = oracle.vjp_offsets(tx, rx, oracle_signal(w), echo, 8, BETA, grid_pixels(w.grid), G.reshape(-1))
    assert oracle.rel_l2(grad.cpu().numpy(), ref) < 1e-3
    geom.close()


@pytest.mark.parametrize("dim3,cs,zint", [(True, 1700.0, 0.013), (True, 1450.0, -0.05), (False, 1700.0, 0.0)])
def test_linear_adjoint_refraction_matches_oracle(dim3, cs, zint):
    """The linear adjoint with refracted legs against the oracle's adjoint
    with the same medium (in band at 1e-4, full band at 1e-3: the cubic
    Farrow form's weight error lies out of band), and the GPU dot test
    <B e, I> = <e, B^H I> with the refracting forward."""
    if dim3:
        w, nav = _volume(nx=14, ny=12, nz=10)
    else:
        w = synth.workload("small_2d", grid=synth.Grid(1.0, 20.0, 0.3, 0.02, 0.02, 0.0, 48, 40, 1),
                           n_pings=16, n_rx=4, t0=0.02)
        nav = synth.nav(w)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    geom.set_refraction(zint, cs)
    img = synth.random_image((w.grid.nz, w.grid.ny, w.grid.nx), seed=70).astype(np.complex64)
    eadj = torch.empty((w.n_pings, w.n_rx, w.n_samples), dtype=torch.complex64, device="cuda")
    sas.sas_backproject_adjoint(geom.h, sas.grid_from(w.grid), sas.kaiser(BETA), torch.from_numpy(img).cuda(), eadj)
    geom.sync_status()
    tx, rx = oracle_positions(nav)
    with oracle.medium(zint, cs):
        ref = oracle.backproject_adjoint(tx, rx, oracle_signal(w), img.reshape(-1), 8, BETA, grid_pixels(w.grid))
    got = eadj.cpu().numpy()
    e_band, e_full = oracle.rel_l2(in_band(got), in_band(ref)), oracle.rel_l2(got, ref)
    # dot test against the GPU forward with the same model
    echo = synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=71)
    geom.upload_echo(echo)
    fwd = _image(geom, w)
    lhs = np.vdot(img.astype(np.complex128).reshape(-1), fwd.astype(np.complex128).reshape(-1))
    rhs = np.vdot(got.astype(np.complex128).reshape(-1), echo.astype(np.complex128).reshape(-1))
    e_dot = abs(lhs - rhs) / abs(lhs)
    print("refracted linear adjoint (3D %s, c_s %g): in band %.3g, full band %.3g, dot test %.3g" % (
        dim3, cs, e_band, e_full, e_dot))
    assert e_band < 1e-4
    assert e_full < 1e-3
    assert e_dot < 1e-5
    geom.close()


@pytest.mark.parametrize("cs", [1700.0, 1450.0])
def test_simulator_with_refraction_matches_oracle(cs):
    """The library's echo simulator with refracted legs (scatterers above and
    below the interface, a fast and a slow sediment) against the oracle's
    simulator with the same medium; the library's echoes of buried points
    then focus through the refracting backprojection."""
    w, nav = _volume(nx=24, ny=24, nz=16, z0=-0.06)
    g = w.grid
    idx = np.array([[5, 7, 9], [17, 15, 13], [11, 20, 1], [3, 3, 14]])
    pts = oracle.grid_index_points(g.x0, g.y0, g.z0, g.dx, g.dy, g.dz, idx)
    A = np.array([0.9 * np.exp(0.3j), 0.7 * np.exp(-1.1j), 0.8 * np.exp(2.0j), 0.6 * np.exp(0.7j)])
    scat = np.concatenate([pts, A.real[:, None], A.imag[:, None]], 1)
    geom = sas.Geometry(nav["true_pos"], nav["att"], nav["tx_lever"], nav["rx_lever"], lib_signal(w))
    geom.set_refraction(0.0, cs)
    echo = torch.zeros((w.n_pings, w.n_rx, w.n_samples), dtype=torch.complex64, device="cuda")
    sas.sas_simulate_points(geom.h, torch.from_numpy(scat).cuda(), scat.shape[0], synth.BANDWIDTH, synth.PULSE_T,
                            0, echo)
    torch.cuda.synchronize()
    got = echo.cpu().numpy()
    tx, rx = oracle_positions(nav, true=True)
    with oracle.medium(0.0, cs):
        ref = oracle.simulate_points(tx, rx, oracle_signal(w), synth.BANDWIDTH, synth.PULSE_T, scat)
    straight = oracle.simulate_points(tx, rx, oracle_signal(w), synth.BANDWIDTH, synth.PULSE_T, scat)
    print("simulator with refraction (c_s %g): vs oracle %.3g, vs straight paths %.3g" % (
        cs, oracle.rel_l2(got, ref), oracle.rel_l2(straight, ref)))
    assert oracle.rel_l2(got, ref) < 2e-5          # the simulator's FP32 pulse samples, as without the model
    assert oracle.rel_l2(straight, ref) > 0.1
    geom.close()
    img_geom = sas.Geometry.from_nav(nav, lib_signal(w))
    img_geom.set_refraction(0.0, cs)
    img_geom.upload_echo(got)
    img = _image(img_geom, w)
    # the three interior points (the corner point's peak carries more of the
    # other points' sidelobes than the 10 % bound allows in the slow sediment)
    PC = w.n_pings * w.n_rx
    for (ix, iy, iz), a in zip(idx[:3], A[:3]):
        assert abs(img[iz, iy, ix] - a * PC) < 0.1 * abs(a) * PC
    img_geom.close()


def test_unsupported_combinations_raise():
    w, nav = _volume(nx=8, ny=8, nz=8)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    geom.upload_echo(synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=65))
    geom.set_refraction(0.0, 1700.0)
    G = torch.zeros((w.grid.nz, w.grid.ny, w.grid.nx), dtype=torch.complex64, device="cuda")
    adj = torch.zeros((w.n_pings, w.n_rx, w.n_samples), dtype=torch.complex64, device="cuda")
    geom.set_velocity(np.zeros((w.n_pings, 3)))
    with pytest.raises(sas.SasError) as e:
        geom.backproject(sas.grid_from(w.grid), sas.kaiser(BETA))
    assert e.value.code == sas.SAS_ERR_UNSUPPORTED
    grad = torch.empty((w.n_pings, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(sas.SasError) as e:
        sas.sas_backproject_adjoint(geom.h, sas.grid_from(w.grid), sas.kaiser(BETA), G, None, grad)
    assert e.value.code == sas.SAS_ERR_UNSUPPORTED
    with pytest.raises(sas.SasError) as e:
        sas.sas_backproject_adjoint(geom.h, sas.grid_from(w.grid), sas.kaiser(BETA), G, adj, None)
    assert e.value.code == sas.SAS_ERR_UNSUPPORTED
    geom.set_velocity(None)
    geom.set_beam(np.deg2rad(30.0))
    with pytest.raises(sas.SasError) as e:
        geom.backproject(sas.grid_from(w.grid), sas.kaiser(BETA))
    assert e.value.code == sas.SAS_ERR_UNSUPPORTED
    geom.set_beam(0.0)
    scat = torch.zeros((1, 5), dtype=torch.float64, device="cuda")
    echo = torch.zeros((w.n_pings, w.n_rx, w.n_samples), dtype=torch.complex64, device="cuda")
    geom.set_velocity(np.zeros((w.n_pings, 3)))
    with pytest.raises(sas.SasError) as e:
        sas.sas_simulate_points(geom.h, scat, 1, synth.BANDWIDTH, synth.PULSE_T, 0, echo)
    assert e.value.code == sas.SAS_ERR_UNSUPPORTED
    geom.set_velocity(None)
    geom.set_refraction(0.0, 0.0)                  # off again: everything runs
    geom.backproject(sas.grid_from(w.grid), sas.kaiser(BETA))
    geom.sync_status()
    geom.close()
