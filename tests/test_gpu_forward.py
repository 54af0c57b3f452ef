"""GPU parity of the forward backprojection against the FP64 oracle.

Every case runs the CUDA path through the C ABI (via the ctypes binding) and
the oracle on the same seeded inputs.  Tolerance for the FP32 path: relative
complex L2 <= 1e-4 against the oracle with the same 8-tap interpolator."""
import numpy as np
import pytest

import oracle
import paper_2101_05888_gb300 as sas
from paper_2101_05888_gb300 import synth

from _scene import grid_pixels, image_at, index_pixels, lib_signal, oracle_positions, oracle_signal, point_echo

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-4
BETA = 4.0


def _run(geom, w_grid, echo, store=sas.SAS_ECHO_C64, interp=None, accumulate=False, image=None):
    geom.upload_echo(echo, store)
    img = geom.backproject(sas.grid_from(w_grid), interp or sas.kaiser(BETA), image=image, accumulate=accumulate)
    geom.sync_status()
    return img.cpu().numpy()


def test_geometry_positions_match_oracle():
    w = synth.scaled(synth.workload("stripmap_2d"), n_pings=300, n_rx=5, n_samples=1024)
    nav = synth.nav(w)
    nav["att"] = np.random.default_rng(5).uniform(-0.3, 0.3, size=nav["att"].shape)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    tx, rx = geom.positions()
    otx, orx = oracle_positions(nav)
    assert np.abs(tx.cpu().numpy() - otx).max() < 1e-12
    assert np.abs(rx.cpu().numpy() - orx).max() < 1e-12
    off = np.random.default_rng(6).normal(0, 0.01, size=(w.n_pings, 3))
    geom.set_offsets(off)
    tx, rx = geom.positions()
    otx, orx = oracle_positions(nav, offsets=off)
    assert np.abs(rx.cpu().numpy() - orx).max() < 1e-12
    geom.close()


@pytest.mark.parametrize("beta,bound", [(4.0, 4.3e-4), (6.0, 4.4e-4)])
def test_interpolator_farrow_form_matches_definition(beta, bound):
    """The Farrow form (a cubic on each half of the sample interval, Chebyshev
    interpolation at 4 nodes per half) against the definition; bound = the
    weight error of that construction with FP32 coefficients (4.18e-4 at
    beta 4, 4.26e-4 at beta 6) plus FP32 rounding.  On echoes sampled at twice
    their band (|nu| <= 1/4, the workloads' band) the interpolated value is
    within 5e-5 rms of the definition's: the weight error is concentrated
    where such signals have no energy."""
    rng = np.random.default_rng(1)
    f = rng.random(4000).astype(np.float32)
    taps = torch.empty((4000, 8), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.float64, device="cuda")
    sas.sas_interp_eval(sas.kaiser(beta), torch.from_numpy(f).cuda(), 4000, taps, err)
    ref = np.stack([oracle.kaiser_sinc_weights(float(x), 8, beta) for x in f])
    got = taps.cpu().numpy().astype(np.float64)
    assert np.abs(got - ref).max() < bound
    assert float(err.item()) < bound
    row = synth.bandlimited_noise((1, 8192), synth.NU_BAND, 1.0, 5)[0]
    i0 = rng.integers(8, 8192 - 8, 4000)
    win = np.stack([row[i - 3:i + 5] for i in i0])
    s_ref, s_got = (ref * win).sum(1), (got * win).sum(1)
    band_err = np.linalg.norm(s_got - s_ref) / np.linalg.norm(s_ref)
    print("Farrow form, beta %g: max weight error %.3g, band-limited value error %.3g rms" % (
        beta, np.abs(got - ref).max(), band_err))
    assert band_err < 5e-5


@pytest.mark.parametrize("beta,bound", [(4.0, 4.9e-3), (6.0, 4.87e-3)])
def test_interpolator_quadratic_form_matches_definition(beta, bound):
    """The quadratic Farrow form the 16-bit forward pass applies (Chebyshev
    interpolation at 3 nodes per half) against the definition; bound = the
    weight error of that construction (4.895e-3 at beta 4, 4.862e-3 at beta
    6, FP64 fit) plus FP32 rounding.  On echoes band-limited to |nu| <= 1/4 the
    interpolated value is within 1e-3 rms of the definition's (7.5e-4 for this
    construction): the 16-bit path's budget is 3e-3."""
    rng = np.random.default_rng(2)
    f = rng.random(4000).astype(np.float32)
    taps = torch.empty((4000, 8), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.float64, device="cuda")
    sas.sas_interp_eval_form(sas.kaiser(beta), 2, torch.from_numpy(f).cuda(), 4000, taps, err)
    ref = np.stack([oracle.kaiser_sinc_weights(float(x), 8, beta) for x in f])
    got = taps.cpu().numpy().astype(np.float64)
    assert np.abs(got - ref).max() < bound
    assert float(err.item()) < bound
    # the cubic form is the other degree, and only 2 and 3 exist
    sas.sas_interp_eval_form(sas.kaiser(beta), 3, torch.from_numpy(f).cuda(), 4000, taps, err)
    assert np.abs(taps.cpu().numpy().astype(np.float64) - ref).max() < 4.5e-4
    with pytest.raises(sas.SasError):
        sas.sas_interp_eval_form(sas.kaiser(beta), 4, torch.from_numpy(f).cuda(), 4000, taps, err)
    row = synth.bandlimited_noise((1, 8192), synth.NU_BAND, 1.0, 6)[0]
    i0 = rng.integers(8, 8192 - 8, 4000)
    win = np.stack([row[i - 3:i + 5] for i in i0])
    s_ref, s_got = (ref * win).sum(1), (got * win).sum(1)
    band_err = np.linalg.norm(s_got - s_ref) / np.linalg.norm(s_ref)
    print("quadratic Farrow form, beta %g: max weight error %.3g, band-limited value error %.3g rms" % (
        beta, np.abs(got - ref).max(), band_err))
    assert band_err < 1e-3


def test_small_2d_full_image():
    """128 pings x 4 RX x 2048 samples, 256^2 pixels at 2 cm, 10 points at 20 dB."""
    w = synth.workload("small_2d")
    nav = synth.nav(w)
    scat = synth.scatterers(w)
    echo = point_echo(w, nav, scat)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    img = _run(geom, w.grid, echo.astype(np.complex64))
    tx, rx = oracle_positions(nav)
    ref = oracle.backproject(tx, rx, oracle_signal(w), echo.astype(np.complex64), 8, BETA,
                             grid_pixels(w.grid)).reshape(img.shape)
    assert oracle.rel_l2(img, ref) < TOL_FP32
    # the image focuses: the brightest pixel is one of the scatterers
    ij = synth.scatterer_indices(w, scat)
    iy, ix = np.unravel_index(np.argmax(np.abs(img[0])), img.shape[1:])
    assert any((ix == a and iy == b) for a, b, _ in ij)
    geom.close()


def _ragged_workload():
    return synth.scaled(synth.workload("small_2d"), n_pings=37, n_rx=3, nx=70, ny=45, n_samples=1024)


def test_ragged_sizes_edges_and_accumulate():
    """Grid not a multiple of the tile, pairs not a multiple of the stage or
    group size, rows whose tap windows run off both ends of the echo."""
    w = _ragged_workload()
    # put the grid across the start of the echo window: t0 at the middle of the scene
    g = w.grid
    w = synth.workload("small_2d", grid=g, n_pings=37, n_rx=3, n_samples=1024, t0=0.0305)
    nav = synth.nav(w)
    echo = synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=11)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    img = _run(geom, w.grid, echo)
    tx, rx = oracle_positions(nav)
    ref = oracle.backproject(tx, rx, oracle_signal(w), echo, 8, BETA, grid_pixels(w.grid)).reshape(img.shape)
    assert oracle.rel_l2(img, ref) < TOL_FP32
    assert (np.abs(ref) == 0).any()  # part of the grid lies before the echo window
    # accumulate adds onto the existing image
    t = torch.from_numpy(img).cuda()
    geom.backproject(sas.grid_from(w.grid), sas.kaiser(BETA), image=t, accumulate=True)
    geom.sync_status()
    assert oracle.rel_l2(t.cpu().numpy(), 2 * ref) < TOL_FP32
    geom.close()


def test_edge_window_start_and_end():
    """Scene straddling both ends of a short echo window."""
    base = synth.workload("small_2d")
    g = synth.Grid(base.grid.x0, 19.0, 0.0, 0.03, 0.03, 0.0, 64, 200, 1)
    w = synth.workload("small_2d", grid=g, n_pings=24, n_rx=2, n_samples=256, t0=0.0295)
    nav = synth.nav(w)
    echo = synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=12)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    img = _run(geom, w.grid, echo)
    tx, rx = oracle_positions(nav)
    ref = oracle.backproject(tx, rx, oracle_signal(w), echo, 8, BETA, grid_pixels(w.grid)).reshape(img.shape)
    assert oracle.rel_l2(img, ref) < TOL_FP32
    col = np.abs(ref[0]).mean(axis=1)        # near and far rows see only part of the window
    assert col[0] < 0.2 * col.max() and col[-1] < 0.2 * col.max()
    geom.close()


def test_one_cta_per_tile_path():
    """Enough tiles that every tile runs in a single CTA (no pair split)."""
    base = synth.workload("small_2d")
    g = synth.Grid(base.grid.x0 - 3.0, 18.0, 0.0, 0.015, 0.015, 0.0, 1024, 640, 1)
    w = synth.workload("small_2d", grid=g, n_pings=6, n_rx=2, n_samples=2048)
    nav = synth.nav(w)
    echo = synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=13)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    img = _run(geom, w.grid, echo)
    tx, rx = oracle_positions(nav)
    idx = synth.random_pixel_indices(w.grid, 3000, seed=14)
    ref = oracle.backproject(tx, rx, oracle_signal(w), echo, 8, BETA, index_pixels(w.grid, idx))
    assert oracle.rel_l2(image_at(img, idx), ref) < TOL_FP32
    geom.close()


def test_3d_small_volume():
    """4x4 ping lattice, 2x2 planar receiver array, ragged 36 x 20 x 11 voxels."""
    base = synth.workload("volume_3d")
    g = synth.Grid(0.5, 0.7, 0.0, 0.02, 0.02, 0.02, 36, 20, 11)
    w = synth.workload("volume_3d", grid=g, n_pings=16, n_rx=4, n_samples=2048, lattice=4,
                       lattice_pitch=0.4, echo_dtype="c64")
    assert base.lattice == 32
    nav = synth.nav(w)
    echo = synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=15)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    img = _run(geom, w.grid, echo)
    tx, rx = oracle_positions(nav)
    ref = oracle.backproject(tx, rx, oracle_signal(w), echo, 8, BETA, grid_pixels(w.grid)).reshape(img.shape)
    assert oracle.rel_l2(img, ref) < TOL_FP32
    geom.close()


@pytest.mark.parametrize("store", [sas.SAS_ECHO_C32_F16, sas.SAS_ECHO_C32_BF16])
def test_16bit_echo_storage(store):
    """16-bit storage: the kernel (quadratic Farrow form, FP32 rows and
    accumulation) applied to the stored echo matches the oracle on that echo to
    1e-3, and the whole path is within 3e-3 of the FP64 oracle on the unrounded
    echo."""
    w = synth.workload("small_2d")
    nav = synth.nav(w)
    scat = synth.scatterers(w)
    echo = point_echo(w, nav, scat).astype(np.complex64)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    img = _run(geom, w.grid, echo, store=store)
    stored = geom.download_echo().cpu().numpy()
    q = oracle.rel_l2(stored, echo)
    assert q < (2e-3 if store == sas.SAS_ECHO_C32_F16 else 8e-3)
    tx, rx = oracle_positions(nav)
    pix = grid_pixels(w.grid)
    ref_q = oracle.backproject(tx, rx, oracle_signal(w), stored, 8, BETA, pix).reshape(img.shape)
    ref = oracle.backproject(tx, rx, oracle_signal(w), echo, 8, BETA, pix).reshape(img.shape)
    e_kernel, e_total = oracle.rel_l2(img, ref_q), oracle.rel_l2(img, ref)
    print("16-bit echo (%d): kernel arithmetic %.3g, total vs FP64 on the unrounded echo %.3g" % (store, e_kernel, e_total))
    assert e_kernel < 1e-3      # the quadratic form's interpolation error
    assert e_total < 3e-3
    geom.close()


def test_stripmap_full_size_sampled():
    """Full-size 2D stripmap (2048 pings x 32 RX x 16384 samples, 4096^2 pixels
    at 1.5 cm, sway/heave/yaw motion), same launch as the benchmark; checked on
    a 16 x 16 patch straddling a tile corner and 240 random pixels."""
    w = synth.workload("stripmap_2d")
    nav = synth.nav(w)
    echo = synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=w.seed)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    geom.upload_echo(echo)
    img_t = geom.backproject(sas.grid_from(w.grid), sas.kaiser(BETA))
    geom.sync_status()
    px, py = np.meshgrid(np.arange(48, 64), np.arange(56, 72), indexing="xy")
    patch = np.stack([px.reshape(-1), py.reshape(-1), np.zeros(256, dtype=np.int64)], 1)
    rand = synth.random_pixel_indices(w.grid, 240, seed=3)
    rand[-4:] = [[0, 0, 0], [w.grid.nx - 1, 0, 0], [0, w.grid.ny - 1, 0], [w.grid.nx - 1, w.grid.ny - 1, 0]]
    idx = np.concatenate([patch, rand])
    got = img_t[idx[:, 2], idx[:, 1], idx[:, 0]].cpu().numpy()
    tx, rx = oracle_positions(nav)
    ref = oracle.backproject(tx, rx, oracle_signal(w), echo, 8, BETA, index_pixels(w.grid, idx))
    assert oracle.rel_l2(got, ref) < TOL_FP32
    geom.close()


def test_bounded_wait_reports_timeout():
    """Failure detection without a fault: starve the bulk copies so that the
    kernel's bounded waits run out; the status comes back as SAS_ERR_TIMEOUT
    and the handle keeps working afterwards."""
    w = synth.scaled(synth.workload("small_2d"), n_pings=8, n_rx=2, nx=64, ny=64)
    nav = synth.nav(w)
    echo = synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=16)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    geom.upload_echo(echo)
    sas.sas_debug_starve_copies(geom.h, 1, 100)
    geom.backproject(sas.grid_from(w.grid), sas.kaiser(BETA))
    with pytest.raises(sas.SasError) as e:
        geom.sync_status()
    assert e.value.code == sas.SAS_ERR_TIMEOUT
    sas.sas_debug_starve_copies(geom.h, 0, 0)
    img = geom.backproject(sas.grid_from(w.grid), sas.kaiser(BETA))
    geom.sync_status()
    tx, rx = oracle_positions(nav)
    ref = oracle.backproject(tx, rx, oracle_signal(w), echo, 8, BETA, grid_pixels(w.grid))
    assert oracle.rel_l2(img.cpu().numpy().reshape(-1), ref) < TOL_FP32
    geom.close()


def test_sharpness_matches_oracle():
    z = synth.random_image((300, 257), seed=17).astype(np.complex64)
    z[10, 20] = 40.0
    t = torch.from_numpy(z).cuda()
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    g = torch.empty_like(t)
    sas.sas_sharpness(t, z.size, out, g)
    (S, N, D), og = oracle.sharpness(z.astype(np.complex128), want_grad=True)
    o = out.cpu().numpy()
    assert abs(o[0] - S) <= 1e-12 * S and abs(o[1] - N) <= 1e-12 * N and abs(o[2] - D) <= 1e-12 * D
    assert oracle.rel_l2(g.cpu().numpy().reshape(-1), og) < 1e-6


def test_argument_and_state_errors():
    w = synth.scaled(synth.workload("small_2d"), n_pings=4, n_rx=2, nx=32, ny=32)
    geom = sas.Geometry.from_nav(synth.nav(w), lib_signal(w))
    img = torch.empty((1, 32, 32), dtype=torch.complex64, device="cuda")
    with pytest.raises(sas.SasError) as e:
        sas.sas_backproject_2d(geom.h, sas.grid_from(w.grid), sas.kaiser(), img)
    assert e.value.code == sas.SAS_ERR_STATE
    geom.upload_echo(synth.random_echo(4, 2, w.n_samples, seed=1))
    with pytest.raises(sas.SasError) as e:
        sas.sas_backproject_2d(geom.h, sas.grid_from(w.grid), sas.kaiser(6.0, taps=32), img)
    assert e.value.code == sas.SAS_ERR_UNSUPPORTED
    bad = sas.make_grid(0, 0, 0, 0.01, 0.01, 0.01, 32, 32, 2)
    with pytest.raises(sas.SasError) as e:
        sas.sas_backproject_2d(geom.h, bad, sas.kaiser(), img)
    assert e.value.code == sas.SAS_ERR_ARG
    geom.close()
