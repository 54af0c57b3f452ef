"""GPU parity of the DPC micronavigation kernels (Sec. II-D, Eqs. 3-8)
against the FP64 oracle: time-delay estimation (FP32 correlation sums:
same peak lag, delays to a small fraction of a sample / carrier cycle),
footprints and model delays (FP64: 1e-9 m, 1e-15 s), the Levenberg-Marquardt
solution of Eq. 8 (the same minimum as the oracle's solver), and the whole
chain on simulated seafloor echoes (the sway and heave velocities are
recovered)."""
import numpy as np
import pytest

import oracle
from oracle import micronav as mn
import paper_2101_05888_gb300 as sas

import _dpc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C_SOUND, FC, FS = 1500.0, 100e3, 40e3


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda()


class _Problem:
    """The device arrays of a sas_dpc_problem (kept alive with the struct)."""

    def __init__(self, pl, meas, z_dvl, lam1, lam2, huber=0.0, ps=None):
        P, C = pl.P, pl.rx_lever.shape[0]
        self.arrays = dict(p0=_dev(pl.p0), vx=_dev(pl.vx), att=_dev(pl.att), dt=_dev(pl.dt),
                           tx=_dev(pl.tx_lever), rx=_dev(pl.rx_lever), t=_dev(meas.t[:meas.t.size // ((P - 1) * (C - meas.shift))]),
                           delay=_dev(meas.delay), weight=_dev(meas.weight), z=_dev(z_dvl),
                           ps=_dev(np.zeros((meas.ping.size, 3)) if ps is None else ps))
        a = self.arrays
        K = a["t"].numel()
        self.pr = sas.sas_dpc_problem(P=P, C=C, shift=meas.shift, K=K, side=pl.side, c=C_SOUND, lambda1=lam1,
                                      lambda2=lam2, huber=huber, d_p0=a["p0"].data_ptr(), d_vx=a["vx"].data_ptr(),
                                      d_att=a["att"].data_ptr(), d_dt=a["dt"].data_ptr(),
                                      d_tx_lever=a["tx"].data_ptr(), d_rx_lever=a["rx"].data_ptr(),
                                      d_t=a["t"].data_ptr(), d_delay=a["delay"].data_ptr(),
                                      d_weight=a["weight"].data_ptr(), d_z_dvl=a["z"].data_ptr(),
                                      d_ps=a["ps"].data_ptr())


def _scene(P=12, K=8, seed=4):
    pl = _dpc.platform(P=P)
    vy, vz = _dpc.true_velocities(P, seed=seed)
    meas = _dpc.measurements(pl, K, 0.025, 0.05, 2)
    return pl, vy, vz, meas


def test_footprints_and_model_delays_match_oracle():
    pl, vy, vz, meas = _scene()
    P = pl.P
    vy0, vz0 = 0.3 * vy, -0.5 * vz                      # some prior
    prob = _Problem(pl, meas, mn.heave_positions(pl, vz), 0.0, 0.0)
    ps = torch.empty((meas.ping.size, 3), dtype=torch.float64, device="cuda")
    sas.sas_dpc_footprints(prob.pr, _dev(vy0), _dev(vz0), ps)
    ref_ps = mn.footprints(pl, vy0, vz0, meas, C_SOUND)
    assert np.abs(ps.cpu().numpy() - ref_ps).max() < 1e-9
    prob.arrays["ps"].copy_(ps)
    out = torch.empty(meas.ping.size, dtype=torch.float64, device="cuda")
    sas.sas_dpc_model_delays(prob.pr, _dev(vy), _dev(vz), out)
    ref = mn.model_delays(pl, vy, vz, meas, ref_ps, C_SOUND)
    assert np.abs(out.cpu().numpy() - ref).max() < 1e-15
    assert np.abs(ref).max() > 1e-6


@pytest.mark.parametrize("huber,chunk", [(0.0, 0), (2e-4, 0), (0.0, 8), (2e-4, 16)])
def test_solve_matches_oracle(huber, chunk):
    """chunk: rows of the banded solve's shared-memory chunks (0: 512, one
    chunk here; 8 and 16: the 32 unknowns cross 3 and 1 chunk boundaries)."""
    pl, vy, vz, meas = _scene(P=16, K=6, seed=9)
    P = pl.P
    ps = mn.footprints(pl, np.zeros(P), np.zeros(P), meas, C_SOUND)
    rng = np.random.default_rng(3)
    meas.delay = mn.model_delays(pl, vy, vz, meas, ps, C_SOUND) + rng.normal(0, 5e-8, meas.ping.size)
    if huber:
        bad = rng.choice(meas.delay.size, meas.delay.size // 30, replace=False)
        meas.delay[bad] += 4e-6
    meas.weight = rng.uniform(0.5, 1.0, meas.ping.size)
    z_dvl = mn.heave_positions(pl, vz) + rng.normal(0, 0.002, P)
    lam1, lam2 = 1e-3, 1e-2
    ry, rz, rloss = mn.solve(pl, np.zeros(P), np.zeros(P), meas, ps, C_SOUND, z_dvl, lam1, lam2, huber=huber)
    prob = _Problem(pl, meas, z_dvl, lam1, lam2, huber=huber, ps=ps)
    gy, gz = torch.zeros(P, dtype=torch.float64, device="cuda"), torch.zeros(P, dtype=torch.float64, device="cuda")
    sas.sas_debug_dpc_solve_chunk(chunk)
    try:
        loss, iters = sas.sas_dpc_solve(prob.pr, gy, gz, 200)
    finally:
        sas.sas_debug_dpc_solve_chunk(0)
    gy, gz = gy.cpu().numpy(), gz.cpu().numpy()
    assert iters > 0
    # the same minimum: loss to 1e-9 relative; velocities to 1e-6 m/s (of ~3e-2)
    # for squares; the Huber loss is flatter (outliers on its linear part: 5e-6)
    assert abs(loss - rloss) <= 1e-9 * rloss
    assert abs(mn.total_loss(pl, gy, gz, meas, ps, C_SOUND, z_dvl, lam1, lam2, huber) - loss) <= 1e-9 * loss
    tol = 5e-6 if huber else 1e-6
    assert np.abs(gy - ry).max() < tol and np.abs(gz - rz).max() < tol


def _speckle_echo(pl, vy, vz, Ns=2304, n_points=4000, seed=5):
    """Echoes of a seafloor speckle patch abeam of the track, simulated by the
    oracle with the receivers moving during reception (the DPC model)."""
    p = mn.positions(pl, vy, vz)
    tx, rx = oracle.sensor_positions(p, pl.att, pl.tx_lever, pl.rx_lever)
    vel = np.stack([pl.vx, vy, vz], 1)
    scat = _dpc.seafloor_points(n_points, -0.6, 1.4, 12.0, 42.0, seed=seed)
    sig = oracle.Signal(FC, FS, C_SOUND, 0.0, Ns)
    return oracle.simulate_points(tx, rx, sig, 20e3, 5e-3, scat, half_width=24, vel=vel), p


def test_delays_match_oracle():
    pl, vy, vz, meas = _scene(P=6, K=10)
    echo, p = _speckle_echo(pl, vy, vz)
    geom = sas.Geometry(p, pl.att, pl.tx_lever, pl.rx_lever, sas.make_signal(FC, FS, C_SOUND, 0.0, echo.shape[2]))
    geom.upload_echo(echo.astype(np.complex64))
    K, W, L = 10, 128, 8
    centres = np.round(np.linspace(0.025, 0.05, K) * FS).astype(np.int32)
    M = meas.ping.size
    co, fi, rh = (torch.empty(M, dtype=torch.float64, device="cuda") for _ in range(3))
    sas.sas_dpc_delays(geom.h, 2, _dev(centres, torch.int32), K, W, L, co, fi, rh)
    torch.cuda.synchronize()
    co, fi, rh = co.cpu().numpy(), fi.cpu().numpy(), rh.cpu().numpy()
    e32 = echo.astype(np.complex64).astype(np.complex128)
    checked = 0
    for m in range(M):
        i, c, k = meas.ping[m], meas.chan[m], m % K
        R = np.abs(mn.correlate(e32[i, c + 2], e32[i + 1, c], int(centres[k]), W, L))
        top = np.sort(R)[-2:]
        if top[1] < top[0] * (1 + 1e-4):
            continue                                    # near-tie of the peak lag: FP32 and FP64 may differ
        rc, rf, rr = mn.estimate_delay(e32[i, c + 2], e32[i + 1, c], int(centres[k]), W, L, FS, FC)
        assert abs(co[m] - rc) < 1e-4 / FS
        assert abs(((fi[m] - rf) * FC + 0.5) % 1.0 - 0.5) < 1e-4      # phase, modulo a cycle
        assert abs(rh[m] - rr) < 1e-5
        checked += 1
    assert checked > 0.9 * M
    # coherent DPC pairs
    assert np.median(rh) > 0.8
    geom.close()


@pytest.mark.parametrize("store", [sas.SAS_ECHO_C32_F16, sas.SAS_ECHO_C32_BF16])
def test_delays_16bit_storage_match_oracle(store):
    """The delay estimator on 16-bit echo storage (four-byte staging copies
    and the per-row scale in the kernel) against the oracle's estimator on the
    stored echo as the library decodes it (the same precision budget as on
    complex64: the kernel's arithmetic, not the rounding of the storage)."""
    pl, vy, vz, meas = _scene(P=6, K=10)
    echo, p = _speckle_echo(pl, vy, vz)
    geom = sas.Geometry(p, pl.att, pl.tx_lever, pl.rx_lever, sas.make_signal(FC, FS, C_SOUND, 0.0, echo.shape[2]))
    geom.upload_echo(echo.astype(np.complex64), store)
    stored = geom.download_echo().cpu().numpy().astype(np.complex128)
    assert oracle.rel_l2(stored, echo) < (2e-3 if store == sas.SAS_ECHO_C32_F16 else 8e-3)
    K, W, L = 10, 128, 8
    centres = np.round(np.linspace(0.025, 0.05, K) * FS).astype(np.int32)
    M = meas.ping.size
    co, fi, rh = (torch.empty(M, dtype=torch.float64, device="cuda") for _ in range(3))
    sas.sas_dpc_delays(geom.h, 2, _dev(centres, torch.int32), K, W, L, co, fi, rh)
    torch.cuda.synchronize()
    co, fi, rh = co.cpu().numpy(), fi.cpu().numpy(), rh.cpu().numpy()
    checked = 0
    for m in range(M):
        i, c, k = meas.ping[m], meas.chan[m], m % K
        R = np.abs(mn.correlate(stored[i, c + 2], stored[i + 1, c], int(centres[k]), W, L))
        top = np.sort(R)[-2:]
        if top[1] < top[0] * (1 + 1e-4):
            continue                                    # near-tie of the peak lag: FP32 and FP64 may differ
        rc, rf, rr = mn.estimate_delay(stored[i, c + 2], stored[i + 1, c], int(centres[k]), W, L, FS, FC)
        assert abs(co[m] - rc) < 1e-4 / FS
        assert abs(((fi[m] - rf) * FC + 0.5) % 1.0 - 0.5) < 1e-4
        assert abs(rh[m] - rr) < 1e-5
        checked += 1
    assert checked > 0.9 * M
    assert np.median(rh) > 0.8
    geom.close()


@pytest.mark.parametrize("W,L,edge", [(100, 3, False), (128, 15, False), (37, 0, False), (64, 8, True),
                                      (130, 8, True)])
def test_delay_shapes_match_oracle(W, L, edge):
    """Window lengths that are not a multiple of the 32-sample staging chunk,
    no lag search (L = 0) and the widest one (L = 15), windows that run past
    either end of the rows (zero there), and a last warp of measurements only
    partly filled (M = 5 x 6 x 10 = 300): rows where ping i + 1, receiver c
    repeats ping i, receiver c + 2, three samples later, under noise."""
    pl, vy, vz, _ = _scene(P=6, K=10)
    P, C, Ns, shift, K = 6, 8, 1024, 2, 10
    rng = np.random.default_rng(W + 10 * L)
    noise = lambda: rng.normal(size=Ns) + 1j * rng.normal(size=Ns)
    echo = np.zeros((P, C, Ns), complex)
    for c in range(C):
        echo[0, c] = noise()
    for i in range(1, P):
        for c in range(C):
            echo[i, c] = np.roll(echo[i - 1, c + shift], 3) * 0.9 + 0.3 * noise() if c + shift < C else noise()
    if edge:
        centres = np.concatenate([[5, Ns - 3], np.linspace(100, Ns - 100, K - 2)])
    else:
        centres = np.linspace(80, Ns - 80, K)
    centres = np.round(centres).astype(np.int32)
    p = mn.positions(pl, vy, vz)
    geom = sas.Geometry(p, pl.att, pl.tx_lever, pl.rx_lever, sas.make_signal(FC, FS, C_SOUND, 0.0, Ns))
    geom.upload_echo(echo.astype(np.complex64))
    nc = C - shift
    M = (P - 1) * nc * K
    co, fi, rh = (torch.empty(M, dtype=torch.float64, device="cuda") for _ in range(3))
    sas.sas_dpc_delays(geom.h, shift, _dev(centres, torch.int32), K, W, L, co, fi, rh)
    torch.cuda.synchronize()
    co, fi, rh = co.cpu().numpy(), fi.cpu().numpy(), rh.cpu().numpy()
    e32 = echo.astype(np.complex64).astype(np.complex128)
    checked = 0
    for m in range(M):
        i, c, k = m // (nc * K), (m // K) % nc, m % K
        R = np.abs(mn.correlate(e32[i, c + shift], e32[i + 1, c], int(centres[k]), W, L))
        top = np.sort(R)[-2:]
        if L > 0 and top[1] < top[0] * (1 + 1e-4):
            continue                                    # near-tie of the peak lag: FP32 and FP64 may differ
        rc, rf, rr = mn.estimate_delay(e32[i, c + shift], e32[i + 1, c], int(centres[k]), W, L, FS, FC)
        assert abs(co[m] - rc) < 1e-4 / FS
        assert abs(((fi[m] - rf) * FC + 0.5) % 1.0 - 0.5) < 1e-4
        assert abs(rh[m] - rr) < 1e-5
        checked += 1
    assert checked > 0.9 * M
    if L >= 3:
        assert np.median(co) == pytest.approx(3 / FS, abs=0.5 / FS)    # the planted three-sample delay
    geom.close()


def test_end_to_end_recovers_sway_and_heave():
    """Simulated speckle echoes -> GPU delays -> coarse solve -> unwrapped fine
    delays -> fine solve: the sway and heave velocities come back to a few
    mm/s (of up to 3 cm/s), far closer than the prior (zero)."""
    P, K, W, L = 12, 16, 128, 8
    pl, vy, vz, meas = _scene(P=P, K=K, seed=11)
    echo, p = _speckle_echo(pl, vy, vz)
    nav_p = mn.positions(pl, np.zeros(P), np.zeros(P))            # navigation prior: no sway / heave
    geom = sas.Geometry(nav_p, pl.att, pl.tx_lever, pl.rx_lever, sas.make_signal(FC, FS, C_SOUND, 0.0, echo.shape[2]))
    geom.upload_echo(echo.astype(np.complex64))
    centres = np.round(np.linspace(0.025, 0.05, K) * FS).astype(np.int32)
    meas.t = np.tile(centres / FS, (P - 1) * (pl.rx_lever.shape[0] - 2))
    M = meas.ping.size
    co, fi, rh = (torch.empty(M, dtype=torch.float64, device="cuda") for _ in range(3))
    sas.sas_dpc_delays(geom.h, 2, _dev(centres, torch.int32), K, W, L, co, fi, rh)
    z_dvl = mn.heave_positions(pl, vz) + np.random.default_rng(1).normal(0, 0.003, P)
    prob = _Problem(pl, meas, z_dvl, 1e-4, 1e-3)
    zero = torch.zeros(P, dtype=torch.float64, device="cuda")
    ps = prob.arrays["ps"]
    sas.sas_dpc_footprints(prob.pr, zero, zero, ps)
    prob.arrays["delay"].copy_(co)
    prob.arrays["weight"].copy_(rh)
    gy, gz = zero.clone(), zero.clone()
    sas.sas_dpc_solve(prob.pr, gy, gz, 100)
    ref = torch.empty(M, dtype=torch.float64, device="cuda")
    sas.sas_dpc_model_delays(prob.pr, gy, gz, ref)
    fine = fi.cpu().numpy()
    prob.arrays["delay"].copy_(_dev(mn.unwrap(fine, ref.cpu().numpy(), FC)))
    sas.sas_dpc_solve(prob.pr, gy, gz, 100)
    gy, gz = gy.cpu().numpy(), gz.cpu().numpy()
    err = np.hypot(gy - vy, gz - vz)
    prior = np.hypot(vy, vz)
    assert np.sqrt(np.mean(err ** 2)) < 0.1 * np.sqrt(np.mean(prior ** 2))
    geom.close()
