"""GPU parity of the conditioning kernels (Sec. II-E, Eqs. 9-12) and the
matched filter against the FP64 oracle: FP32 FFT paths within 1e-5
(relative L2), order statistics bit-exact (both sides select on the same
FP32 values), gains and maps within 1e-6."""
import numpy as np
import pytest

import oracle
from oracle import conditioning as cond
import paper_2101_05888_gb300 as sas
from paper_2101_05888_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _colored(rows, n, seed):
    rng = np.random.default_rng(seed)
    w = rng.normal(size=(rows, n + 4)) + 1j * rng.normal(size=(rows, n + 4))
    h = np.array([1.0, 0.7 - 0.2j, 0.3, -0.1j, 0.05])
    return np.stack([np.convolve(r, h, mode="valid") for r in w]).astype(np.complex64)


@pytest.mark.parametrize("rows,n,L", [(6, 1000, 200), (3, 16384, 200), (4, 777, 1), (2, 5000, 4096),
                                      (5, 3000, 100), (3, 7000, 500), (2, 9000, 1000), (2, 20000, 2000)])
def test_matched_filter_matches_oracle(rows, n, L):
    """Ragged row lengths, a one-tap replica and the largest replica."""
    rng = np.random.default_rng(n + L)
    raw = (rng.normal(size=(rows, n)) + 1j * rng.normal(size=(rows, n))).astype(np.complex64)
    rep = cond.lfm_replica(20e3, L / 40e3, 40e3).astype(np.complex64) if L > 1 else np.array([0.5 - 0.5j], np.complex64)
    out = torch.empty((rows, n), dtype=torch.complex64, device="cuda")
    sas.sas_matched_filter(torch.from_numpy(raw).cuda(), rows, n, torch.from_numpy(rep).cuda(), rep.size, out)
    torch.cuda.synchronize()
    ref = cond.matched_filter(raw, rep)
    assert oracle.rel_l2(out.cpu().numpy(), ref) < 1e-5


def test_matched_filter_compresses_simulated_raw_echo():
    """Raw LFM echoes of the small-2D scene compress on the GPU to the same
    rows as the oracle's matched filter of the same raw data."""
    w = synth.scaled(synth.workload("small_2d"), n_pings=4, n_rx=2, n_samples=2048)
    nav = synth.nav(w)
    tx, rx = oracle.sensor_positions(nav["true_pos"], nav["att"], nav["tx_lever"], nav["rx_lever"])
    sig = oracle.Signal(synth.FC, synth.FS, synth.C_SOUND, w.t0, w.n_samples)
    scat = synth.scatterers(w)[:4]
    raw = cond.simulate_raw_points(tx, rx, sig, synth.BANDWIDTH, synth.PULSE_T, scat).reshape(-1, w.n_samples)
    rep = cond.lfm_replica(synth.BANDWIDTH, synth.PULSE_T, synth.FS)
    out = torch.empty(raw.shape, dtype=torch.complex64, device="cuda")
    sas.sas_matched_filter(torch.from_numpy(raw.astype(np.complex64)).cuda(), raw.shape[0], raw.shape[1],
                           torch.from_numpy(rep.astype(np.complex64)).cuda(), rep.size, out)
    torch.cuda.synchronize()
    ref = cond.matched_filter(raw.astype(np.complex64), rep.astype(np.complex64))
    assert oracle.rel_l2(out.cpu().numpy(), ref) < 1e-5
    assert np.abs(ref).max() > 0.5          # the scatterers compressed to peaks


@pytest.mark.parametrize("rows,n,gamma", [(40, 256, 0.0), (64, 1024, 0.1), (9, 16384, 0.05), (1, 8, 1.0),
                                            (7, 2048, 0.1), (3, 4096, 0.0), (5, 8192, 0.2), (17, 512, 0.3)])
def test_whitening_matches_oracle(rows, n, gamma):
    e = _colored(rows, n, n + rows)
    d_in = torch.from_numpy(e).cuda()
    out = torch.empty_like(d_in)
    gain = torch.empty(n, dtype=torch.float32, device="cuda")
    sas.sas_whiten(d_in, out, rows, n, gamma, gain)
    torch.cuda.synchronize()
    ref, Gh = cond.whiten(e, gamma)
    assert oracle.rel_l2(out.cpu().numpy(), ref) < 1e-5
    # FP32 spectra: the gain sqrt(G / max G) of Eq. 9 carries the spectrum's
    # rounding (about 2^-24 sqrt(log2 n) of the rms bin) amplified by
    # sqrt(kappa), kappa = mean P / (gamma mean P + min P) = mean(1 / Gh) / (1 + gamma)
    kappa = np.mean(1.0 / Gh) / (1.0 + gamma)
    tol = max(1e-6, 2.0 ** -23 * np.sqrt(np.log2(n) * kappa))
    assert np.abs(gain.cpu().numpy() - np.sqrt(Gh)).max() < tol
    assert gain.max().item() == 1.0
    # in place
    sas.sas_whiten(d_in, d_in, rows, n, gamma)
    torch.cuda.synchronize()
    assert oracle.rel_l2(d_in.cpu().numpy(), ref) < 1e-5


def test_whitening_output_not_16_byte_aligned():
    """An output that starts 8 bytes past a 16-byte boundary (a complex64 view
    one element in) takes the 8-byte-load path of the power sums."""
    rows, n, gamma = 6, 2048, 0.1
    e = _colored(rows, n, 77)
    store = torch.empty(rows * n + 1, dtype=torch.complex64, device="cuda")
    out = store[1:].view(rows, n)
    assert out.data_ptr() % 16 == 8
    sas.sas_whiten(torch.from_numpy(e).cuda(), out, rows, n, gamma)
    torch.cuda.synchronize()
    ref, _ = cond.whiten(e, gamma)
    assert oracle.rel_l2(out.cpu().numpy(), ref) < 1e-5


@pytest.mark.parametrize("rows,n", [(20000, 37), (65537, 24)])
def test_tvg_bracketed_select_matches_oracle(rows, n):
    """Row counts that take the bracketed select (a sample's bracket, one
    collecting pass, a select among the collected values), with columns that
    force the exact fallback: a constant column (every value inside the
    bracket: the collection overflows), a column whose lower half is one value
    (the bracket's lower end ties with half the column) and zeros; medians
    exact, gains and output as for the direct select."""
    rng = np.random.default_rng(rows + n)
    env = np.exp(-np.linspace(0, 4, n))
    e = ((rng.normal(size=(rows, n)) + 1j * rng.normal(size=(rows, n))) * env).astype(np.complex64)
    e[:, 3] = 0.5 - 0.25j                                   # constant column
    e[: rows // 2 + 1, 5] = 0.3                             # a tie across the lower half and the median
    e[:7, 0] = 0.0
    d_in = torch.from_numpy(e).cuda()
    out = torch.empty_like(d_in)
    gain = torch.empty(n, dtype=torch.float32, device="cuda")
    med = torch.empty(n, dtype=torch.float64, device="cuda")
    sas.sas_tvg(d_in, out, rows, n, 0.2, gain, med)
    torch.cuda.synchronize()
    ref, G, Pmed = cond.tvg(e, 0.2)
    assert np.array_equal(med.cpu().numpy(), Pmed)            # exact selection
    assert np.abs(gain.cpu().numpy() - np.sqrt(G)).max() <= 1e-6 * np.sqrt(G).max()
    assert oracle.rel_l2(out.cpu().numpy(), ref) < 1e-6


@pytest.mark.parametrize("rows,n,alpha", [(41, 300, 0.0), (64, 333, 0.25), (1, 40, 0.1), (2, 65, 0.0),
                                            (700, 50, 0.2), (300, 17, 0.0)])
def test_tvg_matches_oracle(rows, n, alpha):
    rng = np.random.default_rng(rows * n)
    env = np.exp(-np.linspace(0, 4, n))
    e = ((rng.normal(size=(rows, n)) + 1j * rng.normal(size=(rows, n))) * env).astype(np.complex64)
    e[0, :7] = 0.0                         # ties and zeros in the selection
    e[1 % rows, 3:9] = e[0, 3:9]
    d_in = torch.from_numpy(e).cuda()
    out = torch.empty_like(d_in)
    gain = torch.empty(n, dtype=torch.float32, device="cuda")
    med = torch.empty(n, dtype=torch.float64, device="cuda")
    sas.sas_tvg(d_in, out, rows, n, alpha, gain, med)
    torch.cuda.synchronize()
    ref, G, Pmed = cond.tvg(e, alpha)
    assert np.array_equal(med.cpu().numpy(), Pmed)            # exact selection
    assert np.abs(gain.cpu().numpy() - np.sqrt(G)).max() <= 1e-6 * np.sqrt(G).max()
    assert oracle.rel_l2(out.cpu().numpy(), ref) < 1e-6


@pytest.mark.parametrize("shape,b", [((63, 63), 0.35), ((64, 64), 0.2), ((1, 1), 0.5), ((1000, 999), 0.3)])
def test_drc_matches_oracle(shape, b):
    rng = np.random.default_rng(shape[0])
    img = (rng.standard_exponential(shape) ** 3 * np.exp(1j * rng.uniform(0, 6.28, shape))).astype(np.complex64)
    if img.size > 4:
        img.reshape(-1)[:5] = img.reshape(-1)[5]          # ties at one value
    n = img.size
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    stats = torch.empty(3, dtype=torch.float64, device="cuda")
    sas.sas_drc(torch.from_numpy(img).cuda(), n, b, out, stats)
    torch.cuda.synchronize()
    ref, q, med = cond.drc(img, b)
    st = stats.cpu().numpy()
    assert st[1] == med and st[2] == float(cond.magnitude_f32(img).max())    # exact selection and maximum
    assert abs(st[0] - q) <= 1e-12 * abs(q)
    assert np.abs(out.cpu().numpy() - ref.reshape(-1)).max() < 1e-6


def test_drc_without_stats_output():
    """The scratch-held statistics path (no d_stats) gives the same image."""
    rng = np.random.default_rng(9)
    img = (rng.standard_exponential((257, 130)) * np.exp(1j * rng.uniform(0, 6.28, (257, 130)))).astype(np.complex64)
    out = torch.empty(img.size, dtype=torch.float32, device="cuda")
    sas.sas_drc(torch.from_numpy(img).cuda(), img.size, 0.3, out)
    torch.cuda.synchronize()
    ref, _, _ = cond.drc(img, 0.3)
    assert np.abs(out.cpu().numpy() - ref.reshape(-1)).max() < 1e-6


@pytest.mark.parametrize("kind", ["constant", "mostly_dark", "speckle_2M", "half_dark_even", "one_bin_8M"])
def test_drc_selection_edge_cases(kind):
    """The radix selection on the degenerate medians (all pixels at the
    maximum: the identity map; a dark median: every lit pixel to 1), on an even
    count whose two middle values differ, on a 2M-pixel speckle image that
    spans many blocks and 1/8-octave bins, and on 8M distinct magnitudes in
    one 1/8-octave bin (every pixel a level-3 candidate: the blocks' candidate
    buffers overflow into the list): median and maximum exact, map to 1e-6."""
    rng = np.random.default_rng(len(kind))
    if kind == "constant":
        img = np.full(1000, 0.3 - 0.4j, np.complex64)
    elif kind == "one_bin_8M":
        n = 1 << 23
        img = ((1.0 + 0.05 * rng.random(n)) * np.exp(1j * rng.uniform(0, 6.28, n))).astype(np.complex64)
    elif kind == "mostly_dark":
        img = np.zeros(4097, np.complex64)
        img[::3] = (rng.standard_normal(1366) + 1j).astype(np.complex64)
    elif kind == "half_dark_even":
        img = np.zeros(2 * 33333, np.complex64)
        img[33333:] = (1.0 + rng.standard_exponential(33333)).astype(np.complex64)
    else:
        n = 1 << 21
        img = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    out = torch.empty(img.size, dtype=torch.float32, device="cuda")
    stats = torch.empty(3, dtype=torch.float64, device="cuda")
    sas.sas_drc(torch.from_numpy(img).cuda(), img.size, 0.3, out, stats)
    torch.cuda.synchronize()
    ref, q, med = cond.drc(img, 0.3)
    st = stats.cpu().numpy()
    mag = cond.magnitude_f32(img)
    assert st[1] == med and st[2] == float(mag.max())
    assert st[0] == q or abs(st[0] - q) <= 1e-12 * abs(q)
    # the FP32 map's error is the rounding of I_n times the map's slope
    # q / ((q - 1) I_n + 1)^2, which exceeds 1 when the median is near the
    # maximum (one 1/8-octave bin: m > 0.9)
    In = mag.astype(np.float64).reshape(-1) / float(mag.max())
    slope = 1.0 if not np.isfinite(q) else float(np.abs(q / ((q - 1.0) * In + 1.0) ** 2).max())
    assert np.abs(out.cpu().numpy() - ref.reshape(-1)).max() < 1e-6 * max(1.0, slope)
