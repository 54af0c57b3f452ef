"""GPU parity of the full-size 3D volume (Sec. III-B: a layered volume imaged
voxel by voxel): 1024 pings on a 32 x 32 lattice, an 8 x 8 planar receive
array, 8192 samples stored as FP16 or BF16 complex, 1024^2 x 128 voxels at
2 cm, in the launch the benchmark times (8 x 28 x 8-voxel tiles, 64 channels,
1024 (ping, channel) pairs per tile and 32 per stage).

The FP64 oracle evaluates a sample of voxels one by one: 4096 random voxels
and the 64 voxels around a corner where eight tiles meet.  Tolerances: the
whole 16-bit path within 3e-3 of the 8-tap oracle on the unrounded echo (the
reduced-precision budget), the kernel arithmetic on the stored echo within
1e-3; the error against the 32-tap truth (beta = 10) is printed."""
import numpy as np
import pytest

import oracle
import paper_2101_05888_gb300 as sas
from paper_2101_05888_gb300 import synth

from _scene import index_pixels, lib_signal, oracle_positions, oracle_signal

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BETA = 4.0
TRUTH_BETA = 10.0


@pytest.fixture(scope="module")
def volume():
    w = synth.workload("volume_3d")
    g = w.grid
    assert (w.n_pings, w.n_rx, w.n_samples, g.nx, g.ny, g.nz) == (1024, 64, 8192, 1024, 1024, 128)
    nav = synth.nav(w)
    echo = synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=w.seed)
    # 4096 random voxels and the 4 x 4 x 4 block around the corner shared by
    # the tiles at (ix, iy, iz) = (8 * 61, 28 * 17, 8 * 9)
    rand = synth.random_pixel_indices(g, 4096, seed=21)
    cx, cy, cz = np.meshgrid(np.arange(8 * 61 - 2, 8 * 61 + 2), np.arange(28 * 17 - 2, 28 * 17 + 2),
                             np.arange(8 * 9 - 2, 8 * 9 + 2), indexing="ij")
    corner = np.stack([cx.reshape(-1), cy.reshape(-1), cz.reshape(-1)], 1)
    idx = np.concatenate([rand, corner])
    tx, rx = oracle_positions(nav)
    pts = index_pixels(g, idx)
    sig = oracle_signal(w)
    ref8 = oracle.backproject(tx, rx, sig, echo, 8, BETA, pts)
    truth = oracle.backproject(tx, rx, sig, echo, 32, TRUTH_BETA, pts)
    return dict(w=w, nav=nav, echo=echo, idx=idx, tx=tx, rx=rx, pts=pts, sig=sig, ref8=ref8, truth=truth,
                n_corner=len(corner))


@pytest.mark.parametrize("store", [sas.SAS_ECHO_C32_F16, sas.SAS_ECHO_C32_BF16])
def test_volume_3d_full_size_sampled(volume, store):
    v = volume
    w = v["w"]
    geom = sas.Geometry.from_nav(v["nav"], lib_signal(w))
    geom.upload_echo(v["echo"], store)
    img = geom.backproject(sas.grid_from(w.grid), sas.kaiser(BETA))
    geom.sync_status()
    idx = v["idx"]
    got = img[idx[:, 2], idx[:, 1], idx[:, 0]].cpu().numpy()
    del img
    stored = geom.download_echo().cpu().numpy()
    geom.close()
    ref_q = oracle.backproject(v["tx"], v["rx"], v["sig"], stored, 8, BETA, v["pts"])
    e_kernel = oracle.rel_l2(got, ref_q)
    e_total = oracle.rel_l2(got, v["ref8"])
    e_corner = oracle.rel_l2(got[-v["n_corner"]:], v["ref8"][-v["n_corner"]:])
    e_truth = oracle.rel_l2(got, v["truth"])
    e_truth_k = oracle.rel_l2(v["ref8"], v["truth"])
    name = {sas.SAS_ECHO_C32_F16: "FP16", sas.SAS_ECHO_C32_BF16: "BF16"}[store]
    print("volume_3d %s: kernel on the stored echo %.3g, vs 8-tap FP64 oracle %.3g (tile corner %.3g), "
          "vs 32-tap truth %.3g (8-tap FP64 itself %.3g)" % (name, e_kernel, e_total, e_corner, e_truth, e_truth_k))
    assert e_kernel < 1e-3
    assert e_total < 3e-3
    assert e_corner < 3e-3
