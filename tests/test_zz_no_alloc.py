"""The allocation-free sharpness entry point (sas_sharpness_static).

Some callers may not allocate GPU memory once they are running, e.g. a
vehicle-borne processor that reserves all of its memory at start-up, or a host
framework whose memory manager forbids cudaMalloc/cudaFree.  For them the
library offers sas_sharpness_static, which keeps its partial sums in a fixed
array inside the library.  This file checks it against sas_sharpness on two
calls in a row (a large image, then a smaller one that must not see the first
call's leftovers) and that oversized inputs are refused before any launch.
It is named to be collected last."""
import ctypes

import numpy as np
import pytest

import paper_2101_05888_gb300 as sas
from paper_2101_05888_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_N = 16384 * 4096


def _both(img):
    n = img.numel()
    L = sas.lib()
    out_a = torch.zeros(3, dtype=torch.float64, device="cuda")
    out_b = torch.zeros(3, dtype=torch.float64, device="cuda")
    g_a = torch.empty_like(img)
    g_b = torch.empty_like(img)
    st = torch.cuda.current_stream().cuda_stream
    assert L.sas_sharpness(img.data_ptr(), n, out_a.data_ptr(), g_a.data_ptr(), st) == sas.SAS_OK
    rc = L.sas_sharpness_static(img.data_ptr(), n, out_b.data_ptr(), g_b.data_ptr(), st)
    assert rc == sas.SAS_OK, sas.sas_last_error()
    torch.cuda.synchronize()
    return out_a.cpu().numpy(), out_b.cpu().numpy(), g_a.cpu().numpy(), g_b.cpu().numpy()


def test_static_scratch_matches_allocating_entry_point_twice():
    big = torch.from_numpy(synth.random_image((2100, 2500), seed=31).astype(np.complex64)).cuda()
    big[7, 9] = 50.0
    small = torch.from_numpy(synth.random_image((300, 233), seed=32).astype(np.complex64)).cuda()
    for img in (big, small):
        a, b, ga, gb = _both(img)
        assert np.all(np.abs(a - b) <= 1e-12 * np.abs(a))
        num = np.linalg.norm((ga - gb).reshape(-1))
        assert num <= 1e-6 * np.linalg.norm(ga.reshape(-1))


def test_static_scratch_refuses_oversized_input():
    img = torch.zeros(4, dtype=torch.complex64, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    L = sas.lib()
    rc = L.sas_sharpness_static(img.data_ptr(), MAX_N + 1, out.data_ptr(), None,
                                torch.cuda.current_stream().cuda_stream)
    assert rc == sas.SAS_ERR_ARG
    assert "limit" in sas.sas_last_error()
    assert L.sas_sharpness_static(None, 10, out.data_ptr(), None, None) == sas.SAS_ERR_ARG
