"""The checked build: the library compiled with -DSAS_CHECKED, in which the
backprojection and adjoint kernels record a Farrow-row index that left the
window the host sized for its tile (status bit, SAS_ERR_CHECK from
sas_sync_status) instead of only clamping it.  It stands in for a memory
checker: the parity cases of the forward, adjoint, beam, motion, refraction
and 3D-volume paths run against it in a child process, and every launch must
leave the status word clear (each handle's status is read before it is
destroyed)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PARITY = ["test_gpu_forward.py", "test_gpu_adjoint.py", "test_gpu_beam.py", "test_gpu_motion.py",
          "test_gpu_refraction.py", "test_gpu_volume.py"]


def test_checked_build_parity_cases_leave_status_clear():
    from paper_2101_05888_gb300 import build
    path = build.build(checked=True)
    assert os.path.exists(path)
    env = dict(os.environ, SAS_CHECKED="1")
    flags = subprocess.run([sys.executable, "-c", "import paper_2101_05888_gb300 as s; print(s.sas_build_flags())"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert flags.returncode == 0, flags.stderr
    assert flags.stdout.strip() == "1"          # the checked library is the one loaded
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu", "-p", "no:cacheprovider",
                        *[os.path.join("tests", f) for f in PARITY]],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    print(r.stdout[-3000:])
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
