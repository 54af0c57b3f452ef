"""GB300-native time-domain backprojection (TDBP) for synthetic-aperture sonar.

The computation lives in ``libsas.so`` (CUDA, sm_103a) behind the C ABI of
``include/sas.h``.  This module is the thin Python binding: ctypes structures
mirroring the header, one function per C entry point with the same name
(argument marshalling and error checking only), and a small ``Geometry``
convenience class.  PyTorch supplies device memory and the current stream.

There is no CPU fallback: every call raises if the library is not built or no
CUDA device is present.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SAS_CHECKED=1 in the environment loads the checked build (index checks in
# the kernels report through sas_sync_status; build it with build(checked=True))
CHECKED = os.environ.get("SAS_CHECKED") == "1"
LIB_PATH = os.path.join(_HERE, "libsas_checked.so" if CHECKED else "libsas.so")

SAS_OK = 0
SAS_ERR_ARG = -1
SAS_ERR_CUDA = -2
SAS_ERR_OOM = -3
SAS_ERR_TIMEOUT = -4
SAS_ERR_UNSUPPORTED = -5
SAS_ERR_STATE = -6
SAS_ERR_CHECK = -7

SAS_ECHO_C64 = 0
SAS_ECHO_C32_F16 = 1
SAS_ECHO_C32_BF16 = 2

SAS_INTERP_KAISER_SINC = 0
SAS_INTERP_TABLE = 1

SAS_MLP_NPARAMS = 4808

ENTRY_POINTS = [
    "sas_version", "sas_last_error", "sas_geometry_create", "sas_geometry_set_offsets", "sas_geometry_set_beam",
    "sas_geometry_set_velocity", "sas_geometry_set_refraction",
    "sas_geometry_positions", "sas_geometry_destroy", "sas_echo_upload", "sas_echo_download",
    "sas_backproject_2d", "sas_backproject_3d", "sas_backproject_adjoint", "sas_sharpness",
    "sas_sharpness_static", "sas_simulate_points",
    "sas_interp_eval", "sas_interp_eval_form", "sas_mlp_make_windows", "sas_mlp_workspace_bytes", "sas_mlp_loss_grad",
    "sas_mlp_adam", "sas_interp_tabulate_mlp", "sas_sync_status", "sas_build_flags", "sas_cull_stats",
    "sas_matched_filter", "sas_whiten", "sas_tvg", "sas_drc",
    "sas_debug_starve_copies",
    "sas_dpc_delays", "sas_dpc_footprints", "sas_dpc_model_delays", "sas_dpc_solve", "sas_debug_dpc_solve_chunk",
]


class sas_signal(ctypes.Structure):
    _fields_ = [("fc", ctypes.c_double), ("fs", ctypes.c_double), ("c", ctypes.c_double),
                ("t0", ctypes.c_double), ("n_samples", ctypes.c_int32)]


class sas_nav(ctypes.Structure):
    _fields_ = [("n_pings", ctypes.c_int32), ("n_rx", ctypes.c_int32),
                ("ping_pos", ctypes.c_void_p), ("ping_att", ctypes.c_void_p),
                ("tx_lever", ctypes.c_void_p), ("rx_lever", ctypes.c_void_p)]


class sas_grid(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_double), ("y0", ctypes.c_double), ("z0", ctypes.c_double),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32)]


class sas_interp(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("taps", ctypes.c_int32), ("kaiser_beta", ctypes.c_double),
                ("table_n", ctypes.c_int32), ("d_table", ctypes.c_void_p)]


class sas_dpc_problem(ctypes.Structure):
    _fields_ = [("P", ctypes.c_int32), ("C", ctypes.c_int32), ("shift", ctypes.c_int32), ("K", ctypes.c_int32),
                ("side", ctypes.c_int32), ("c", ctypes.c_double), ("lambda1", ctypes.c_double),
                ("lambda2", ctypes.c_double), ("huber", ctypes.c_double),
                ("d_p0", ctypes.c_void_p), ("d_vx", ctypes.c_void_p), ("d_att", ctypes.c_void_p),
                ("d_dt", ctypes.c_void_p), ("d_tx_lever", ctypes.c_void_p), ("d_rx_lever", ctypes.c_void_p),
                ("d_t", ctypes.c_void_p), ("d_delay", ctypes.c_void_p), ("d_weight", ctypes.c_void_p),
                ("d_z_dvl", ctypes.c_void_p), ("d_ps", ctypes.c_void_p)]


class SasError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("libsas error %d: %s" % (code, msg))
        self.code = code


_lock = threading.Lock()
_lib = None


def lib():
    """Loads libsas.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libsas.so is not built (run __graft_entry__.build() or "
                                   "python paper_2101_05888_gb300/build.py)")
            L = ctypes.CDLL(LIB_PATH)
            V, I, I64, D, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_float
            P = ctypes.POINTER
            sig = {
                "sas_version": ([], I),
                "sas_last_error": ([], ctypes.c_char_p),
                "sas_geometry_create": ([P(sas_nav), P(sas_signal), V, P(V)], I),
                "sas_geometry_set_offsets": ([V, V, I, V], I),
                "sas_geometry_set_beam": ([V, D, I], I),
                "sas_geometry_set_velocity": ([V, V, I, V], I),
                "sas_geometry_set_refraction": ([V, D, D], I),
                "sas_geometry_positions": ([V, V, V, V], I),
                "sas_geometry_destroy": ([V], I),
                "sas_echo_upload": ([V, V, I, I, V], I),
                "sas_echo_download": ([V, V, V], I),
                "sas_backproject_2d": ([V, P(sas_grid), P(sas_interp), V, I, V], I),
                "sas_backproject_3d": ([V, P(sas_grid), P(sas_interp), V, I, V], I),
                "sas_backproject_adjoint": ([V, P(sas_grid), P(sas_interp), V, V, V, V], I),
                "sas_sharpness": ([V, I64, V, V, V], I),
                "sas_sharpness_static": ([V, I64, V, V, V], I),
                "sas_simulate_points": ([V, V, I64, D, D, ctypes.c_int32, V, V], I),
                "sas_interp_eval": ([P(sas_interp), V, I64, V, V, V], I),
                "sas_interp_eval_form": ([P(sas_interp), I, V, I64, V, V, V], I),
                "sas_mlp_make_windows": ([V, ctypes.c_int32, ctypes.c_int32, V, V, V, I64, D, D, V, V, V], I),
                "sas_mlp_workspace_bytes": ([I64], I64),
                "sas_mlp_loss_grad": ([V, V, V, V, I64, V, V, V, V], I),
                "sas_mlp_adam": ([V, V, V, V, ctypes.c_int32, F, F, F, F, V], I),
                "sas_interp_tabulate_mlp": ([V, ctypes.c_int32, D, V, V], I),
                "sas_sync_status": ([V, V], I),
                "sas_build_flags": ([], I),
                "sas_cull_stats": ([V, ctypes.POINTER(ctypes.c_longlong), I, V], I),
                "sas_matched_filter": ([V, I64, ctypes.c_int32, V, ctypes.c_int32, V, V], I),
                "sas_whiten": ([V, V, I64, ctypes.c_int32, D, V, V], I),
                "sas_tvg": ([V, V, I64, ctypes.c_int32, D, V, V, V], I),
                "sas_drc": ([V, I64, D, V, V, V], I),
                "sas_debug_starve_copies": ([V, I, ctypes.c_int32], I),
                "sas_debug_dpc_solve_chunk": ([ctypes.c_int32], I),
                "sas_dpc_delays": ([V, ctypes.c_int32, V, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, V, V, V,
                                    V], I),
                "sas_dpc_footprints": ([P(sas_dpc_problem), V, V, V, V], I),
                "sas_dpc_model_delays": ([P(sas_dpc_problem), V, V, V, V], I),
                "sas_dpc_solve": ([P(sas_dpc_problem), V, V, ctypes.c_int32, P(ctypes.c_double),
                                   P(ctypes.c_int32), V], I),
            }
            for name, (args, res) in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def _check(rc: int):
    if rc != SAS_OK:
        raise SasError(rc, lib().sas_last_error().decode(errors="replace"))
    return rc


def _ptr(x):
    """Device/host address of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        assert x.flags.c_contiguous
        return x.ctypes.data
    raise TypeError(type(x))


def _stream(stream=None):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch
    return torch.cuda.current_stream().cuda_stream


# ---------------------------------------------------------------------------
# One wrapper per C entry point (same names).

def sas_version() -> int:
    return lib().sas_version()


def sas_last_error() -> str:
    return lib().sas_last_error().decode(errors="replace")


def sas_geometry_create(nav: sas_nav, sig: sas_signal, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(lib().sas_geometry_create(ctypes.byref(nav), ctypes.byref(sig), _stream(stream), ctypes.byref(h)))
    return h.value


def sas_geometry_set_offsets(h, offsets, on_device: int, stream=None):
    _check(lib().sas_geometry_set_offsets(h, _ptr(offsets), on_device, _stream(stream)))


def sas_geometry_set_velocity(h, vel, on_device: int, stream=None):
    _check(lib().sas_geometry_set_velocity(h, _ptr(vel), on_device, _stream(stream)))


def sas_geometry_set_refraction(h, z_interface: float, c_sediment: float):
    _check(lib().sas_geometry_set_refraction(h, float(z_interface), float(c_sediment)))


def sas_geometry_set_beam(h, beam_width: float, side: int = 1):
    _check(lib().sas_geometry_set_beam(h, float(beam_width), int(side)))


def sas_geometry_positions(h, d_tx, d_rx, stream=None):
    _check(lib().sas_geometry_positions(h, _ptr(d_tx), _ptr(d_rx), _stream(stream)))


def sas_geometry_destroy(h):
    _check(lib().sas_geometry_destroy(h))


def sas_echo_upload(h, echo, on_device: int, store_dtype: int, stream=None):
    _check(lib().sas_echo_upload(h, _ptr(echo), on_device, store_dtype, _stream(stream)))


def sas_echo_download(h, d_out, stream=None):
    _check(lib().sas_echo_download(h, _ptr(d_out), _stream(stream)))


def sas_backproject_2d(h, grid: sas_grid, interp: sas_interp, d_image, accumulate: int = 0, stream=None):
    _check(lib().sas_backproject_2d(h, ctypes.byref(grid), ctypes.byref(interp), _ptr(d_image), accumulate,
                                    _stream(stream)))


def sas_backproject_3d(h, grid: sas_grid, interp: sas_interp, d_image, accumulate: int = 0, stream=None):
    _check(lib().sas_backproject_3d(h, ctypes.byref(grid), ctypes.byref(interp), _ptr(d_image), accumulate,
                                    _stream(stream)))


def sas_backproject_adjoint(h, grid: sas_grid, interp: sas_interp, d_grad_image, d_echo_adj=None,
                            d_grad_offsets=None, stream=None):
    _check(lib().sas_backproject_adjoint(h, ctypes.byref(grid), ctypes.byref(interp), _ptr(d_grad_image),
                                         _ptr(d_echo_adj), _ptr(d_grad_offsets), _stream(stream)))


def sas_sharpness(d_image, n: int, d_out3, d_grad=None, stream=None):
    _check(lib().sas_sharpness(_ptr(d_image), n, _ptr(d_out3), _ptr(d_grad), _stream(stream)))


def sas_sharpness_static(d_image, n: int, d_out3, d_grad=None, stream=None):
    """sas_sharpness without device allocation (built-in 64 KiB scratch,
    n <= 67,108,864; see include/sas.h)."""
    _check(lib().sas_sharpness_static(_ptr(d_image), n, _ptr(d_out3), _ptr(d_grad), _stream(stream)))


def sas_simulate_points(h, d_scat, n: int, bandwidth: float, pulse_T: float, half_width: int, d_echo,
                        stream=None):
    _check(lib().sas_simulate_points(h, _ptr(d_scat), n, bandwidth, pulse_T, half_width, _ptr(d_echo),
                                     _stream(stream)))


def sas_interp_eval(interp: sas_interp, d_f, n: int, d_taps, d_max_err=None, stream=None):
    _check(lib().sas_interp_eval(ctypes.byref(interp), _ptr(d_f), n, _ptr(d_taps), _ptr(d_max_err),
                                 _stream(stream)))


def sas_interp_eval_form(interp: sas_interp, degree: int, d_f, n: int, d_taps, d_max_err=None, stream=None):
    _check(lib().sas_interp_eval_form(ctypes.byref(interp), degree, _ptr(d_f), n, _ptr(d_taps), _ptr(d_max_err),
                                      _stream(stream)))


def sas_mlp_make_windows(d_echo, rows: int, n_samples: int, d_frac, d_row, d_pos, n: int, target_beta: float,
                         prior_beta: float, d_windows, d_targets, stream=None):
    _check(lib().sas_mlp_make_windows(_ptr(d_echo), rows, n_samples, _ptr(d_frac), _ptr(d_row), _ptr(d_pos), n,
                                      target_beta, prior_beta, _ptr(d_windows), _ptr(d_targets), _stream(stream)))


def sas_mlp_workspace_bytes(n: int) -> int:
    return lib().sas_mlp_workspace_bytes(n)


def sas_mlp_loss_grad(d_theta, d_frac, d_windows, d_targets, n: int, d_loss, d_grad, d_work, stream=None):
    _check(lib().sas_mlp_loss_grad(_ptr(d_theta), _ptr(d_frac), _ptr(d_windows), _ptr(d_targets), n,
                                   _ptr(d_loss), _ptr(d_grad), _ptr(d_work), _stream(stream)))


def sas_mlp_adam(d_theta, d_grad, d_m, d_v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().sas_mlp_adam(_ptr(d_theta), _ptr(d_grad), _ptr(d_m), _ptr(d_v), step, lr, beta1, beta2, eps,
                              _stream(stream)))


def sas_interp_tabulate_mlp(d_theta, table_n: int, prior_beta: float, d_table_out, stream=None):
    _check(lib().sas_interp_tabulate_mlp(_ptr(d_theta), table_n, prior_beta, _ptr(d_table_out), _stream(stream)))


def sas_sync_status(h, stream=None):
    _check(lib().sas_sync_status(h, _stream(stream)))


def sas_build_flags() -> int:
    return int(lib().sas_build_flags())


def sas_cull_stats(h, reset: int = 0, stream=None):
    """(candidate, computed, beam-edge) (ping, channel, tile) block counts."""
    out = (ctypes.c_longlong * 3)()
    _check(lib().sas_cull_stats(h, out, reset, _stream(stream)))
    return tuple(int(v) for v in out)


def sas_matched_filter(d_raw, rows: int, n: int, d_replica, L: int, d_out, stream=None):
    _check(lib().sas_matched_filter(_ptr(d_raw), rows, n, _ptr(d_replica), L, _ptr(d_out), _stream(stream)))


def sas_whiten(d_in, d_out, rows: int, n: int, gamma: float, d_gain=None, stream=None):
    _check(lib().sas_whiten(_ptr(d_in), _ptr(d_out), rows, n, float(gamma), _ptr(d_gain), _stream(stream)))


def sas_tvg(d_in, d_out, rows: int, n: int, alpha: float, d_gain=None, d_median=None, stream=None):
    _check(lib().sas_tvg(_ptr(d_in), _ptr(d_out), rows, n, float(alpha), _ptr(d_gain), _ptr(d_median),
                         _stream(stream)))


def sas_drc(d_image, npix: int, b: float, d_out, d_stats=None, stream=None):
    _check(lib().sas_drc(_ptr(d_image), npix, float(b), _ptr(d_out), _ptr(d_stats), _stream(stream)))


def sas_dpc_delays(h, shift: int, d_centres, K: int, W: int, max_lag: int, d_coarse=None, d_fine=None, d_rho=None,
                   stream=None):
    _check(lib().sas_dpc_delays(h, shift, _ptr(d_centres), K, W, max_lag, _ptr(d_coarse), _ptr(d_fine), _ptr(d_rho),
                                _stream(stream)))


def sas_dpc_footprints(pr: sas_dpc_problem, d_vy, d_vz, d_ps, stream=None):
    _check(lib().sas_dpc_footprints(ctypes.byref(pr), _ptr(d_vy), _ptr(d_vz), _ptr(d_ps), _stream(stream)))


def sas_dpc_model_delays(pr: sas_dpc_problem, d_vy, d_vz, d_out, stream=None):
    _check(lib().sas_dpc_model_delays(ctypes.byref(pr), _ptr(d_vy), _ptr(d_vz), _ptr(d_out), _stream(stream)))


def sas_dpc_solve(pr: sas_dpc_problem, d_vy, d_vz, max_iter: int = 100, stream=None):
    """Returns (final loss, accepted steps); d_vy, d_vz updated in place."""
    loss = ctypes.c_double(0.0)
    iters = ctypes.c_int32(0)
    _check(lib().sas_dpc_solve(ctypes.byref(pr), _ptr(d_vy), _ptr(d_vz), int(max_iter), ctypes.byref(loss),
                               ctypes.byref(iters), _stream(stream)))
    return loss.value, iters.value


def sas_debug_starve_copies(h, skip: int, wait_limit_ms: int):
    _check(lib().sas_debug_starve_copies(h, skip, wait_limit_ms))


def sas_debug_dpc_solve_chunk(rows: int):
    _check(lib().sas_debug_dpc_solve_chunk(int(rows)))


# ---------------------------------------------------------------------------
# Convenience layer

def make_signal(fc, fs, c, t0, n_samples) -> sas_signal:
    return sas_signal(float(fc), float(fs), float(c), float(t0), int(n_samples))


def make_grid(x0, y0, z0, dx, dy, dz, nx, ny, nz=1) -> sas_grid:
    return sas_grid(float(x0), float(y0), float(z0), float(dx), float(dy), float(dz), int(nx), int(ny), int(nz))


def grid_from(g) -> sas_grid:
    """sas_grid from any object with x0 y0 z0 dx dy dz nx ny nz attributes."""
    return make_grid(g.x0, g.y0, g.z0, g.dx, g.dy, g.dz, g.nx, g.ny, g.nz)


def kaiser(beta: float = 4.0, taps: int = 8) -> sas_interp:
    return sas_interp(SAS_INTERP_KAISER_SINC, taps, float(beta), 0, None)


def table_interp(d_table, table_n: int, taps: int = 8) -> sas_interp:
    """Interpolator from a device table [table_n + 1][taps] (torch tensor)."""
    it = sas_interp(SAS_INTERP_TABLE, taps, 0.0, int(table_n), _ptr(d_table))
    it._keep = d_table  # keep the table alive while the struct is in use
    return it


class Geometry:
    """Owns a libsas handle: navigation, sensor positions and the echo."""

    def __init__(self, pos, att, tx_lever, rx_lever, signal: sas_signal, stream=None):
        self._arrays = [np.ascontiguousarray(a, dtype=np.float64) for a in (pos, att, tx_lever, rx_lever)]
        pos_, att_, txl, rxl = self._arrays
        self.P = pos_.shape[0]
        self.C = rxl.reshape(-1, 3).shape[0]
        self.signal = signal
        nav = sas_nav(self.P, self.C, pos_.ctypes.data, att_.ctypes.data, txl.ctypes.data, rxl.ctypes.data)
        self.h = sas_geometry_create(nav, signal, stream)

    @classmethod
    def from_nav(cls, nav: dict, signal: sas_signal, stream=None, use_true=False):
        pos = nav["true_pos"] if use_true else nav["pos"]
        return cls(pos, nav["att"], nav["tx_lever"], nav["rx_lever"], signal, stream)

    def close(self):
        if getattr(self, "h", None):
            sas_geometry_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_offsets(self, offsets, stream=None):
        if offsets is None:
            sas_geometry_set_offsets(self.h, None, 0, stream)
        elif hasattr(offsets, "is_cuda") and offsets.is_cuda:
            sas_geometry_set_offsets(self.h, offsets.contiguous(), 1, stream)
        else:
            a = np.ascontiguousarray(offsets, dtype=np.float64)
            sas_geometry_set_offsets(self.h, a, 0, stream)

    def set_velocity(self, vel, stream=None):
        """Receiver velocity during reception [P,3] m/s (None = stop-and-hop)."""
        if vel is None:
            sas_geometry_set_velocity(self.h, None, 0, stream)
        elif hasattr(vel, "is_cuda") and vel.is_cuda:
            sas_geometry_set_velocity(self.h, vel.contiguous(), 1, stream)
        else:
            sas_geometry_set_velocity(self.h, np.ascontiguousarray(vel, dtype=np.float64), 0, stream)

    def set_refraction(self, z_interface: float, c_sediment: float):
        """Seabed refraction: flat interface at z_interface, sediment sound
        speed c_sediment [m/s] (<= 0 = off)."""
        sas_geometry_set_refraction(self.h, z_interface, c_sediment)

    def set_beam(self, beam_width: float, side: int = 1):
        """Beam field of view of full azimuth width beam_width [rad] (0 = off)."""
        sas_geometry_set_beam(self.h, beam_width, side)

    def positions(self):
        import torch
        tx = torch.empty((self.P, 3), dtype=torch.float64, device="cuda")
        rx = torch.empty((self.P, self.C, 3), dtype=torch.float64, device="cuda")
        sas_geometry_positions(self.h, tx, rx)
        return tx, rx

    def upload_echo(self, echo, store_dtype: int = SAS_ECHO_C64, stream=None):
        if hasattr(echo, "is_cuda"):
            e = echo.contiguous()
            assert e.dtype.is_complex and e.element_size() == 8
            sas_echo_upload(self.h, e, 1 if e.is_cuda else 0, store_dtype, stream)
        else:
            e = np.ascontiguousarray(echo, dtype=np.complex64)
            sas_echo_upload(self.h, e, 0, store_dtype, stream)

    def download_echo(self):
        import torch
        out = torch.empty((self.P, self.C, self.signal.n_samples), dtype=torch.complex64, device="cuda")
        sas_echo_download(self.h, out)
        return out

    def backproject(self, grid: sas_grid, interp: sas_interp | None = None, image=None, accumulate=False,
                    stream=None):
        import torch
        interp = interp or kaiser()
        if image is None:
            image = torch.empty((grid.nz, grid.ny, grid.nx), dtype=torch.complex64, device="cuda")
        if grid.nz == 1:
            sas_backproject_2d(self.h, grid, interp, image, 1 if accumulate else 0, stream)
        else:
            sas_backproject_3d(self.h, grid, interp, image, 1 if accumulate else 0, stream)
        return image

    def sync_status(self, stream=None):
        sas_sync_status(self.h, stream)

    def cull_stats(self, reset: bool = True, stream=None):
        return sas_cull_stats(self.h, 1 if reset else 0, stream)
