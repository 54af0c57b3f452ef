"""FP64 CPU oracle for synthetic-aperture-sonar time-domain backprojection.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library (``paper_2101_05888_gb300``)
and the library never imports it.

This module is a thin ctypes layer over ``oracle.c`` (compiled here with gcc on
first use) plus small helpers that state the pixel-grid convention.  The
independent NumPy restatement lives in ``oracle.brute`` and the FP64 learned
interpolator maths in ``oracle.mlp``.

Paper: arXiv 2101.05888 (ASASIN).  Eq. 1 forward model, Sec. II-A per-pixel
backprojection, Eq. 2 attitude rotation, Sec. II-B NED frame.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP, strict IEEE FP64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared",
               "-fPIC", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            D = ctypes.c_double
            I = ctypes.c_int
            Lg = ctypes.c_long
            P = ctypes.c_void_p
            L.oracle_max_threads.restype = I
            L.oracle_attitude_matrix.argtypes = [D, D, D, P]
            L.oracle_sensor_positions.argtypes = [I, I, P, P, P, P, P, P, P]
            L.oracle_bessel_i0.argtypes = [D]
            L.oracle_bessel_i0.restype = D
            L.oracle_bessel_i1_over_x.argtypes = [D]
            L.oracle_bessel_i1_over_x.restype = D
            L.oracle_kaiser_sinc_weights.argtypes = [D, I, D, P, P]
            L.oracle_backproject.argtypes = [I, I, P, P, D, D, D, D, I, P, I, I, D, Lg, P, P, P, D, I, P, I]
            L.oracle_backproject_beam_split.argtypes = [I, I, P, P, D, D, D, D, I, P, I, I, D, Lg, P, P, D, I, D,
                                                        P, P, P, I]
            L.oracle_backproject_adjoint.argtypes = [I, I, P, P, D, D, D, D, I, I, D, Lg, P, P, P, P, D, I, P, I]
            L.oracle_vjp_offsets.argtypes = [I, I, P, P, D, D, D, D, I, P, I, D, Lg, P, P, P, P, D, I, P, I]
            L.oracle_delay_eval.argtypes = [P, P, P, P, D, P]
            L.oracle_set_medium.argtypes = [D, D]
            L.oracle_sharpness.argtypes = [Lg, P, P, P]
            L.oracle_lfm_compressed_pulse.argtypes = [D, D, D]
            L.oracle_lfm_compressed_pulse.restype = D
            L.oracle_simulate_points.argtypes = [I, I, P, P, D, D, D, D, I, D, D, Lg, P, I, P, P, I]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def max_threads() -> int:
    return lib().oracle_max_threads()


@dataclass(frozen=True)
class Signal:
    """Signal parameters: carrier fc [Hz], complex sample rate fs [Hz], sound
    speed c [m/s], time of sample 0 after transmit t0 [s], samples per row."""
    fc: float
    fs: float
    c: float
    t0: float
    n_samples: int


# --------------------------------------------------------------------------
# Geometry (Eq. 2, Sec. II-B/C)

def attitude_matrix(roll: float, pitch: float, yaw: float) -> np.ndarray:
    R = np.zeros(9)
    lib().oracle_attitude_matrix(float(roll), float(pitch), float(yaw), _p(R))
    return R.reshape(3, 3)


def sensor_positions(pos, att, tx_lever, rx_lever, offsets=None):
    """Returns (tx [P,3], rx [P,C,3]) in metres, NED frame."""
    pos, att = _f64(pos), _f64(att)
    tx_lever, rx_lever = _f64(tx_lever).reshape(3), _f64(rx_lever).reshape(-1, 3)
    P, C = pos.shape[0], rx_lever.shape[0]
    off = None if offsets is None else _f64(offsets).reshape(P, 3)
    tx = np.zeros((P, 3))
    rx = np.zeros((P, C, 3))
    lib().oracle_sensor_positions(P, C, _p(pos), _p(att), _p(tx_lever), _p(rx_lever),
                                  None if off is None else _p(off), _p(tx), _p(rx))
    return tx, rx


# --------------------------------------------------------------------------
# Interpolator

def bessel_i0(x: float) -> float:
    return lib().oracle_bessel_i0(float(x))


def bessel_i1_over_x(x: float) -> float:
    return lib().oracle_bessel_i1_over_x(float(x))


def kaiser_sinc_weights(f: float, taps: int, beta: float, deriv: bool = False):
    w = np.zeros(taps)
    dw = np.zeros(taps) if deriv else None
    lib().oracle_kaiser_sinc_weights(float(f), int(taps), float(beta), _p(w),
                                     None if dw is None else _p(dw))
    return (w, dw) if deriv else w


def tap_offsets(taps: int) -> np.ndarray:
    """Offset k_m of tap m from floor(u): m - taps/2 + 1."""
    return np.arange(taps) - taps // 2 + 1


# --------------------------------------------------------------------------
# Pixel grid: pixel (ix, iy, iz) sits at (x0 + ix dx, y0 + iy dy, z0 + iz dz);
# images are stored [nz][ny][nx] with x (along-track, N) fastest.

def grid_points(x0, y0, z0, dx, dy, dz, nx, ny, nz=1) -> np.ndarray:
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pts = np.stack([x0 + ix * dx, y0 + iy * dy, z0 + iz * dz], axis=-1)
    return pts.reshape(-1, 3).astype(np.float64)


def grid_index_points(x0, y0, z0, dx, dy, dz, idx) -> np.ndarray:
    """Pixel coordinates for integer indices idx [n,3] = (ix, iy, iz)."""
    idx = np.asarray(idx, dtype=np.float64).reshape(-1, 3)
    return np.stack([x0 + idx[:, 0] * dx, y0 + idx[:, 1] * dy, z0 + idx[:, 2] * dz], axis=-1)


# --------------------------------------------------------------------------
# Backprojection and its adjoints

def _echo_c128(echo) -> np.ndarray:
    e = np.ascontiguousarray(echo, dtype=np.complex128)
    assert e.ndim == 3
    return e


def _vel(vel, P):
    return None if vel is None else _p(_f64(vel).reshape(P, 3))


class medium:
    """Context manager: the sediment-water interface at depth z_interface
    (NED z) with sediment sound speed c_sediment for every oracle call inside
    (refraction model; stop-and-hop delays only)."""

    def __init__(self, z_interface: float, c_sediment: float):
        self.z, self.c = float(z_interface), float(c_sediment)

    def __enter__(self):
        lib().oracle_set_medium(self.z, self.c)
        return self

    def __exit__(self, *exc):
        lib().oracle_set_medium(0.0, 0.0)
        return False


def delay(x, t, r, v, c):
    """(tau, kappa) of one (pixel, transmitter, receiver): stop-and-hop for
    v None, else the receiver moving with velocity v during reception."""
    out = np.zeros(2)
    vv = None if v is None else _f64(v)
    lib().oracle_delay_eval(_p(_f64(x)), _p(_f64(t)), _p(_f64(r)), None if vv is None else _p(vv), float(c), _p(out))
    return float(out[0]), float(out[1])


def backproject(tx, rx, sig: Signal, echo, taps: int, beta: float, pix, nthreads: int = 0,
                att=None, beam_width: float = 0.0, side: int = 1, vel=None):
    """I(x) at the given pixels [n,3]; returns complex128 [n].  A complex64
    echo is read in place (widened exactly to FP64), others as complex128.
    att [P,3] and beam_width (full azimuth width, radians) > 0 apply the
    beam field of view looking to ``side`` (+1 starboard, -1 port).  vel
    [P,3]: receiver velocity during reception (continuous motion), None =
    stop-and-hop."""
    tx, rx, pix = _f64(tx), _f64(rx), _f64(pix).reshape(-1, 3)
    if isinstance(echo, np.ndarray) and echo.dtype == np.complex64 and echo.flags.c_contiguous:
        e, f32 = echo, 1
    else:
        e, f32 = _echo_c128(echo), 0
    P, C = tx.shape[0], rx.shape[1]
    assert e.shape == (P, C, sig.n_samples)
    out = np.zeros((pix.shape[0], 2))
    a = None if att is None else _f64(att).reshape(P, 3)
    btan = float(np.tan(0.5 * beam_width)) if (beam_width and beam_width > 0) else 0.0
    lib().oracle_backproject(P, C, _p(tx), _p(rx), sig.fc, sig.fs, sig.c, sig.t0, sig.n_samples,
                             _p(e), f32, int(taps), float(beta), pix.shape[0], _p(pix), _p(out),
                             None if a is None else _p(a), btan, int(side), _vel(vel, P), int(nthreads))
    return out[:, 0] + 1j * out[:, 1]


def backproject_beam_split(tx, rx, sig: Signal, echo, taps: int, beta: float, pix, att, beam_width: float,
                           side: int = 1, eps: float = 2e-6, nthreads: int = 0, vel=None):
    """Beam-limited image split by decision margin: (sure [n] complex128,
    amb [n] float64).  ``sure`` sums the terms whose transmitter and receiver
    see the pixel by a relative margin above eps, ``amb`` the magnitudes of
    the terms within eps of a beam edge; any beam test accurate to eps gives
    an image I with |I - sure| <= amb pixel by pixel."""
    tx, rx, pix = _f64(tx), _f64(rx), _f64(pix).reshape(-1, 3)
    if isinstance(echo, np.ndarray) and echo.dtype == np.complex64 and echo.flags.c_contiguous:
        e, f32 = echo, 1
    else:
        e, f32 = _echo_c128(echo), 0
    P, C = tx.shape[0], rx.shape[1]
    assert e.shape == (P, C, sig.n_samples) and beam_width > 0
    out = np.zeros((pix.shape[0], 2))
    amb = np.zeros(pix.shape[0])
    a = _f64(att).reshape(P, 3)
    lib().oracle_backproject_beam_split(P, C, _p(tx), _p(rx), sig.fc, sig.fs, sig.c, sig.t0, sig.n_samples,
                                        _p(e), f32, int(taps), float(beta), pix.shape[0], _p(pix), _p(a),
                                        float(np.tan(0.5 * beam_width)), int(side), float(eps), _p(out), _p(amb),
                                        _vel(vel, P), int(nthreads))
    return out[:, 0] + 1j * out[:, 1], amb


def _beam_args(att, beam_width, P):
    a = None if att is None else _f64(att).reshape(P, 3)
    btan = float(np.tan(0.5 * beam_width)) if (beam_width and beam_width > 0) else 0.0
    return a, btan


def backproject_adjoint(tx, rx, sig: Signal, img, taps: int, beta: float, pix, nthreads: int = 0,
                        att=None, beam_width: float = 0.0, side: int = 1, vel=None):
    """Linear adjoint: image values at pixels -> echo [P,C,Ns] complex128."""
    tx, rx, pix = _f64(tx), _f64(rx), _f64(pix).reshape(-1, 3)
    im = np.ascontiguousarray(np.asarray(img, dtype=np.complex128).reshape(-1))
    P, C = tx.shape[0], rx.shape[1]
    out = np.zeros((P, C, sig.n_samples), dtype=np.complex128)
    a, btan = _beam_args(att, beam_width, P)
    lib().oracle_backproject_adjoint(P, C, _p(tx), _p(rx), sig.fc, sig.fs, sig.c, sig.t0,
                                     sig.n_samples, int(taps), float(beta), pix.shape[0], _p(pix),
                                     _p(im), _p(out), None if a is None else _p(a), btan, int(side),
                                     _vel(vel, P), int(nthreads))
    return out


def vjp_offsets(tx, rx, sig: Signal, echo, taps: int, beta: float, pix, g, nthreads: int = 0,
                att=None, beam_width: float = 0.0, side: int = 1, vel=None):
    """dL/d(dp) [P,3] given g = dL/dI* at the pixels."""
    tx, rx, pix = _f64(tx), _f64(rx), _f64(pix).reshape(-1, 3)
    e = _echo_c128(echo)
    gg = np.ascontiguousarray(np.asarray(g, dtype=np.complex128).reshape(-1))
    P, C = tx.shape[0], rx.shape[1]
    out = np.zeros((P, 3))
    a, btan = _beam_args(att, beam_width, P)
    lib().oracle_vjp_offsets(P, C, _p(tx), _p(rx), sig.fc, sig.fs, sig.c, sig.t0, sig.n_samples,
                             _p(e), int(taps), float(beta), pix.shape[0], _p(pix), _p(gg),
                             _p(out), None if a is None else _p(a), btan, int(side), _vel(vel, P), int(nthreads))
    return out


def sharpness(img, want_grad: bool = False):
    """Returns (S, N, D) and optionally g = dS/dI*."""
    im = np.ascontiguousarray(np.asarray(img, dtype=np.complex128).reshape(-1))
    out = np.zeros(3)
    g = np.zeros(im.shape[0], dtype=np.complex128) if want_grad else None
    lib().oracle_sharpness(im.shape[0], _p(im), _p(out), None if g is None else _p(g))
    return (tuple(out), g) if want_grad else tuple(out)


# --------------------------------------------------------------------------
# Test-input simulator (Eq. 1 with point scatterers)

def lfm_compressed_pulse(t: float, B: float, T: float) -> float:
    return lib().oracle_lfm_compressed_pulse(float(t), float(B), float(T))


def simulate_points(tx, rx, sig: Signal, B: float, T: float, scat, half_width: int = 0,
                    nthreads: int = 0, echo=None, vel=None):
    """Matched-filtered echo of point scatterers scat [n,5] = (x,y,z,ReA,ImA).
    Accumulates into ``echo`` (complex128 [P,C,Ns]) if given."""
    tx, rx = _f64(tx), _f64(rx)
    sc = _f64(scat).reshape(-1, 5)
    P, C = tx.shape[0], rx.shape[1]
    if echo is None:
        echo = np.zeros((P, C, sig.n_samples), dtype=np.complex128)
    assert echo.dtype == np.complex128 and echo.flags.c_contiguous
    lib().oracle_simulate_points(P, C, _p(tx), _p(rx), sig.fc, sig.fs, sig.c, sig.t0,
                                 sig.n_samples, float(B), float(T), sc.shape[0], _p(sc),
                                 int(half_width), _p(echo), _vel(vel, P), int(nthreads))
    return echo


def rel_l2(a, b) -> float:
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
