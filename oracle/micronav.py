"""FP64 oracle for displaced-phase-centre (DPC) micronavigation (Sec. II-D,
Eqs. 3-8): time-delay estimation between overlapping receivers of
consecutive pings, the DPC residual g (Eq. 4), the robust loss (Eqs. 3, 5),
the smoothness and DVL regularisers (Eqs. 6, 7) and the minimisation of
their sum (Eq. 8) over the per-ping sway and heave velocities.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Plain definitions in
NumPy; scipy's ``least_squares`` (Levenberg-Marquardt / trust region) is the
library step that minimises Eq. 8.  Readings where the paper is silent,
ambiguous or garbled (all recorded in the repository's design notes):

* Kinematics (Sec. II-D: transmission instantaneous, the platform keeps
  moving during reception with p = v t): ping i is sent at T_i from the
  platform position p_i; during its reception the platform moves with the
  constant velocity v_i, and the next ping leaves from
  p_{i+1} = p_i + v_i D_i, D_i = T_{i+1} - T_i.  A ping's attitude is constant
  during its reception.  Transmitter: p_i + R_i l_TX (at t = 0); receiver c
  at time t after the transmission: p_i + v_i t + R_i l_c (R_i from Eq. 2).
* Unknowns: v_y and v_z of every ping; the surge v_x, the attitude, the lever
  arms and the first position p_0 are given.
* DPC pairs: receiver c + s of ping i with receiver c of ping i + 1, c = 0 ..
  C - 1 - s, where s is the number of phase-centre spacings (half an element
  pitch) the array advances per ping (given).
* Footprint p_s (Eq. 4) of window k of the pair (i, c): the point of the flat
  seafloor z = 0 (Sec. II-D: p_s,z = 0) abeam of ping i's phase centre
  (midpoint of its transmitter and receiver c + s, from the navigation prior)
  on the imaging side, at slant range c t_k / 2 from it; fixed while Eq. 8 is
  minimised.  Both receivers of Eq. 4 are taken at t = t_k, the window's
  centre time.
* g is in seconds; the solver works with r = c g (metres).  Eq. 5 with
  h(a) = a^2 is plain least squares; Eq. 3 (Huber) is applied to r / s_h with
  a scale s_h in metres, i.e. the term is s_h^2 h(r / s_h) (up to the factor 2
  of the loss, which does not move the minimum), minimised by iteratively
  reweighted least squares.  Optional weights (the correlation
  coefficients) multiply the squared residuals.
* Eq. 6: v''[i] = v[i+1] - 2 v[i] + v[i-1] (unscaled second differences of
  the per-ping velocities, i = 1 .. P-2), for v_y and v_z.
* Eq. 7 (its index is garbled): the heave position of ping i,
  z_i = z_0 + sum_{n<i} v_z[n] D_n, against the DVL's z_DVL[i] (the depth
  of the platform implied by the DVL altitude over the flat seafloor).
* Time-delay estimation (after the method the paper cites, restated): for a
  window of W samples centred on sample n_k, R(tau) = sum_n e2[n] conj(e1[n -
  tau]) over integer lags |tau| <= L (e1: ping i, receiver c + s; e2: ping
  i + 1, receiver c; samples outside the row read zero); the coarse delay is
  the lag of the largest |R| refined by the parabola through |R| at the peak
  and its two neighbours; the fine delay is -arg(R) / (2 pi fc) with R taken
  at the coarse delay by the same three-point (quadratic) interpolation of
  the complex values; it is unwrapped to the nearest multiple of 1/fc from a
  reference delay (the prediction of the coarse solution).  A peak on the
  edge of the lag range uses the edge lag without refinement.  The
  correlation coefficient is |R(peak)| / sqrt(sum |e2|^2 sum |e1(shifted)|^2).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

import oracle


# --------------------------------------------------------------------------
# Trajectory and sensors

@dataclass
class Platform:
    """Known navigation: p0 [3] (position at ping 0), vx [P] (surge), att [P,3]
    (roll, pitch, yaw), dt [P-1] (ping intervals D_i), tx_lever [3],
    rx_lever [C,3], side (+1 starboard, -1 port)."""
    p0: np.ndarray
    vx: np.ndarray
    att: np.ndarray
    dt: np.ndarray
    tx_lever: np.ndarray
    rx_lever: np.ndarray
    side: int = 1

    @property
    def P(self) -> int:
        return self.vx.size


def positions(pl: Platform, vy, vz) -> np.ndarray:
    """p_i [P,3] from p_0 and the velocities: p_{i+1} = p_i + v_i D_i."""
    v = np.stack([pl.vx, vy, vz], 1)
    p = np.zeros((pl.P, 3))
    p[0] = pl.p0
    for i in range(pl.P - 1):
        p[i + 1] = p[i] + v[i] * pl.dt[i]
    return p


def sensors_at(pl: Platform, vy, vz, i: int, t: float):
    """(transmitter [3] at t = 0, receivers [C,3] at time t) of ping i."""
    p = positions(pl, vy, vz)
    R = oracle.attitude_matrix(*pl.att[i])
    v = np.array([pl.vx[i], vy[i], vz[i]])
    tx = p[i] + R @ pl.tx_lever
    rx = p[i] + v * t + (R @ np.asarray(pl.rx_lever, float).T).T
    return tx, rx


# --------------------------------------------------------------------------
# Eq. 4 residuals

@dataclass
class Measurements:
    """DPC delay measurements: pair ping i [m], receiver c [m] (of ping i + 1;
    ping i uses c + shift), window centre time t [m] (s after transmission),
    delay [m] (s), weight [m]; shift s."""
    ping: np.ndarray
    chan: np.ndarray
    t: np.ndarray
    delay: np.ndarray
    weight: np.ndarray
    shift: int


def footprints(pl: Platform, vy0, vz0, meas: Measurements, c: float) -> np.ndarray:
    """p_s [m,3] from the prior velocities (vy0, vz0): abeam of ping i's
    phase centre on the seafloor z = 0 at slant range c t / 2."""
    p = positions(pl, vy0, vz0)
    out = np.zeros((meas.ping.size, 3))
    for m in range(meas.ping.size):
        i, ch = int(meas.ping[m]), int(meas.chan[m])
        R = oracle.attitude_matrix(*pl.att[i])
        tx = p[i] + R @ pl.tx_lever
        rx = p[i] + R @ np.asarray(pl.rx_lever[ch + meas.shift], float)
        pc = 0.5 * (tx + rx)
        yaw = pl.att[i][2]
        across = np.array([-np.sin(yaw), np.cos(yaw), 0.0]) * pl.side
        rng = 0.5 * c * meas.t[m]
        ground = np.sqrt(max(rng * rng - pc[2] * pc[2], 0.0))
        out[m] = np.array([pc[0], pc[1], 0.0]) + ground * across
    return out


def dpc_residuals(pl: Platform, vy, vz, meas: Measurements, ps, c: float) -> np.ndarray:
    """r = c g (Eq. 4, metres) for every measurement."""
    p = positions(pl, vy, vz)
    v = np.stack([pl.vx, vy, vz], 1)
    lev = np.asarray(pl.rx_lever, float)
    r = np.zeros(meas.ping.size)
    for m in range(meas.ping.size):
        i, ch, t = int(meas.ping[m]), int(meas.chan[m]), float(meas.t[m])
        R1 = oracle.attitude_matrix(*pl.att[i])
        R2 = oracle.attitude_matrix(*pl.att[i + 1])
        tx1 = p[i] + R1 @ pl.tx_lever
        rx1 = p[i] + v[i] * t + R1 @ lev[ch + meas.shift]
        tx2 = p[i + 1] + R2 @ pl.tx_lever
        rx2 = p[i + 1] + v[i + 1] * t + R2 @ lev[ch]
        path1 = np.linalg.norm(tx1 - ps[m]) + np.linalg.norm(ps[m] - rx1)
        path2 = np.linalg.norm(tx2 - ps[m]) + np.linalg.norm(ps[m] - rx2)
        r[m] = path1 - path2 + c * meas.delay[m]
    return r


def model_delays(pl: Platform, vy, vz, meas: Measurements, ps, c: float) -> np.ndarray:
    """The delays that make Eq. 4 vanish: (path2 - path1) / c."""
    zero = Measurements(meas.ping, meas.chan, meas.t, np.zeros_like(meas.delay), meas.weight, meas.shift)
    return -dpc_residuals(pl, vy, vz, zero, ps, c) / c


# --------------------------------------------------------------------------
# Eqs. 6-8

def smooth_residuals(v) -> np.ndarray:
    v = np.asarray(v, float)
    return v[2:] - 2.0 * v[1:-1] + v[:-2]


def heave_positions(pl: Platform, vz) -> np.ndarray:
    z = np.zeros(pl.P)
    z[0] = pl.p0[2]
    for i in range(pl.P - 1):
        z[i + 1] = z[i] + vz[i] * pl.dt[i]
    return z


def total_loss(pl, vy, vz, meas, ps, c, z_dvl, lam1, lam2, huber=0.0) -> float:
    """Eq. 8: sum of weighted h(r) + lam1 (Eq. 6) + lam2 (Eq. 7)."""
    r = dpc_residuals(pl, vy, vz, meas, ps, c)
    if huber > 0:
        a = np.abs(r) / huber
        h = np.where(a <= 1.0, 0.5 * a * a, a - 0.5) * huber * huber * 2.0
    else:
        h = r * r
    dvl = heave_positions(pl, vz) - z_dvl
    return float(np.sum(meas.weight * h) + lam1 * (np.sum(smooth_residuals(vy) ** 2) +
                                                   np.sum(smooth_residuals(vz) ** 2))
                 + lam2 * np.sum(dvl * dvl))


def solve(pl: Platform, vy0, vz0, meas: Measurements, ps, c: float, z_dvl, lam1: float, lam2: float,
          huber: float = 0.0):
    """Minimises Eq. 8 over (v_y, v_z) from the start (vy0, vz0); returns
    (vy, vz, final loss)."""
    from scipy.optimize import least_squares
    P = pl.P
    sw = np.sqrt(meas.weight)

    def f(x):
        vy, vz = x[:P], x[P:]
        r = sw * dpc_residuals(pl, vy, vz, meas, ps, c)
        return r

    def reg(x):
        vy, vz = x[:P], x[P:]
        return np.concatenate([np.sqrt(lam1) * smooth_residuals(vy), np.sqrt(lam1) * smooth_residuals(vz),
                               np.sqrt(lam2) * (heave_positions(pl, vz) - z_dvl)])

    x0 = np.concatenate([vy0, vz0])
    if huber > 0:
        # Huber by iteratively reweighted least squares: each pass minimises the
        # weighted squares with the weights min(1, s_h / |r|) of the previous
        # solution, whose fixed point is the minimum of the Huber loss
        x = x0
        for _ in range(100):
            r = dpc_residuals(pl, x[:P], x[P:], meas, ps, c)
            w = np.sqrt(np.minimum(1.0, huber / np.maximum(np.abs(r), 1e-300)))
            res = least_squares(lambda x_: np.concatenate([w * f(x_), reg(x_)]), x, method="lm", xtol=1e-15,
                                ftol=1e-15, gtol=1e-15, max_nfev=2000)
            step = np.abs(res.x - x).max()
            x = res.x
            if step <= 1e-14 * max(np.abs(x).max(), 1e-3):
                break
        res.x = x
    else:
        res = least_squares(lambda x: np.concatenate([f(x), reg(x)]), x0, method="lm", xtol=1e-15,
                            ftol=1e-15, gtol=1e-15, max_nfev=2000)
    vy, vz = res.x[:P], res.x[P:]
    return vy, vz, total_loss(pl, vy, vz, meas, ps, c, z_dvl, lam1, lam2, huber)


# --------------------------------------------------------------------------
# Time-delay estimation

def correlate(e1, e2, n_centre: int, W: int, L: int) -> np.ndarray:
    """R(tau) for tau = -L .. L over the window [n_centre - W/2, n_centre + W/2)."""
    e1 = np.asarray(e1, np.complex128)
    e2 = np.asarray(e2, np.complex128)
    N = e1.size
    n0 = n_centre - W // 2
    n = np.arange(n0, n0 + W)
    R = np.zeros(2 * L + 1, np.complex128)
    for j, tau in enumerate(range(-L, L + 1)):
        a = np.where((n >= 0) & (n < N), e2[np.clip(n, 0, N - 1)], 0.0)
        m = n - tau
        b = np.where((m >= 0) & (m < N), e1[np.clip(m, 0, N - 1)], 0.0)
        R[j] = np.sum(a * np.conj(b))
    return R


def estimate_delay(e1, e2, n_centre: int, W: int, L: int, fs: float, fc: float):
    """(coarse delay [s], fine delay wrapped to (-1/(2fc), 1/(2fc)] [s],
    correlation coefficient) of e2 against e1 around sample n_centre."""
    R = correlate(e1, e2, n_centre, W, L)
    mag = np.abs(R)
    j = int(np.argmax(mag))
    if 0 < j < 2 * L:
        ym, y0, yp = mag[j - 1], mag[j], mag[j + 1]
        den = ym - 2.0 * y0 + yp
        d = 0.5 * (ym - yp) / den if den != 0.0 else 0.0
        # complex value at the refined lag by the same three-point interpolation
        Rc = R[j] + 0.5 * d * (R[j + 1] - R[j - 1]) + 0.5 * d * d * (R[j + 1] - 2.0 * R[j] + R[j - 1])
    else:
        d = 0.0
        Rc = R[j]
    tau = (j - L) + d
    fine = -np.angle(Rc) / (2.0 * np.pi * fc)
    # correlation coefficient at the integer peak lag
    e1 = np.asarray(e1, np.complex128)
    e2 = np.asarray(e2, np.complex128)
    N = e1.size
    n = np.arange(n_centre - W // 2, n_centre - W // 2 + W)
    a = np.where((n >= 0) & (n < N), e2[np.clip(n, 0, N - 1)], 0.0)
    m = n - (j - L)
    b = np.where((m >= 0) & (m < N), e1[np.clip(m, 0, N - 1)], 0.0)
    den = np.sqrt(np.sum(np.abs(a) ** 2) * np.sum(np.abs(b) ** 2))
    rho = float(mag[j] / den) if den > 0 else 0.0
    return tau / fs, fine, rho


def unwrap(fine, ref, fc: float):
    """fine + k / fc with the integer k that brings it nearest to ref."""
    fine = np.asarray(fine, float)
    k = np.round((np.asarray(ref, float) - fine) * fc)
    return fine + k / fc
