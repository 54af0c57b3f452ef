"""Pins for the oracle's geometry: Eq. 2 attitude rotation and lever arms."""
import os

import numpy as np
import pytest

import oracle
from oracle import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "eq2_sign_conventions.txt")


def _angles(n, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-np.pi, np.pi, size=(n, 3))


def test_rotation_orthonormal_det1():
    for r, p, y in _angles(50, 1):
        R = oracle.attitude_matrix(r, p, y)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1.0) < 1e-13


def test_rotation_equals_textbook_product():
    """Eq. 2's printed entries equal Rz(yaw) Ry(pitch) Rx(roll) built from the
    single-axis rotations (independent construction in brute.py)."""
    for r, p, y in _angles(50, 2):
        assert np.allclose(oracle.attitude_matrix(r, p, y), brute.attitude_matrix(r, p, y), atol=1e-14)


def test_rotation_single_axis_cases():
    a = 0.37
    c, s = np.cos(a), np.sin(a)
    assert np.allclose(oracle.attitude_matrix(a, 0, 0), [[1, 0, 0], [0, c, -s], [0, s, c]], atol=1e-15)
    assert np.allclose(oracle.attitude_matrix(0, a, 0), [[c, 0, s], [0, 1, 0], [-s, 0, c]], atol=1e-15)
    assert np.allclose(oracle.attitude_matrix(0, 0, a), [[c, -s, 0], [s, c, 0], [0, 0, 1]], atol=1e-15)
    assert np.allclose(oracle.attitude_matrix(0, 0, 0), np.eye(3))


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if not line:
            continue
        t = line.split()
        rows.append((float(t[0]), float(t[1]), float(t[2]), [float(t[3]), float(t[4]), float(t[5])],
                     "xyz".index(t[6]), int(t[7])))
    assert len(rows) >= 6
    return rows


@pytest.mark.parametrize("row", _golden_rows())
def test_rotation_sign_conventions(row):
    roll, pitch, yaw, body, comp, sign = row
    v = oracle.attitude_matrix(roll, pitch, yaw) @ np.array(body)
    assert np.sign(v[comp]) == sign
    assert abs(v[comp]) > 0.1


def test_positions_zero_attitude_is_translation():
    P, C = 5, 3
    rng = np.random.default_rng(3)
    pos = rng.normal(size=(P, 3))
    txl = rng.normal(size=3)
    rxl = rng.normal(size=(C, 3))
    tx, rx = oracle.sensor_positions(pos, np.zeros((P, 3)), txl, rxl)
    assert np.allclose(tx, pos + txl, atol=1e-15)
    assert np.allclose(rx, pos[:, None, :] + rxl[None], atol=1e-15)


def test_positions_yaw_quarter_turn():
    """Heading east (yaw +90 deg): a lever along the bow (+x) points east (+y)."""
    tx, rx = oracle.sensor_positions(np.zeros((1, 3)), [[0, 0, np.pi / 2]], [1.0, 0, 0], [[0, 2.0, 0]])
    assert np.allclose(tx[0], [0, 1, 0], atol=1e-15)
    assert np.allclose(rx[0, 0], [-2, 0, 0], atol=1e-15)


def test_positions_offsets_shift_everything():
    P, C = 4, 2
    rng = np.random.default_rng(4)
    pos, att = rng.normal(size=(P, 3)), rng.normal(scale=0.1, size=(P, 3))
    txl, rxl = rng.normal(size=3), rng.normal(size=(C, 3))
    off = rng.normal(size=(P, 3))
    tx0, rx0 = oracle.sensor_positions(pos, att, txl, rxl)
    tx1, rx1 = oracle.sensor_positions(pos, att, txl, rxl, off)
    assert np.allclose(tx1 - tx0, off, atol=1e-14)
    assert np.allclose(rx1 - rx0, off[:, None, :], atol=1e-14)


def test_positions_match_brute():
    P, C = 6, 4
    rng = np.random.default_rng(5)
    pos, att = rng.normal(size=(P, 3)), rng.uniform(-0.5, 0.5, size=(P, 3))
    txl, rxl = rng.normal(size=3), rng.normal(size=(C, 3))
    a = oracle.sensor_positions(pos, att, txl, rxl)
    b = brute.sensor_positions(pos, att, txl, rxl)
    assert np.allclose(a[0], b[0], atol=1e-14) and np.allclose(a[1], b[1], atol=1e-14)
