"""Pins of the oracle's rotation square root (Section III-C-1, Eqs. rodrigues, halfangle).

Checked against what fixes a principal rotation square root: S^2 = R, S orthogonal with
det S = 1, rotation angle |theta|/2 about the same axis, and agreement with the library
routine scipy.linalg.sqrtm away from theta = pi; plus the paper's Table 2 error statistics on
its own angle sweep (tests/golden/table2_rotation_sqrt.json).
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.linalg import sqrtm
from scipy.spatial.transform import Rotation

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_rotation_sqrt.json")


def _rot(axis, theta):
    return Rotation.from_rotvec(np.asarray(axis) / np.linalg.norm(axis) * theta).as_matrix()


def _angle(S):
    return math.acos(max(-1.0, min(1.0, 0.5 * (np.trace(S) - 1.0))))


def _sweep():
    g = json.load(open(GOLDEN))["sweep"]
    return np.linspace(g["theta_lo"], math.pi + g["theta_hi_minus_pi"], g["n_angles"])


def test_paper_sweep_accuracy_and_table2(orc):
    g = json.load(open(GOLDEN))
    rng = np.random.default_rng(20)
    errs = []
    for trial in range(10):
        axis = rng.standard_normal(3)
        for th in _sweep():
            R = _rot(axis, th)
            S = orc.rot_sqrt(R)
            err = np.linalg.norm(S @ S - R)
            errs.append(err)
            assert err < 1e-13
            assert np.abs(S.T @ S - np.eye(3)).max() < 1e-14
            assert abs(np.linalg.det(S) - 1.0) < 1e-14
            # principal root: half of the principal angle of R, same axis (up to orientation)
            th_p = _angle(R)
            assert abs(_angle(S) - 0.5 * th_p) < 1e-7
    errs = np.array(errs)
    # at least as accurate as the paper's CUDA routine on the same sweep (Table 2)
    assert errs.mean() <= g["cuda_error"]["mean"]
    assert np.median(errs) <= 2 * g["cuda_error"]["median"]
    assert errs.max() <= g["cuda_error"]["std_or_max"]


def test_matches_scipy_sqrtm_away_from_pi(orc):
    rng = np.random.default_rng(21)
    for _ in range(200):
        axis = rng.standard_normal(3)
        th = rng.uniform(-3.0, 3.0)
        R = _rot(axis, th)
        S = orc.rot_sqrt(R)
        Sref = np.real(sqrtm(R))
        assert np.abs(S - Sref).max() < 1e-12


def test_endpoints(orc):
    # identity
    assert np.array_equal(orc.rot_sqrt(np.eye(3)), np.eye(3))
    rng = np.random.default_rng(22)
    for th in (1e-14, 1e-10, 1e-6, 1e-3, math.pi - 1e-3, math.pi - 1e-8, math.pi):
        for _ in range(20):
            axis = rng.standard_normal(3)
            R = _rot(axis, th)
            S = orc.rot_sqrt(R)
            assert np.linalg.norm(S @ S - R) < 1e-13
            assert np.abs(S.T @ S - np.eye(3)).max() < 1e-14
    # exactly pi about a coordinate axis: S is a quarter turn about that axis (either sense)
    for a in range(3):
        e = np.zeros(3)
        e[a] = 1.0
        R = 2.0 * np.outer(e, e) - np.eye(3)
        S = orc.rot_sqrt(R)
        assert np.linalg.norm(S @ S - R) < 1e-15
        assert abs(_angle(S) - math.pi / 2) < 1e-14
        assert np.allclose(S @ e, e)


def test_small_angle_keeps_half_angle(orc):
    """A small nonzero rotation must not collapse to S = I: S is the rotation by theta/2."""
    axis = np.array([0.3, -0.4, 0.5])
    for th in (1e-9, 1e-5, 1e-2):
        S = orc.rot_sqrt(_rot(axis, th))
        np.testing.assert_allclose(S, _rot(axis, th / 2), atol=5e-16, rtol=0)
