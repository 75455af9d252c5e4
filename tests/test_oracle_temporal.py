"""Pins of the oracle's temporal accumulation (paper Sec. 4.3) against closed
forms, exact special cases and invariants (CPU only)."""
import numpy as np
import pytest

from oracle import temporal as ot
import synth


def _flat_geometry(H, W):
    P = np.zeros((3, H, W), np.float32)
    P[2] = 5.0
    n = np.zeros((3, H, W), np.float32)
    n[2] = -1.0
    return P, n


def _rad(g, H, W):
    return g.uniform(0.1, 2.0, (3, H, W)).astype(np.float32)


def test_static_running_mean_then_ema_closed_form():
    # motion 0, identical geometry: running mean for 1 / alpha_min frames, then
    # an exponential moving average with factor alpha_min
    H, W, T = 5, 7, 11
    g = np.random.default_rng(0)
    P, n = _flat_geometry(H, W)
    m = np.zeros((2, H, W), np.float32)
    cs = [_rad(g, H, W) for _ in range(T)]
    st = ot.TemporalState(H, W)
    for t in range(T):
        A = ot.accumulate(st, cs[t], P, n, m)
        k = t + 1
        if k <= 5:
            ref = np.mean(np.stack(cs[:k]).astype(np.float64), axis=0)
        else:
            ref = 0.8 ** (k - 5) * np.mean(np.stack(cs[:5]).astype(np.float64), axis=0)
            for j in range(6, k + 1):
                ref = ref + 0.2 * 0.8 ** (k - j) * cs[j - 1].astype(np.float64)
        np.testing.assert_allclose(A, ref, rtol=1e-12, atol=0)
        np.testing.assert_allclose(st.h, k)


def test_constant_signal_is_a_fixed_point_under_fractional_motion():
    H, W = 9, 12
    g = np.random.default_rng(1)
    P, n = _flat_geometry(H, W)
    st = ot.TemporalState(H, W)
    c = np.full((3, H, W), 0.7, np.float32)
    for t in range(4):
        m = g.uniform(-1.5, 1.5, (2, H, W)).astype(np.float32)
        A = ot.accumulate(st, c, P, n, m)
        np.testing.assert_allclose(A, 0.7, rtol=1e-6)


def test_first_frame_and_inconsistent_normals_keep_the_1spp_value():
    H, W = 6, 8
    g = np.random.default_rng(2)
    P, n = _flat_geometry(H, W)
    m = np.zeros((2, H, W), np.float32)
    st = ot.TemporalState(H, W)
    for t in range(3):
        c = _rad(g, H, W)
        nn = n if t % 2 == 0 else -n  # normals flip every frame: dot = -1
        A = ot.accumulate(st, c, P, nn, m)
        np.testing.assert_array_equal(A, c.astype(np.float64))
        np.testing.assert_array_equal(st.h, 1.0)


def test_integer_motion_is_an_exact_shift():
    H, W = 7, 9
    g = np.random.default_rng(3)
    P, n = _flat_geometry(H, W)
    st = ot.TemporalState(H, W)
    c1, c2 = _rad(g, H, W), _rad(g, H, W)
    ot.accumulate(st, c1, P, n, np.zeros((2, H, W), np.float32))
    m = np.zeros((2, H, W), np.float32)
    m[0], m[1] = -2.0, 1.0
    A = ot.accumulate(st, c2, P, n, m)
    for y in range(H):
        for x in range(W):
            qx, qy = x - 2, y + 1
            if 0 <= qx < W and 0 <= qy < H:
                ref = 0.5 * (c1[:, qy, qx].astype(np.float64) + c2[:, y, x])
            else:
                ref = c2[:, y, x].astype(np.float64)
            np.testing.assert_allclose(A[:, y, x], ref, rtol=1e-12)


def test_half_pixel_motion_averages_two_neighbours():
    H, W = 4, 6
    g = np.random.default_rng(4)
    P, n = _flat_geometry(H, W)
    st = ot.TemporalState(H, W)
    c1, c2 = _rad(g, H, W), _rad(g, H, W)
    ot.accumulate(st, c1, P, n, np.zeros((2, H, W), np.float32))
    m = np.zeros((2, H, W), np.float32)
    m[0] = 0.5
    A = ot.accumulate(st, c2, P, n, m)
    for x in range(W - 1):
        prev = 0.5 * (c1[:, :, x].astype(np.float64) + c1[:, :, x + 1])
        np.testing.assert_allclose(A[:, :, x], 0.5 * (prev + c2[:, :, x]), rtol=1e-12)
    # last column: only the in-image tap (weight 0.5 > min_weight) is kept, renormalised
    np.testing.assert_allclose(A[:, :, W - 1], 0.5 * (c1[:, :, W - 1].astype(np.float64) + c2[:, :, W - 1]),
                               rtol=1e-12)


def test_position_threshold_and_min_weight():
    H, W = 3, 4
    g = np.random.default_rng(5)
    P, n = _flat_geometry(H, W)
    st = ot.TemporalState(H, W)
    c1, c2 = _rad(g, H, W), _rad(g, H, W)
    ot.accumulate(st, c1, P, n, np.zeros((2, H, W), np.float32))
    P2 = P.copy()
    P2[0, 0, 0] += 0.099   # kept (0.099^2 < 0.1^2)
    P2[0, 0, 1] += 0.101   # rejected
    A = ot.accumulate(st, c2, P2, n, np.zeros((2, H, W), np.float32))
    np.testing.assert_allclose(A[:, 0, 0], 0.5 * (c1[:, 0, 0].astype(np.float64) + c2[:, 0, 0]), rtol=1e-12)
    np.testing.assert_array_equal(A[:, 0, 1], c2[:, 0, 1].astype(np.float64))
    # a reprojection whose only in-image tap has weight 1e-4 (< min_weight) restarts
    st = ot.TemporalState(H, W)
    ot.accumulate(st, c1, P, n, np.zeros((2, H, W), np.float32))
    m = np.zeros((2, H, W), np.float32)
    m[0] = np.float32(-0.9999)   # q = x - 0.9999: taps x-1 (weight 0.9999) and x (weight 1e-4)
    A = ot.accumulate(st, c2, P, n, m)
    np.testing.assert_array_equal(A[:, :, 0], c2[:, :, 0].astype(np.float64))


@pytest.mark.parametrize("T", [6])
def test_accumulation_reduces_noise_on_a_moving_camera_sequence(T):
    seq = synth.make_sequence(48, 64, T, seed=3)
    st = ot.TemporalState(48, 64)
    # expected radiance per pixel: clean x E[lognormal(0,1)] x E[firefly factor]
    scale = np.exp(0.5) * (0.98 + 0.02 * 50.0)
    errs_in, errs_acc = [], []
    for f in seq:
        A = ot.accumulate(st, f["radiance"], f["position"], f["normal"], f["motion"])
        ex = scale * f["clean"].astype(np.float64)
        errs_in.append(np.median(np.abs(f["radiance"] / ex - 1.0)))
        errs_acc.append(np.median(np.abs(A / ex - 1.0)))
    assert errs_acc[0] == pytest.approx(errs_in[0])
    assert all(b < a for a, b in zip(errs_acc, errs_acc[1:]))  # error falls frame after frame
    assert errs_acc[-1] < 0.85 * errs_in[-1]
    assert np.mean(st.h) > 3.0
