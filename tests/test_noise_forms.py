"""The lane-centred synthesis of the mode noise (Sec. 2's K SALT modes), checked on the
CPU against the oracle's direct sum dU_i = sum_k xi_k(x_i) (dW_k + lambda_k dt).

The warp kernels hold 2H consecutive nodes a lane and sum the step's increment about the
lane's centre theta_c: dU/4 (theta_c -+ d) = E(d) -+ O(d), E(d) = sum_j v_j cos(j d),
O(d) = sum_j q_j sin(j d), with (v_j, q_j) the step's weights of harmonic j rotated by
j theta_c.  E and O come either from tabulated cos(j d), sin(j d) of the node offsets, or
(the warp-group kernels, where the host's fit qualifies) from Chebyshev polynomials in
s = (d / d_max)^2 of both.  These tests emulate each form's lane arithmetic in float32
(every multiply-add rounded once) and require it to match the oracle's sum to float
rounding; the GPU tests run the kernels themselves."""
import dataclasses
import math

import numpy as np
import pytest

from tests.helpers import noise_poly_expected, oracle_model
from workloads import get_config, mode_amplitudes

WNP = 4
f32 = np.float32


def fma32(a, b, c):
    # a b + c rounded once to float32 (the product of two floats is exact in double)
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def lane_centre(n, H, t):
    # sin and cos of the lane centre 2 pi (2 H t + H - 1/2) / n, rounded to float
    ang = math.pi * (2 * (2 * H) * t + 2 * H - 1) / n
    return f32(math.sin(ang)), f32(math.cos(ang))


def rotated_weights(wq, sc, cc):
    # (v_j, q_j) by the rotation recurrence of (sin, cos)(j theta_c) in float32
    K2 = len(wq) // 2
    v, q = np.empty(K2, f32), np.empty(K2, f32)
    sj, cj = sc, cc
    for j in range(K2):
        a, b = wq[2 * j], wq[2 * j + 1]
        v[j] = fma32(a, sj, f32(b * cj))
        q[j] = fma32(a, cj, -f32(b * sj))
        sj, cj = fma32(sj, cc, f32(cj * sc)), fma32(cj, cc, -f32(sj * sc))
    return v, q


def even_odd_tables(v, q, n, H):
    # E(d_m), O(d_m), m < H, from float tables of cos(j d_m), sin(j d_m)
    d = (np.arange(H) + 0.5) * 2 * math.pi / n
    E, O = np.zeros(H, f32), np.zeros(H, f32)
    for j in range(len(v)):
        co = np.cos((j + 1) * d).astype(f32)
        si = np.sin((j + 1) * d).astype(f32)
        for m in range(H):
            E[m] = fma32(v[j], co[m], E[m])
            O[m] = fma32(q[j], si[m], O[m])
    return E, O


def poly_coefficients(n, H, K2):
    # per harmonic, the interpolants in s of cos(x sqrt s) and sin(x sqrt s) / sqrt s at the
    # WNP Chebyshev points of [0, 1], x = j d_max, rounded to float
    dmax = 2 * math.pi * (H - 0.5) / n
    sn = 0.5 * (1 + np.cos(np.pi * (np.arange(WNP) + 0.5) / WNP))
    P = np.polynomial.polynomial
    c = np.empty((K2, WNP, 2))
    for j in range(1, K2 + 1):
        x = j * dmax
        c[j - 1, :, 0] = P.polyfit(sn, np.cos(x * np.sqrt(sn)), WNP - 1)
        c[j - 1, :, 1] = P.polyfit(sn, np.sin(x * np.sqrt(sn)) / np.sqrt(sn), WNP - 1)
    return c.astype(f32)


def even_odd_poly(v, q, n, H):
    c = poly_coefficients(n, H, len(v))
    e, o = np.zeros(WNP, f32), np.zeros(WNP, f32)
    for j in range(len(v)):
        for k in range(WNP):
            e[k] = fma32(v[j], c[j, k, 0], e[k])
            o[k] = fma32(q[j], c[j, k, 1], o[k])
    E, O = np.empty(H, f32), np.empty(H, f32)
    for m in range(H):
        tau = f32(f32(2 * m + 1) / f32(2 * H - 1))
        s = f32(tau * tau)
        ev, ov = e[WNP - 1], o[WNP - 1]
        for k in range(WNP - 2, -1, -1):
            ev = fma32(ev, s, e[k])
            ov = fma32(ov, s, o[k])
        E[m], O[m] = ev, f32(ov * tau)
    return E, O


def lane_values(E, O, H):
    # the lane's 2H nodes in order: theta_c - d_{H-1} .. theta_c - d_0, theta_c + d_0 .. + d_{H-1}
    first = np.array([f32(E[H - 1 - k] - O[H - 1 - k]) for k in range(H)])
    second = np.array([f32(E[k] + O[k]) for k in range(H)])
    return np.concatenate([first, second])


@pytest.mark.parametrize("rule", ["inv_j", "const"])
@pytest.mark.parametrize("n,H,K", [(4096, 16, 32), (2048, 8, 32), (4096, 16, 64), (1024, 16, 8), (4096, 16, 42),
                                   (4096, 8, 6)])
def test_lane_centred_noise_matches_oracle(n, H, K, rule):
    # the workload's amplitudes a_j = 0.05 / j, and equal ones, under which the high harmonics
    # (where the polynomials' last terms matter) weigh as much as the low ones.  The bound,
    # 2^-21.5 of sum_j |v_j| + |q_j|, is twice the largest error of either form here (2^-22.5),
    # and below what dropping the polynomials' last coefficient gives (2^-21.2 at K = 32 with
    # equal amplitudes, 2^-19.1 at K = 42)
    cfg = dataclasses.replace(get_config("cfg5_f32"), n=n, K=K, amp_rule=rule)
    om = oracle_model(cfg)
    rng = np.random.default_rng(7 + n + K)
    amps = np.repeat(np.asarray(mode_amplitudes(cfg)), 2)
    poly = noise_poly_expected(n, H, K // 2)
    for t in rng.choice(n // (2 * H), size=8, replace=False):
        w = rng.normal(0.0, math.sqrt(cfg.dt), K)
        exact = (om.modes().T @ w)[2 * H * t: 2 * H * (t + 1)] / 4
        wq = (amps * w / 4).astype(f32)
        sc, cc = lane_centre(n, H, t)
        v, q = rotated_weights(wq, sc, cc)
        scale = float(np.abs(v).sum() + np.abs(q).sum())
        forms = [even_odd_tables(v, q, n, H)] + ([even_odd_poly(v, q, n, H)] if poly else [])
        for E, O in forms:
            got = lane_values(E, O, H)
            assert np.abs(got - exact).max() <= 2.0 ** -21.5 * scale, (n, H, K, t)


def test_poly_fits_hold_where_chosen():
    # where the rule takes the polynomials, the fits in double precision reproduce cos(j d)
    # and sin(j d) at every offset to 2^-30; at the largest K they take (21 harmonics at
    # n = 4096, 32 nodes a lane) and not beyond it
    assert noise_poly_expected(4096, 16, 21) and not noise_poly_expected(4096, 16, 22)
    for n, H, K2 in [(4096, 16, 16), (4096, 16, 21), (2048, 8, 16)]:
        c = poly_coefficients(n, H, K2).astype(np.float64)
        dmax = 2 * math.pi * (H - 0.5) / n
        tau = (np.arange(H) + 0.5) / (H - 0.5)
        P = np.polynomial.polynomial
        for j in range(1, K2 + 1):
            # float-rounded coefficients: within 2^-24 of the double fit, itself within 2^-30
            ec = P.polyval(tau * tau, c[j - 1, :, 0])
            es = tau * P.polyval(tau * tau, c[j - 1, :, 1])
            assert np.abs(ec - np.cos(j * dmax * tau)).max() <= 2.0 ** -23
            assert np.abs(es - np.sin(j * dmax * tau)).max() <= 2.0 ** -23
