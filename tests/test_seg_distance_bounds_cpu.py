"""CPU check of the segmentation's distance-form choice (the assignment kernel's 32-bit DOT32 form): the
host picks it only when 3 wc' vmax^2 + 6 ws' R^2 < 2^31, and then every partial sum of the kernel's
five multiply-adds, evaluated exactly in Python integers at the extreme positions and colours, stays
below 2^31 in magnitude. Also pins which form the benchmark workloads take.

Quantities (1/16 units): vmax = 16 (2^bd - 1); R = 16 (127 + 3S) bounds tile-relative positions;
wc = S^2, ws = m^2 with the 8-bit colour scale (ws * 4^(bd-8) above 8 bits, wc * 4^(8-bd) below),
wc', ws' the gcd-reduced weights. The staged cell is a = (K, -2 ws' x_k, -2 ws' y_k, -2 wc' Y_k),
b = (-2 wc' Cb_k, -2 wc' Cr_k) with K = wc' |c_k|^2 + ws' |x_k|^2.
"""
from __future__ import annotations

import itertools
import math

TILE_W = 128


def weights(S, m, bd):
    wc, ws = S * S, m * m
    if bd > 8:
        ws <<= 2 * (bd - 8)
    if bd < 8:
        wc <<= 2 * (8 - bd)
    g = math.gcd(wc, ws)
    return wc // g, ws // g


def form(S, m, bd):
    wcn, wsn = weights(S, m, bd)
    vmax, dmax, R = 16 * ((1 << bd) - 1), 48 * S, 16 * (TILE_W - 1 + 3 * S)
    direct = wcn * 3 * vmax * vmax + wsn * 2 * dmax * dmax
    dot = wcn * 3 * vmax * vmax + wsn * 6 * R * R
    if dot < (1 << 31):
        return "DOT32"
    if direct < (1 << 32):
        return "NARROW"
    return "WIDE" if bd <= 11 else "WIDE_COLOUR"


def partial_sums(wcn, wsn, xk, yk, ck, vx, vy, v):
    K = wcn * sum(c * c for c in ck) + wsn * (xk * xk + yk * yk)
    terms = [vx * (-2 * wsn * xk), vy * (-2 * wsn * yk), v[0] * (-2 * wcn * ck[0]), v[1] * (-2 * wcn * ck[1]),
             v[2] * (-2 * wcn * ck[2])]
    out, acc = [K], K
    for t in terms:
        acc += t
        out.append(acc)
    return out


def test_dot32_partial_sums_fit_in_32_bits_wherever_the_host_picks_it():
    n_dot = 0
    for bd in (6, 8, 10, 12):
        for S in (1, 2, 3, 5, 8, 10, 13, 16, 24, 32, 64):
            for m in (0, 1, 5, 10, 40):
                if form(S, m, bd) != "DOT32":
                    continue
                n_dot += 1
                wcn, wsn = weights(S, m, bd)
                vmax, R = 16 * ((1 << bd) - 1), 16 * (TILE_W - 1 + 3 * S)
                ext_pos, ext_pix, ext_col = (-R, R), (0, 16 * (TILE_W - 1)), (0, vmax)
                for xk, yk, vx, vy in itertools.product(ext_pos, ext_pos, ext_pix, ext_pix):
                    for ck in itertools.product(ext_col, repeat=3):
                        for v in itertools.product(ext_col, repeat=3):
                            for p in partial_sums(wcn, wsn, xk, yk, ck, vx, vy, v):
                                assert abs(p) < (1 << 31), (S, m, bd, xk, yk, ck, vx, vy, v)
    assert n_dot > 20


def test_benchmark_workloads_take_the_documented_forms():
    assert form(10, 5, 10) == "DOT32"   # 1920x1080 views, S = 10, 10-bit
    assert form(13, 5, 10) == "WIDE"    # 3840x2160 views, S = 13, 10-bit
    assert form(11, 5, 12) in ("WIDE", "WIDE_COLOUR", "NARROW")
    assert form(11, 5, 16) == "WIDE_COLOUR"
