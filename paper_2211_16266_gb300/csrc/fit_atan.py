"""Fit the arctangent polynomial used by the device projection (fast_atan2).

atan(r) on r in [0, 1] is approximated as r * P(r^2) with P of degree n,
minimising the maximum absolute error by the Remez exchange algorithm
(E. Remez, 1934; see e.g. Muller, "Elementary Functions", ch. 3). In the
variable s = r^2 the target is g(s) = atan(sqrt(s)) / sqrt(s) with weight
sqrt(s). The script prints the coefficients, the minimax error in exact
arithmetic and the error of the FP32 Horner evaluation the kernel performs,
and with --write regenerates atan_coeffs.cuh next to it.
"""
from __future__ import annotations

import argparse
import os

import mpmath as mp
import numpy as np

mp.mp.dps = 40


def target(s):
    s = mp.mpf(s)
    if s == 0:
        return mp.mpf(1)
    r = mp.sqrt(s)
    return mp.atan(r) / r


def weight(s):
    return mp.sqrt(mp.mpf(s))


def solve(ref, n):
    # sum_k c_k s_i^k - (-1)^i E / w(s_i) = g(s_i)
    m = n + 2
    A = mp.matrix(m, m)
    b = mp.matrix(m, 1)
    for i, s in enumerate(ref):
        for k in range(n + 1):
            A[i, k] = mp.mpf(s) ** k
        A[i, n + 1] = -((-1) ** i) / weight(s)
        b[i] = target(s)
    x = mp.lu_solve(A, b)
    return [x[k] for k in range(n + 1)], x[n + 1]


def err_fn(c, s):
    p = mp.mpf(0)
    for ck in reversed(c):
        p = p * s + ck
    return weight(s) * (p - target(s))


def remez(n, iters=30, grid=4000):
    m = n + 2
    ref = [mp.mpf((1 - mp.cos(mp.pi * (i + 0.5) / m)) / 2) for i in range(m)]
    xs = [mp.mpf(i) / grid for i in range(1, grid + 1)]
    for _ in range(iters):
        c, E = solve(ref, n)
        e = [err_fn(c, s) for s in xs]
        # alternating extrema: split the grid at sign changes, keep the largest of each run
        runs, cur = [], [0]
        for i in range(1, len(xs)):
            if mp.sign(e[i]) == mp.sign(e[cur[-1]]):
                cur.append(i)
            else:
                runs.append(cur)
                cur = [i]
        runs.append(cur)
        ext = [max(r, key=lambda i: abs(e[i])) for r in runs]
        while len(ext) > m:  # drop the smallest end extremum
            if abs(e[ext[0]]) < abs(e[ext[-1]]):
                ext = ext[1:]
            else:
                ext = ext[:-1]
        if len(ext) < m:
            break
        new = [xs[i] for i in ext]
        if max(abs(a - b) for a, b in zip(new, ref)) < mp.mpf(10) ** -12:
            ref = new
            break
        ref = new
    c, E = solve(ref, n)
    return [float(ck) for ck in c], float(abs(E))


def fp32_error(c, count=2_000_001):
    r = np.linspace(0.0, 1.0, count).astype(np.float32)
    s = (r * r).astype(np.float32)
    p = np.float32(c[-1])
    for ck in reversed(c[:-1]):
        p = (p * s + np.float32(ck)).astype(np.float32)
    a = (p * r).astype(np.float32)
    exact = np.arctan(r.astype(np.float64))
    return float(np.max(np.abs(a.astype(np.float64) - exact)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--degree", type=int, default=7)
    ap.add_argument("--write", action="store_true")
    a = ap.parse_args()
    c, E = remez(a.degree)
    e32 = fp32_error(c)
    print(f"degree {a.degree}: minimax error {E:.3e}, FP32 Horner error {e32:.3e}")
    for k, ck in enumerate(c):
        print(f"  c{k} = {ck!r}")
    if a.write:
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "atan_coeffs.cuh")
        with open(path, "w") as f:
            f.write("// Generated by fit_atan.py (Remez minimax fit of atan(r) = r * P(r^2) on [0, 1]).\n")
            f.write(f"// Degree {a.degree} in r^2; minimax error {E:.3e} rad, FP32 Horner error {e32:.3e} rad.\n")
            f.write("#pragma once\n\nnamespace pmsp {\n\n")
            f.write("// P(s), s = r^2, by Horner's rule.\n")
            f.write("__device__ __forceinline__ float atan_poly(float s) {\n")
            f.write(f"    float p = {float(np.float32(c[-1]))!r}f;\n")
            for ck in reversed(c[:-1]):
                f.write(f"    p = fmaf(p, s, {float(np.float32(ck))!r}f);\n")
            f.write("    return p;\n}\n\n")
            f.write("// 2 P(s): 2 atan(q) = q * 2 P(q^2) for |q| <= 1 (coefficients doubled, which is exact).\n")
            f.write("__device__ __forceinline__ float atan2x_poly(float s) {\n")
            f.write(f"    float p = {float(np.float32(2 * c[-1]))!r}f;\n")
            for ck in reversed(c[:-1]):
                f.write(f"    p = fmaf(p, s, {float(np.float32(2 * ck))!r}f);\n")
            f.write("    return p;\n}\n\n")
            f.write("// 2 P(s) for two pairs of lanes at once, packed FP32 FMAs interleaved so each\n")
            f.write("// coefficient pair serves both: 2 atan(q) = q * 2 P(q^2) for |q| <= 1, the form\n")
            f.write("// the paired projection uses (coefficients doubled, which is exact).\n")
            f.write("__device__ __forceinline__ void atan2x_poly2_dual(float2 s1, float2 s2, float2& p1, float2& p2) {\n")
            v = float(np.float32(2 * c[-1]))
            f.write(f"    p1 = make_float2({v!r}f, {v!r}f);\n")
            f.write("    p2 = p1;\n")
            for ck in reversed(c[:-1]):
                v = float(np.float32(2 * ck))
                f.write(f"    p1 = __ffma2_rn(p1, s1, make_float2({v!r}f, {v!r}f));\n")
                f.write(f"    p2 = __ffma2_rn(p2, s2, make_float2({v!r}f, {v!r}f));\n")
            f.write("}\n\n}  // namespace pmsp\n")
        print("wrote", path)


if __name__ == "__main__":
    main()
