#!/usr/bin/env python3
"""Writes skew_table.inc: the collision rate of Zipf(s) over [0, 2^32) for
s = 0.30, 0.31, ..., 4.00, the table the batch planner inverts to estimate a
stream's skew from a sample (pss_estimate_skew).

For P(rank r) = r^-s / H(U, s), r = 1..U, two independent draws are equal with
probability  q(s) = H(U, 2s) / H(U, s)^2,  H(U, s) = sum_{r=1}^{U} r^-s.
H is evaluated by the Euler-Maclaurin formula: the first R - 1 terms summed,
the rest as the integral plus end corrections (Bernoulli terms to the
fifth derivative), relative error below 1e-12 for these s and U.

Run it from this directory:  python3 skew_table.py > skew_table.inc
"""
import math

U = 2.0 ** 32
R = 200
S0, STEP, COUNT = 0.30, 0.01, 371


def harmonic(n: float, s: float) -> float:
    head = sum(r ** -s for r in range(1, R))
    if abs(s - 1.0) < 1e-12:
        integral = math.log(n / R)
    else:
        integral = (n ** (1.0 - s) - R ** (1.0 - s)) / (1.0 - s)
    f = lambda x: x ** -s
    d1 = lambda x: -s * x ** (-s - 1)
    d3 = lambda x: -s * (s + 1) * (s + 2) * x ** (-s - 3)
    d5 = lambda x: -s * (s + 1) * (s + 2) * (s + 3) * (s + 4) * x ** (-s - 5)
    corr = (f(R) + f(n)) / 2 + (d1(n) - d1(R)) / 12 - (d3(n) - d3(R)) / 720 \
        + (d5(n) - d5(R)) / 30240
    return head + integral + corr


def main():
    print("// Generated by skew_table.py: collision rate q(s) = H(U, 2s) / H(U, s)^2 of")
    print(f"// Zipf(s) over U = 2^32 for s = {S0:.2f} + {STEP:.2f} i, i = 0..{COUNT - 1}.")
    print(f"constexpr double SKEW_TABLE_S0 = {S0!r}, SKEW_TABLE_STEP = {STEP!r};")
    print(f"constexpr int SKEW_TABLE_N = {COUNT};")
    print("constexpr double SKEW_TABLE_Q[SKEW_TABLE_N] = {")
    vals = []
    for i in range(COUNT):
        s = round(S0 + STEP * i, 10)
        vals.append(harmonic(U, 2 * s) / harmonic(U, s) ** 2)
    assert all(a < b for a, b in zip(vals, vals[1:])), "q(s) must increase with s"
    for i in range(0, COUNT, 4):
        print("    " + ", ".join(f"{v:.17g}" for v in vals[i:i + 4]) + ",")
    print("};")


if __name__ == "__main__":
    main()
