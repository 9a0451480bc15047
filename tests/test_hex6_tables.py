"""The coefficient tables of the six-directional stencil (csrc/hex6_tables.h):
the committed header is what its generator writes, and the stencil's integer
evaluation of a tap, emulated here with Python integers on the header's
tables, equals the element's pieces as the generator derives them from the
truncated power (exact rationals).

The stencil evaluates a tap of piece r at x = L_r^-1 ((sigma, tau) - v_r) in
the canonical piece: A_m = sum_k C[k][m] g_k over the 24 window values read at
the piece's offsets, the values offset by 2^95 and split into five limbs of 20
bits (the last 16), the sums in 32-bit integers; F = sum_m A_m x^m / HEX6_DEN."""
import importlib.util
import os
import re
from fractions import Fraction as Fr

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1003_2022_gb300", "csrc")


def _gen():
    spec = importlib.util.spec_from_file_location("hex6_gen", os.path.join(CSRC, "hex6_gen.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    return gen


def _ints(s, name):
    i = s.index(name)
    return [int(x) for x in re.findall(r"-?\d+", s[s.index("= {", i) + 1:s.index("};", i)])]


def _header():
    s = open(os.path.join(CSRC, "hex6_tables.h")).read()
    cc = [int(x) for x in re.findall(r"-?\d+", s[s.index("#define HEX6_CCOEF_INIT"):].split("\n", 1)[1])]
    return {
        "den": int(re.search(r"#define HEX6_DEN (\d+)", s).group(1)),
        "lut": _ints(s, "HEX6_REGION_LUT[16]"),
        "sym": np.array(_ints(s, "HEX6_SYM[HEX6_NREGION]")).reshape(12, 6),
        "di": np.array(_ints(s, "HEX6_DI[HEX6_NREGION]")).reshape(12, 24),
        "dj": np.array(_ints(s, "HEX6_DJ[HEX6_NREGION]")).reshape(12, 24),
        "cc": np.array(cc).reshape(24, 15),
        "ma": _ints(s, "HEX6_MONO_A[HEX6_NMONO]"),
        "mb": _ints(s, "HEX6_MONO_B[HEX6_NMONO]"),
    }


def test_committed_header_is_the_generators_output():
    assert _gen().emit(None) == open(os.path.join(CSRC, "hex6_tables.h")).read()


def test_integer_bounds_of_the_canonical_table():
    t = _header()
    cc = t["cc"]
    assert np.all(cc[:, 0].sum() == t["den"]) and not cc[:, 1:].sum(axis=0).any()
    # 32-bit limb sums: positive and negative parts of every column times the largest 20-bit limb
    lim = (1 << 20) - 1
    assert np.clip(cc, 0, None).sum(axis=0).max() * lim < 2**31
    assert np.clip(-cc, 0, None).sum(axis=0).max() * lim <= 2**31


def _code(s, t):
    one = 1 << 48
    if s + t < one:
        return int(s > t) | (int(2 * s + t > one) << 1) | (int(s + 2 * t > one) << 2)
    return 8 | int(s > t) | (int(2 * s + t > 2 * one) << 1) | (int(s + 2 * t > 2 * one) << 2)


def _tap_kernel(t, sf, tf, g):
    """The stencil's evaluation of one tap (cell-relative 48-bit fractions sf, tf;
    g maps lattice offsets (di, dj) to window values), times HEX6_DEN."""
    one = 1 << 48
    r = t["lut"][_code(sf, tf)]
    li = t["sym"][r]
    xs, xt = sf - int(li[4]) * one, tf - int(li[5]) * one
    x1, x2 = int(li[0]) * xs + int(li[1]) * xt, int(li[2]) * xs + int(li[3]) * xt
    assert 0 <= x1 <= one and 0 <= x2 <= one
    P = [[0] * 15 for _ in range(5)]
    for k in range(24):
        u = g[(int(t["di"][r][k]), int(t["dj"][r][k]))] + (1 << 95)
        assert 0 <= u < 1 << 96
        w = [(u >> (20 * l)) & 0xFFFFF for l in range(5)]
        for m in range(15):
            for l in range(5):
                P[l][m] += int(t["cc"][k][m]) * w[l]
    assert all(-(2**31) <= v < 2**31 for row in P for v in row)
    F = Fr(0)
    for m in range(15):
        A = sum(P[l][m] << (20 * l) for l in range(5)) - (t["den"] << 95 if m == 0 else 0)
        F += A * Fr(x1, one) ** t["ma"][m] * Fr(x2, one) ** t["mb"][m]
    return F


def test_tap_evaluation_equals_the_pieces():
    """Random taps in every piece and random 95-bit window values: the
    canonical-piece evaluation is the piece's own polynomial, exactly."""
    gen = _gen()
    samples, tables, _ = gen.build()
    t = _header()
    rng = np.random.default_rng(11)
    seen = set()
    for it in range(240):
        sf = int(rng.integers(0, 1 << 48))
        tf = int(rng.integers(0, 1 << 48))
        g = {(di, dj): int(rng.integers(-(1 << 62), 1 << 62)) << int(rng.integers(0, 33))
             for di in range(-3, 3) for dj in range(-3, 3)}
        g[(0, 0)] = -(1 << 95) if it == 0 else g[(0, 0)]
        s, tt = Fr(sf, 1 << 48), Fr(tf, 1 << 48)
        r = next(k for k, smp in enumerate(samples) if gen.region_code(*smp) == gen.region_code(s, tt))
        seen.add(r)
        ref = sum(gen.peval(p, s, tt) * g[(di, dj)] for di, dj, p in tables[r]) * t["den"]
        assert _tap_kernel(t, sf, tf, g) == ref
    assert len(seen) == 12
