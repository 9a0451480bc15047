"""The coefficient tables of the six-directional stencil (csrc/hex6_tables.h):
the committed header is what its generator writes, and the integer facts the
stencil's exact arithmetic relies on hold for it.

The stencil evaluates F(y) = sum_ab A_ab sigma^a tau^b / HEX6_DEN per tap with
A_ab = sum_k c_abk g[m_k] over the 24 window values of the tap's piece.  It
adds -HEX6_CMIN to every coefficient (unsigned 32 x 32 -> 64-bit multiply-adds
of 32-bit limbs) and removes the offset with the plain sum of the 24 values;
it offsets the window values by 2^95 and removes that offset with
sum_k c_abk, which is HEX6_DEN for the constant term and 0 for the others
(the partition of unity of the element)."""
import importlib.util
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1003_2022_gb300", "csrc")


def _table():
    s = open(os.path.join(CSRC, "hex6_tables.h")).read()
    i = s.index("HEX6_ICOEF[HEX6_NREGION]")
    body = s[s.index("= {", i) + 1:s.index("};", i)]
    c = np.array([int(x) for x in re.findall(r"-?\d+", body)]).reshape(12, 24, 16)
    den = int(re.search(r"#define HEX6_DEN (\d+)", s).group(1))
    cmin = int(re.search(r"#define HEX6_CMIN \((-?\d+)\)", s).group(1))
    return c, den, cmin


def test_committed_header_is_the_generators_output():
    spec = importlib.util.spec_from_file_location("hex6_gen", os.path.join(CSRC, "hex6_gen.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    assert gen.emit(None) == open(os.path.join(CSRC, "hex6_tables.h")).read()


def test_integer_facts_of_the_table():
    c, den, cmin = _table()
    assert den == 432
    assert c.min() == cmin and not c[..., 15].any()
    sums = c.sum(axis=1)                      # per piece, per monomial, over the 24 slots
    assert np.all(sums[:, 0] == den) and not sums[:, 1:].any()
    # unsigned limb products: (c - cmin) * (2^32 - 1), summed over 24 slots, in 64 bits
    assert (c - cmin).max() * (2**32 - 1) * 24 < 2**64
    # the offset sum of a limb, times -cmin, also in 64 bits
    assert -cmin * (2**32 - 1) * 24 < 2**63
