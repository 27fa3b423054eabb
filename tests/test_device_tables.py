"""The constant tables of the device math in bh_common.cuh, checked on the CPU:
the 2^(j/32) table of d_exp and the reduction tables of the FP64 d_log1p
(factors r_j and T_j = -log r_j - s_j ln 2 as hi + lo) against values computed
here at 40 digits, and the log tables against their generator script."""
import math
import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2605_05635_gb300", "csrc")


def _table(name):
    src = open(os.path.join(CSRC, "bh_common.cuh")).read()
    m = re.search(r"static __device__ const double " + name + r"\[(\d+)\] = \{(.*?)\};", src, re.S)
    assert m, name
    vals = [float(v) for v in m.group(2).replace("\n", " ").split(",") if v.strip()]
    assert len(vals) == int(m.group(1))
    return vals


def test_exp2_table_is_nearest():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for j, v in enumerate(_table("kExp2Tab")):
        assert v == float(mp.mpf(2) ** (mp.mpf(j) / 32)), j


def test_log_tables_reduce_and_are_exact():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    R, TH, TL = _table("kLogR"), _table("kLogTHi"), _table("kLogTLo")
    assert R[0] == 1.0 and R[63] == 0.5 and TH[0] == TH[63] == 0.0
    for j in range(64):
        # every m in the bin [1 + j/64, 1 + (j+1)/64) reduces to |m r_j - 1| <= 1/64
        for m in (1 + j / 64, 1 + (j + 1) / 64 - 2.0 ** -52):
            assert abs(m * R[j] - 1) <= 1 / 64 + 1e-16, (j, m)
        s = 1 if j >= 32 else 0
        t = -mp.log(mp.mpf(R[j])) - s * mp.log(2)
        assert TH[j] == float(t), j
        assert abs(mp.mpf(TH[j]) + mp.mpf(TL[j]) - t) <= mp.mpf(2) ** -106 * max(1, abs(t)), j
        # and, independently of mpmath, within a few units of double log
        assert abs(TH[j] - (-math.log(R[j]) - s * math.log(2))) <= 4e-16, j


def test_log_tables_match_generator():
    pytest.importorskip("mpmath")
    sys.path.insert(0, CSRC)
    try:
        import gen_log_table
    finally:
        sys.path.remove(CSRC)
    r, hi, lo = gen_log_table.tables()
    assert _table("kLogR") == r
    assert _table("kLogTHi") == hi
    assert _table("kLogTLo") == lo
