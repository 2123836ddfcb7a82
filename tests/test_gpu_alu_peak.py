"""The denominator of the annealer's "alu" roofline, measured.

bench.py reports the persistent kernel against 64 IMAD lanes per SM per clock
(4 sub-partitions x 16 lanes; a 32x32->64 multiply takes two lane slots) and
at most 64 / 40 = 1.6 Philox4x32-10 blocks per SM per clock (20 wide
multiplies each).  tests/alu_peak.cu measures both with one 1024-thread CTA
per SM, counting SM cycles with clock64 so that the figures do not depend on
the clock: this test checks that the unit counts the roofline assumes are the
ones the GPU delivers (within 3 %), and that pure Philox does not beat them.
Run with -s to see the table.
"""
import os
import re
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "alu_peak.cu")
EXE = os.path.join(ROOT, "tests", "_build", "alu_peak")


def test_integer_pipe_peaks_match_the_roofline_unit_counts():
    from paper_2505_18508_gb300 import build
    exe = build.build_program(SRC, EXE)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120, check=True).stdout
    print(out)
    per_clk = {m.group(1): float(m.group(2)) for m in re.finditer(r"^(\S+)\s+([0-9.]+) ops/clk/SM", out, re.M)}
    assert set(per_clk) == {"mad.lo", "mul.wide", "lop3", "philox"}
    assert abs(per_clk["mad.lo"] - 64.0) <= 0.03 * 64.0
    assert abs(per_clk["mul.wide"] - 32.0) <= 0.05 * 32.0       # two lane slots per wide multiply
    assert per_clk["philox"] <= 1.6 * 1.01                      # 20 wide multiplies per block
    assert per_clk["philox"] >= 0.8 * 1.6
