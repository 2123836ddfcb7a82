"""Build and run the integer-pipe peak probe (probe/alu_peak.cu) on GPU 0.

    python -m paper_2505_18508_gb300.probe.alu_peak

Prints ops per clock per SM and Tops/s for mad.lo, mul.wide, lop3 and
Philox4x32-10 blocks.  These are the denominators of the annealer's "alu"
roofline (the measured-peaks file covers only HBM and bf16 tensor work).
"""
import subprocess
import sys


def main():
    from paper_2505_18508_gb300.build import build_probe
    r = subprocess.run([build_probe()], check=False)
    return r.returncode


if __name__ == "__main__":
    sys.exit(main())
