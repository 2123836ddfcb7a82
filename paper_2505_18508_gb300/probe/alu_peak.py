"""Build and run the integer-pipe peak probe (probe/alu_peak.cu) on GPU 0.

    python -m paper_2505_18508_gb300.probe.alu_peak

Prints ops per clock per SM and Tops/s for mad.lo, mul.wide, lop3 and
Philox4x32-10 blocks.  These are the denominators of the annealer's "alu"
roofline (the measured-peaks file covers only HBM and bf16 tensor work).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    out_dir = os.path.join(os.path.dirname(HERE), "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "alu_peak")
    from paper_2505_18508_gb300.build import nvcc, ARCH
    subprocess.run([nvcc(), *ARCH, "-O3", "-o", exe, os.path.join(HERE, "alu_peak.cu")], check=True)
    r = subprocess.run([exe], check=False)
    return r.returncode


if __name__ == "__main__":
    sys.exit(main())
