"""Measure the arithmetic-pipe peaks of the current GPU (float32/float64 FMA, ex2, IMAD).

    python -m paper_2603_24688_gb300.peaks

Compiles csrc/probe_peaks.cu for sm_103a and runs it twice (the second run is the
reported one); the figures back the "alu" roofline of the pair kernels.
"""
import os
import shutil
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = os.path.join(tempfile.mkdtemp(), "probe_peaks")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                    os.path.join(HERE, "csrc", "probe_peaks.cu")], check=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    sys.stdout.write(r.stdout)
    return r.returncode


if __name__ == "__main__":
    sys.exit(main())
