"""The register DFT codelets of the CUDA kernels (csrc/ils_dft.cuh) on the host, and the
warp-pair four-step decomposition built from them.

The codelets are __host__ __device__; a small host program (tests/host/dft_codelets.cu)
runs every supported size in both directions and compares with a brute-force DFT in
double precision.  A wrong prime-factor index map, twiddle or sign gives an O(1) error.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_register_dfts_match_bruteforce(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "dftc")
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I",
                    os.path.join(ROOT, "paper_2003_07504_gb300", "csrc"), "-x", "cu",
                    os.path.join(ROOT, "tests", "host", "dft_codelets.cu"), "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    sizes = {}
    for line in out:
        if line.strip():
            r, ef, ei = line.split()
            sizes[int(r)] = (float(ef), float(ei))
    assert set(sizes) >= {2, 3, 4, 5, 6, 8, 9, 10, 12, 15, 16, 20, 24, 25, 27, 30, 32, 36, 40, 45, 48, 54, 60, 64}
    for r, (ef, ei) in sizes.items():
        assert ef < 5e-7 and ei < 5e-7, (r, ef, ei)


def test_warp_pair_four_step_decomposition(tmp_path):
    # the 64 x 30 four-step with a radix-2 join of two 32-point halves that the warp-pair row
    # kernels run for 3840-wide rows, emulated on the host with the same codelets and a
    # 64-wide four-step twiddle table (tests/host/pair_four_step.cu), against a brute-force DFT
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "pfs")
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I",
                    os.path.join(ROOT, "paper_2003_07504_gb300", "csrc"), "-x", "cu",
                    os.path.join(ROOT, "tests", "host", "pair_four_step.cu"), "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    errs = dict((d, float(e)) for d, e in (line.split() for line in out if line.strip()))
    assert set(errs) == {"forward", "inverse"}
    for d, e in errs.items():
        assert e < 1e-6, (d, e)
