"""The FP64 fused multiply-add butterflies and their twiddle records (wp_fft_f64.h),
compiled for the host with the Stockham stage order and index map of the fixed-size
device transform (tests/fft_f64_host.cpp), against numpy's FFT: the DFT behind the
Fourier transforms of eq. (ft) (Sec. 2.1), X_k = sum_j x_j exp(-+ 2 pi i j k / n),
forward and inverse (unnormalised), for every length the fixed-size kernels take and the
shorter ones."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1306_3247_gb300", "csrc")


@pytest.fixture(scope="module")
def fft_host(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("fft") / "fft_f64_host")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "fft_f64_host.cpp"), "-o", exe], check=True)

    def run(x, inv):
        logn = int(np.log2(len(x)))
        inp = struct.pack("ii", logn, 1 if inv else 0) + np.ascontiguousarray(x, dtype=np.complex128).tobytes()
        out = subprocess.run([exe], input=inp, capture_output=True, check=True).stdout
        return np.frombuffer(out, dtype=np.complex128)

    return run


@pytest.mark.parametrize("logn", list(range(1, 15)))
def test_fma_transform_matches_dft(fft_host, logn):
    rng = np.random.default_rng(100 + logn)
    n = 1 << logn
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for inv in (False, True):
        got = fft_host(x, inv)
        ref = np.fft.ifft(x) * n if inv else np.fft.fft(x)
        # a rounding error of a few ulps per stage; a wrong sign, index or record is O(1)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-15 * logn, (logn, inv)


def test_fma_transform_unit_impulses(fft_host):
    # the DFT of e_m is the twiddle row exp(-+ 2 pi i m k / n): every record of every stage
    n = 256
    k = np.arange(n)
    for m in (0, 1, 3, 37, 64, 127, 128, 255):
        x = np.zeros(n, complex)
        x[m] = 1.0
        for inv in (False, True):
            ref = np.exp((2j if inv else -2j) * np.pi * ((m * k) % n) / n)  # exact reduction
            assert np.max(np.abs(fft_host(x, inv) - ref)) < 4e-16 * 8, (m, inv)


def test_fma_round_trip_keeps_the_norm(fft_host):
    # forward then inverse / n: the identity, with no systematic change of the norm
    rng = np.random.default_rng(7)
    n = 256
    drift = []
    for _ in range(40):
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        y = fft_host(fft_host(x, False), True) / n
        assert np.max(np.abs(y - x)) < 2e-15 * np.max(np.abs(x))
        drift.append(np.linalg.norm(y) / np.linalg.norm(x) - 1.0)
    assert abs(np.mean(drift)) < 1e-16
