"""The complex64 tables' potential phase factor exp(-i A tau/hbar) (Sec. 2.1, eq.
(splitop)) as computed on the device (csrc/wp_phase_ff.cuh: the argument reduced modulo
pi/2 in FP64, cosine and sine as float-float Taylor series), compiled for the host
(tests/phase_ff_host.cpp) and checked against numpy's FP64 cosine and sine: every quadrant,
arguments on and next to the multiples of pi/4 and pi/2, large arguments and the FP64
fallback beyond 2^20. The bound is the precision of a table record (high + low FP32
parts, about 48 significant bits); the pairs must be normalised (|lo| <= ulp(hi) / 2)."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1306_3247_gb300", "csrc")
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")


@pytest.fixture(scope="module")
def cis_host(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("no C++ compiler or CUDA headers")
    exe = str(tmp_path_factory.mktemp("phase") / "phase_ff_host")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, "-I", CUDA_INC,
                    os.path.join(ROOT, "tests", "phase_ff_host.cpp"), "-o", exe], check=True)

    def run(theta):
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        inp = struct.pack("q", theta.size) + theta.tobytes()
        out = subprocess.run([exe], input=inp, capture_output=True, check=True).stdout
        return np.frombuffer(out, dtype=np.float32).reshape(-1, 4)

    return run


def arguments():
    rng = np.random.default_rng(3247)
    q = np.arange(-400, 401)
    near = np.concatenate([q * (np.pi / 4) + d for d in (0.0, 1e-12, -1e-12, 1e-6, -1e-6)])
    return np.concatenate([
        [0.0, -0.0, np.pi / 4, -np.pi / 4, np.pi / 2, np.pi, 3 * np.pi / 2],
        rng.uniform(-np.pi / 4, np.pi / 4, 20000),
        rng.uniform(-10.0, 10.0, 20000),
        rng.uniform(-1e3, 1e3, 20000),
        rng.uniform(-1e5, 1e5, 20000),
        rng.uniform(-1e6, 1e6, 2000),
        [2.0 ** 21, -(2.0 ** 21) - 0.5, 1e9],
        near,
    ])


def test_phase_factor_matches_fp64_cos_sin(cis_host):
    th = arguments()
    r = cis_host(th).astype(np.float64)
    c = r[:, 0] + r[:, 1]
    s = r[:, 2] + r[:, 3]
    err = np.maximum(np.abs(c - np.cos(th)), np.abs(s - np.sin(th)))
    print(f"largest |cos|, |sin| error {err.max():.3e} over {th.size} arguments")
    assert err.max() < 2.0 ** -45
    # |cos|^2 + |sin|^2 = 1 to the same precision: no modulus bias in the records
    assert np.max(np.abs(c * c + s * s - 1.0)) < 2.0 ** -44


def test_phase_pairs_are_normalised(cis_host):
    r = cis_host(arguments())
    for hi, lo in ((r[:, 0], r[:, 1]), (r[:, 2], r[:, 3])):
        ulp = np.spacing(np.abs(hi)).astype(np.float64)
        assert np.all(np.abs(lo.astype(np.float64)) <= 0.5 * ulp)


def test_zero_argument_is_exact(cis_host):
    r = cis_host(np.array([0.0]))
    assert r[0].tolist() == [1.0, 0.0, 0.0, 0.0]
