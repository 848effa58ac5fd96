"""Pins for oracle.philox: curand's own Philox4x32-10, the uniform mapping and Box–Muller moments."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import philox

HELPER = os.path.join(os.path.dirname(__file__), "helpers", "curand_philox_host.cu")


@pytest.fixture(scope="module")
def curand_philox():
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available to build the curand host driver")
    tmp = tempfile.mkdtemp()
    exe = os.path.join(tmp, "cph")
    subprocess.run([nvcc, "-o", exe, HELPER], check=True, cwd=tmp, capture_output=True)

    def run(rows):
        inp = "\n".join(" ".join(str(int(v)) for v in r) for r in rows) + "\n"
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
        return np.array([[int(v) for v in line.split()] for line in out.strip().splitlines()], dtype=np.uint64)

    yield run
    shutil.rmtree(tmp, ignore_errors=True)


def test_philox_matches_curand(curand_philox):
    rng = np.random.default_rng(7)
    rows = [[0, 0, 0, 0, 0, 0], [0xFFFFFFFF] * 6, [1, 2, 3, 4, 5, 6]]
    rows += rng.integers(0, 2 ** 32, size=(200, 6), dtype=np.uint64).tolist()
    rows += [[j, 17, 3, 1, 123456789, 0] for j in range(50)]
    ref = curand_philox(rows)
    rows = np.array(rows, dtype=np.uint64)
    got = np.concatenate([philox.philox4x32_10(r[None, :4], (int(r[4]), int(r[5]))) for r in rows])
    np.testing.assert_array_equal(got.astype(np.uint64), ref)


def test_uniform_mapping_exact_and_open():
    x = np.array([0, 1, 511, 512, 2 ** 31, 2 ** 32 - 1], dtype=np.uint64)
    u = philox.to_uniform(x)
    assert np.all(u > 0) and np.all(u < 1)
    assert np.all(u.astype(np.float32).astype(np.float64) == u)      # exact in float32
    assert u[0] == 2.0 ** -24 and u[-1] == 1 - 2.0 ** -24
    assert u[2] == u[0] and u[3] == 3 * 2.0 ** -24


def test_box_muller_moments():
    z = philox.normals4(np.arange(250000), step=3, chain=1, stream=0, seed=42).ravel()
    n = z.size
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / n)
    kurt = np.mean(z ** 4) / np.mean(z ** 2) ** 2
    assert abs(kurt - 3) < 5 * np.sqrt(24 / n)
    # the four slots are uncorrelated
    zz = philox.normals4(np.arange(100000), 0, 0, 1, 5)
    c = np.corrcoef(zz.T)
    assert np.max(np.abs(c - np.eye(4))) < 5 / np.sqrt(100000)


def test_counter_words_change_output():
    base = philox.normals4(np.arange(64), 0, 0, 0, 1)
    for kw in [dict(step=1, chain=0, stream=0, seed=1), dict(step=0, chain=1, stream=0, seed=1),
               dict(step=0, chain=0, stream=1, seed=1), dict(step=0, chain=0, stream=0, seed=2),
               dict(step=0, chain=0, stream=0, seed=1 + 2 ** 32)]:
        other = philox.normals4(np.arange(64), **kw)
        assert abs(np.corrcoef(base.ravel(), other.ravel())[0, 1]) < 0.2
