"""The noise generator's identity against a third implementation.

The CUDA library's Philox4x32-10 and the oracle's were both written from the
published description (Salmon, Moraes, Dror, Shaw, SC'11), so a shared
misreading would pass their bit-for-bit comparison.  cuRAND's device API
implements the same generator independently; its raw words for the same key
and counter must equal both, bit for bit (see tests/curand_philox_check.cu
for how cuRAND's seed, subsequence and offset map onto key and counter)."""
import ctypes as ct
import os
import shutil
import subprocess

import numpy as np
import pytest

import paper_1411_3487_gb300 as sfp
from oracle import oracle as O
from paper_1411_3487_gb300 import build

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_lib():
    build.build()
    out_dir = os.path.join(HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "libcurand_philox_check.so")
    src = os.path.join(HERE, "curand_philox_check.cu")
    if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
        tmp = so + f".tmp{os.getpid()}"
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                        "-Xcompiler", "-fPIC", src, "-o", tmp], check=True)
        os.replace(tmp, so)
    L = ct.CDLL(so)
    L.curand_philox_words.argtypes = [ct.c_uint32, ct.c_uint32, ct.c_ulonglong, ct.c_uint32, ct.c_int,
                                      ct.c_void_p]
    return L


@pytest.mark.parametrize("seed,job,step,tag", [(0, 0, 0, 0), (1, 7, 123456789012, 0), (0xFFFFFFFF, 3, 2**40 + 5, 1),
                                               (1, 4095, 99, 0), (12345, 0xFFFFFFFF, 2**33 - 1, 2)])
def test_words_equal_curand_device_api(curand_lib, seed, job, step, tag):
    n = 4096
    ref = np.zeros((n, 4), dtype=np.uint32)
    assert curand_lib.curand_philox_words(seed, job, step, tag, n, ref.ctypes.data) == 0
    mine = sfp.philox_words(seed, job, step, tag, n)
    assert np.array_equal(mine, ref)
    for i in (0, 1, 31, 2048, n - 1):
        assert np.array_equal(O.philox4x32_10([step & 0xFFFFFFFF, step >> 32, i, tag], [seed, job]), ref[i])
