"""The oracle's Philox4x32-10 against cuRAND's device generator at counters
whose third and fourth words (cuRAND's subsequence) are at or above 2^32,
which the host generator never reaches: the fourth word carries a draw's
purpose.  The helper kernel is built here from its source."""
import ctypes
import subprocess

import numpy as np
import pytest

import oracle

from conftest import ROOT

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = tmp_path_factory.mktemp("curand") / "libcurand_blocks.so"
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-Xcompiler", "-fPIC",
                    "-o", str(out), f"{ROOT}/tests/curand_philox_blocks.cu"], check=True)
    h = ctypes.CDLL(str(out))
    h.curand_philox_blocks.restype = ctypes.c_int
    h.curand_philox_blocks.argtypes = [ctypes.c_ulonglong, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.c_void_p]
    return h


@pytest.mark.parametrize("seed", [1, 0xDEADBEEF12345678, 2**64 - 1])
def test_philox_matches_curand_device_high_subsequences(lib, seed):
    subseq = [2**32, 2**32 + 5, 3 * 2**32 + 1, 2**63 + 1, 2**64 - 1, 0x7FFFFFFF00000002, 2, 0]
    offset = [0, 4 * 7, 4 * 2**33 + 8, 4 * (2**32 - 1), 0, 4 * 123456789, 4 * 2**40, 4 * 3]
    s = np.array(subseq, dtype=np.uint64)
    o = np.array(offset, dtype=np.uint64)
    out = np.zeros(4 * len(subseq), dtype=np.uint32)
    assert lib.curand_philox_blocks(seed, s.ctypes.data, o.ctypes.data, len(subseq), out.ctypes.data) == 0
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i, (sq, off) in enumerate(zip(subseq, offset)):
        c = off // 4
        ctr = [c & 0xFFFFFFFF, c >> 32, sq & 0xFFFFFFFF, sq >> 32]
        got = oracle.philox4x32_10(ctr, key)
        assert (np.array(got, dtype=np.uint32) == out[4 * i:4 * i + 4]).all(), (seed, sq, off)
