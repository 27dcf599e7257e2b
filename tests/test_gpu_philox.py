"""The Philox4x32-10 stream, pinned on the GPU.

1. The oracle's Philox equals cuRAND's Philox4_32_10 generator (a library
   implementation of the same published algorithm, Salmon et al. SC'11) for
   the same key and counter.  cuRAND's curand_init(seed, subsequence, offset)
   starts at counter (offset/4 as a 64-bit pair, subsequence as a 64-bit
   pair) under key (seed_lo, seed_hi); curand4 returns the four words there.
2. The library's device Philox (rosen_philox) equals the oracle's.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest
import torch

import oracle
from paper_1704_04381_gb300 import build as pkg_build

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))

CURAND_PROBE = r"""
#include <curand_kernel.h>
#include <stdint.h>
__global__ void k(unsigned long long seed, const unsigned long long *sub,
                  const unsigned long long *off, uint4 *out, int n) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    curandStatePhilox4_32_10_t st;
    curand_init(seed, sub[q], off[q], &st);
    out[q] = curand4(&st);
}
extern "C" int run(unsigned long long seed, const unsigned long long *sub,
                   const unsigned long long *off, uint4 *out, int n) {
    k<<<(n + 127) / 128, 128>>>(seed, sub, off, out, n);
    return (int)cudaDeviceSynchronize();
}
"""


@pytest.fixture(scope="module")
def curand_probe(tmp_path_factory):
    d = tmp_path_factory.mktemp("curand")
    src = d / "probe.cu"
    src.write_text(CURAND_PROBE)
    so = d / "probe.so"
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-shared",
                    "-Xcompiler", "-fPIC", "-o", str(so), str(src)], check=True)
    lib = ctypes.CDLL(str(so))
    lib.run.argtypes = [ctypes.c_ulonglong, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                        ctypes.c_int]
    return lib


def test_oracle_philox_equals_curand(curand_probe):
    rng = np.random.default_rng(0)
    n = 512
    seed = 0x0123456789ABCDEF
    sub = rng.integers(0, 2 ** 63, size=n, dtype=np.uint64)
    sub[:8] = np.arange(8)
    blocks = rng.integers(0, 2 ** 40, size=n, dtype=np.uint64)
    blocks[:8] = 0
    off = blocks * np.uint64(4)
    t_sub = torch.from_numpy(sub.view(np.int64)).cuda()
    t_off = torch.from_numpy(off.view(np.int64)).cuda()
    out = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    assert curand_probe.run(seed, t_sub.data_ptr(), t_off.data_ptr(), out.data_ptr(), n) == 0
    got = out.cpu().numpy().view(np.uint32)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for q in range(n):
        b, s = int(blocks[q]), int(sub[q])
        ctr = [b & 0xFFFFFFFF, b >> 32, s & 0xFFFFFFFF, s >> 32]
        assert np.array_equal(oracle.philox4x32_10(ctr, key), got[q]), q


def test_device_philox_equals_oracle():
    pkg_build.build()
    from paper_1704_04381_gb300 import rosen
    n = 3000
    out = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    seed = 987654321987
    rosen.rosen_philox(seed, 7, 33, 2, 2 ** 32 - n, n, out)
    got = out.cpu().numpy().view(np.uint32)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for q in range(0, n, 7):
        ctr = [2 ** 32 - n + q, 7, 33, 2]
        assert np.array_equal(oracle.philox4x32_10(ctr, key), got[q]), q
