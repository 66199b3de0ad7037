"""Pins the oracle's Philox4x32-10 to NVIDIA's curand implementation of the
same published generator (Salmon et al., SC'11), by running curand.

curand_init(seed, subsequence, offset) keys the generator with the 64-bit
seed and starts the 128-bit counter at (offset/4) + subsequence * 2^64, i.e.
words (x, y) = offset/4 and (z, w) = subsequence; curand4 returns the block
for that counter. The library draws pixel p of frame t of stream s from the
block with counter (p/4, t, s, 0), so subsequence = s and offset/4 = t*2^32 + p/4.
"""
import ctypes as C
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SRC = r"""
#include <curand_kernel.h>
#include <cuda_runtime.h>
__global__ void blocks(unsigned long long seed, unsigned long long sub,
                       unsigned long long first, int n, uint4* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  curandStatePhilox4_32_10_t st;
  curand_init(seed, sub, 4ull * (first + (unsigned long long)i), &st);
  out[i] = curand4(&st);
}
extern "C" int curand_blocks(unsigned long long seed, unsigned long long sub,
                             unsigned long long first, int n, unsigned int* host) {
  uint4* d = nullptr;
  if (cudaMalloc(&d, sizeof(uint4) * n) != cudaSuccess) return 1;
  blocks<<<(n + 127) / 128, 128>>>(seed, sub, first, n, d);
  cudaError_t e = cudaMemcpy(host, d, sizeof(uint4) * n, cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? 0 : 2;
}
"""


@pytest.fixture(scope="module")
def curand_lib():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    d = tempfile.mkdtemp(prefix="curand_pin_")
    src = os.path.join(d, "pin.cu")
    so = os.path.join(d, "libpin.so")
    open(src, "w").write(SRC)
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                    "-Xcompiler", "-fPIC", "-o", so, src], check=True)
    lib = C.CDLL(so)
    lib.curand_blocks.argtypes = [C.c_ulonglong, C.c_ulonglong, C.c_ulonglong, C.c_int, C.c_void_p]
    lib.curand_blocks.restype = C.c_int
    return lib


@pytest.mark.parametrize("seed,stream,t,q0", [(0, 0, 0, 0), (0xDEADBEEF12345678, 77, 5, 1000),
                                               (1, 3, 239, 2073599), (2 ** 64 - 1, 2 ** 32 - 1, (1 << 30) - 1, 7)])
def test_oracle_philox_equals_curand(orc, curand_lib, seed, stream, t, q0):
    n = 256
    got = np.empty((n, 4), np.uint32)
    assert curand_lib.curand_blocks(seed, stream, (t << 32) + q0, n, got.ctypes.data) == 0
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(n):
        q = q0 + i
        ref = orc.philox([q & 0xFFFFFFFF, t + (q >> 32), stream, 0], key)
        assert np.array_equal(got[i], ref), f"block {i}"
