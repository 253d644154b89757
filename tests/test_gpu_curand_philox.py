"""The oracle's Philox-4x32-10 against CUDA's own curand_Philox4x32_10, run on the GPU.

The oracle writes the generator from the SC'11 definition (Salmon et al.,
"Parallel Random Numbers: As Easy as 1, 2, 3"); the noise of Sec. 3.5 draws
one block per (cone, step) with counter (cone, step, 0, 0) and key (seed low
word, seed high word).  A second, independent implementation of the same
function ships with the CUDA toolkit's device headers; this test compiles a
one-line kernel around it and compares every output word with the oracle's,
bit for bit, on the counters the noise uses and on random 128-bit counters and
64-bit keys.
"""
import ctypes as ct
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

_PROBE = r"""
#include <cstdint>
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void philox_words(const uint4 *ctr, const uint2 *key, uint4 *out, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

// h_ctr: n x 4 words, h_key: n x 2 words, h_out: n x 4 words (host memory).
extern "C" int curand_philox_words(const uint32_t *h_ctr, const uint32_t *h_key, uint32_t *h_out, int n)
{
    if (n <= 0) return 0;
    uint4 *d_ctr = nullptr, *d_out = nullptr;
    uint2 *d_key = nullptr;
    cudaError_t e = cudaMalloc(&d_ctr, sizeof(uint4) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&d_out, sizeof(uint4) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&d_key, sizeof(uint2) * (size_t)n);
    if (e == cudaSuccess) e = cudaMemcpy(d_ctr, h_ctr, sizeof(uint4) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_key, h_key, sizeof(uint2) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        philox_words<<<(n + 255) / 256, 256>>>(d_ctr, d_key, d_out, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(h_out, d_out, sizeof(uint4) * (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(d_ctr);
    cudaFree(d_out);
    cudaFree(d_key);
    return (int)e;
}
"""


@pytest.fixture(scope="module")
def curand_philox(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("curand_probe")
    src, lib = d / "probe.cu", d / "libprobe.so"
    src.write_text(_PROBE)
    subprocess.run([nvcc, "-O2", "-shared", "-Xcompiler", "-fPIC", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-o", str(lib), str(src)], check=True, capture_output=True)
    L = ct.CDLL(str(lib))
    f = L.curand_philox_words
    f.restype = ct.c_int
    f.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int]

    def run(ctr, key):
        ctr = np.ascontiguousarray(ctr, np.uint32)
        key = np.ascontiguousarray(key, np.uint32)
        out = np.zeros_like(ctr)
        rc = f(ctr.ctypes.data, key.ctypes.data, out.ctypes.data, ctr.shape[0])
        assert rc == 0, f"CUDA error {rc}"
        return out
    return run


def test_noise_counters_match_curand(curand_philox):
    """Counters (cone, step, 0, 0) over cones 0..4095 and steps 0, 1, 4999, 2^31 + 7; two seeds."""
    axon = np.arange(4096, dtype=np.uint32)
    rows_c, rows_k = [], []
    for seed in (0x5EED0002, 0xDEADBEEF12345678):
        for step in (0, 1, 4999, (1 << 31) + 7):
            c = np.zeros((axon.size, 4), np.uint32)
            c[:, 0] = axon
            c[:, 1] = step
            rows_c.append(c)
            rows_k.append(np.tile(np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32), (axon.size, 1)))
    ctr, key = np.concatenate(rows_c), np.concatenate(rows_k)
    np.testing.assert_array_equal(oracle.philox4x32_10(ctr, key), curand_philox(ctr, key))


def test_random_counters_and_keys_match_curand(curand_philox):
    rng = np.random.default_rng(2014)
    ctr = rng.integers(0, 1 << 32, (20000, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 1 << 32, (20000, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 0, 0, 0], [0, 0, 0, 1]]
    key[:4] = [[0, 0], [0xFFFFFFFF, 0xFFFFFFFF], [0, 0], [0, 0]]
    np.testing.assert_array_equal(oracle.philox4x32_10(ctr, key), curand_philox(ctr, key))
