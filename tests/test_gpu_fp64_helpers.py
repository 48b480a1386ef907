"""The short-chain FP64 square root / reciprocal square root used by the QL
rotation chase of the Lanczos eigensolver (Goldschmidt's iteration from an
FP32 seed) against CUDA's own sqrt on the device, across the whole exponent
range, and its refusal of the inputs it leaves to the library path."""
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <cstdio>
#include <cstdlib>
#include <cuda_runtime.h>
#include "lrp_fp64.cuh"

__global__ void k(int n, const double* t, double* sq, double* rs, double* ref_sq, int* ok) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = 0.0, b = 0.0;
  ok[i] = lrp::sqrt_rsqrt_gs(t[i], &a, &b) ? 1 : 0;
  sq[i] = a;
  rs[i] = b;
  ref_sq[i] = sqrt(t[i]);
}

int main(int argc, char** argv) {
  FILE* f = fopen(argv[1], "rb");
  int n = 0;
  if (fread(&n, sizeof(int), 1, f) != 1) return 2;
  double* h = (double*)malloc(n * sizeof(double));
  if (fread(h, sizeof(double), n, f) != (size_t)n) return 2;
  fclose(f);
  double *t, *sq, *rs, *ref;
  int* ok;
  cudaMalloc(&t, n * sizeof(double));
  cudaMalloc(&sq, n * sizeof(double));
  cudaMalloc(&rs, n * sizeof(double));
  cudaMalloc(&ref, n * sizeof(double));
  cudaMalloc(&ok, n * sizeof(int));
  cudaMemcpy(t, h, n * sizeof(double), cudaMemcpyHostToDevice);
  k<<<(n + 255) / 256, 256>>>(n, t, sq, rs, ref, ok);
  if (cudaDeviceSynchronize() != cudaSuccess) return 3;
  double* out = (double*)malloc(3 * n * sizeof(double));
  int* hok = (int*)malloc(n * sizeof(int));
  cudaMemcpy(out, sq, n * sizeof(double), cudaMemcpyDeviceToHost);
  cudaMemcpy(out + n, rs, n * sizeof(double), cudaMemcpyDeviceToHost);
  cudaMemcpy(out + 2 * n, ref, n * sizeof(double), cudaMemcpyDeviceToHost);
  cudaMemcpy(hok, ok, n * sizeof(int), cudaMemcpyDeviceToHost);
  f = fopen(argv[2], "wb");
  fwrite(out, sizeof(double), 3 * n, f);
  fwrite(hok, sizeof(int), n, f);
  fclose(f);
  return 0;
}
"""


def test_sqrt_rsqrt_gs_against_cuda_sqrt(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    src = tmp_path / "gs.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "gs"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-I",
                    os.path.join(ROOT, "paper_1703_05638_gb300", "csrc"), str(src), "-o", str(exe)], check=True)
    rng = np.random.default_rng(7)
    # positive normals over the whole exponent range, dense near 1, plus
    # the powers of two and their neighbours, then the refused inputs
    normal = np.concatenate([
        np.ldexp(rng.uniform(1.0, 2.0, 200000), rng.integers(-1022, 1024, 200000)),
        rng.uniform(0.25, 4.0, 100000),
        np.ldexp(1.0, np.arange(-1022, 1024)),
        np.nextafter(np.ldexp(1.0, np.arange(-1021, 1024)), 0.0),
        [np.finfo(np.float64).max, np.finfo(np.float64).tiny],
    ])
    refused = np.array([0.0, -0.0, -1.0, -np.finfo(np.float64).tiny, 5e-324, 1e-310, np.inf, -np.inf, np.nan])
    t = np.concatenate([normal, refused])
    inp = tmp_path / "in.bin"
    with open(inp, "wb") as f:
        f.write(np.int32(t.size).tobytes())
        f.write(t.astype(np.float64).tobytes())
    outp = tmp_path / "out.bin"
    subprocess.run([str(exe), str(inp), str(outp)], check=True)
    raw = np.fromfile(outp, dtype=np.uint8)
    n = t.size
    vals = raw[:24 * n].view(np.float64).reshape(3, n)
    ok = raw[24 * n:].view(np.int32)
    sq, rs, ref = vals
    k = normal.size
    assert np.all(ok[:k] == 1)
    assert np.all(ok[k:] == 0)
    # CUDA's double sqrt is correctly rounded: the helper stays within 2 ulp
    ulp = np.spacing(ref[:k])
    assert np.max(np.abs(sq[:k] - ref[:k]) / ulp) <= 2.0
    # 1/sqrt against the exact value from the correctly rounded root
    # (rel. error of 1/ref <= 1/2 ulp + one division rounding)
    rel = np.abs(rs[:k] * ref[:k] - 1.0)
    assert np.max(rel) <= 4 * np.finfo(np.float64).eps
