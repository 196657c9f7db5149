"""The device Philox4x32-10 of the CUDA path against cuRAND's device Philox4x32-10 (a library
routine, called here, not copied): every counter word and both key words are exercised."""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = r'''
#include <curand_kernel.h>
#include "ms_device.cuh"
extern "C" __global__ void both(const uint4 *ctr, const uint2 *key, uint4 *ours, uint4 *theirs,
                                int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  ours[i] = msk::philox10(ctr[i], key[i]);
  theirs[i] = curand_Philox4x32_10(ctr[i], key[i]);
}
extern "C" int run_both(const uint4 *ctr, const uint2 *key, uint4 *ours, uint4 *theirs, int n) {
  both<<<(n + 127) / 128, 128>>>(ctr, key, ours, theirs, n);
  return (int)cudaDeviceSynchronize();
}
'''


def test_device_philox_matches_curand():
    import torch

    from paper_1508_03167_gb300 import _build

    with tempfile.TemporaryDirectory() as d:
        cu = os.path.join(d, "p.cu")
        so = os.path.join(d, "p.so")
        open(cu, "w").write(SRC)
        subprocess.run([_build.nvcc_path(), "-O2", "-std=c++17", *_build.ARCH, "-shared",
                        "-Xcompiler", "-fPIC", "-I", _build.CSRC, "-o", so, cu], check=True)
        lib = ctypes.CDLL(so)
        rng = np.random.default_rng(3)
        n = 4096
        ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
        ctr[:4] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 2, 3, 4], [7, 0, 0x10005, 0]]
        key[:4] = [[0, 0], [0xFFFFFFFF] * 2, [5, 6], [7, 0]]
        c = torch.from_numpy(ctr.view(np.int32)).cuda()
        k = torch.from_numpy(key.view(np.int32)).cuda()
        ours = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
        theirs = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
        rc = lib.run_both(ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(k.data_ptr()),
                          ctypes.c_void_p(ours.data_ptr()), ctypes.c_void_p(theirs.data_ptr()),
                          n)
        assert rc == 0
        assert torch.equal(ours, theirs)
