"""Arithmetic facts the kernels rely on, checked on the GPU.

The FP32 compact-list walk subtracts the texel position from the lists' FP16
coordinates with the mixed-precision `sub.rn.f32.f16`, and the ray walk and
the discretization evaluate pairs of values with the packed FP32x2
instructions.  Both are claimed to give, bit for bit, what the scalar FP32
code gives: an FP16 value converts to FP32 exactly, so the mixed subtraction
is one correctly rounded FP32 subtraction; the packed FMA, multiply and add
round each component as fmaf, __fmul_rn and __fadd_rn do.  A small CUDA
program compares both forms, for every FP16 bit pattern against a set of
subtrahends and for a few million random FP32 triples.
"""

import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

SOURCE = r"""
#include <cstdio>
#include <cstring>
#include <cuda_fp16.h>

__device__ __forceinline__ bool same(float a, float b) {
    return __float_as_uint(a) == __float_as_uint(b) || (a != a && b != b);
}

// every pair of FP16 patterns (2i, 2i+1) against each subtrahend
__global__ void k_sub(const float* ps, int np, unsigned long long* bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 32768) return;
    const unsigned u = (unsigned(2 * i + 1) << 16) | unsigned(2 * i);
    __half2 h;
    memcpy(&h, &u, 4);
    const float2 f = __half22float2(h);
    for (int j = 0; j < np; ++j) {
        const float p = ps[j];
        float r0, r1;
        asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\t"
            "sub.rn.f32.f16 %0, lo, %3;\n\tsub.rn.f32.f16 %1, hi, %3;\n\t}"
            : "=f"(r0), "=f"(r1) : "r"(u), "f"(p));
        if (!same(r0, __fsub_rn(f.x, p))) atomicAdd(bad, 1ull);
        if (!same(r1, __fsub_rn(f.y, p))) atomicAdd(bad, 1ull);
    }
}

// counter-based random bits (a 32-bit mix of the index), spread over exponents
__device__ __forceinline__ float rnd(unsigned x) {
    x ^= x >> 16; x *= 0x7feb352dU; x ^= x >> 15; x *= 0x846ca68bU; x ^= x >> 16;
    const unsigned e = 97u + (x % 60u);  // exponents 2^-30 .. 2^29
    return __uint_as_float((x & 0x807fffffU) | (e << 23));
}

__global__ void k_packed(int n, unsigned long long* bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float2 a = make_float2(rnd(6 * i), rnd(6 * i + 1));
    const float2 b = make_float2(rnd(6 * i + 2), rnd(6 * i + 3));
    const float2 c = make_float2(rnd(6 * i + 4), rnd(6 * i + 5));
    const float2 f = __ffma2_rn(a, b, c), m = __fmul2_rn(a, b), s = __fadd2_rn(a, c);
    if (!same(f.x, fmaf(a.x, b.x, c.x)) || !same(f.y, fmaf(a.y, b.y, c.y))) atomicAdd(bad, 1ull);
    if (!same(m.x, __fmul_rn(a.x, b.x)) || !same(m.y, __fmul_rn(a.y, b.y))) atomicAdd(bad, 1ull);
    if (!same(s.x, __fadd_rn(a.x, c.x)) || !same(s.y, __fadd_rn(a.y, c.y))) atomicAdd(bad, 1ull);
}

int main() {
    const int np = 64;
    float hp[np];
    for (int j = 0; j < np; ++j) hp[j] = (j - 32) * 37.3125f + 0.001f * j * j - 1e-7f * j;
    hp[0] = 0.f; hp[1] = -0.f; hp[2] = 1024.5f; hp[3] = -511.25f;
    float* dp = nullptr;
    unsigned long long* db = nullptr;
    unsigned long long hb[2] = {0, 0};
    if (cudaMalloc(&dp, sizeof(hp)) || cudaMalloc(&db, 16)) return 2;
    cudaMemcpy(dp, hp, sizeof(hp), cudaMemcpyHostToDevice);
    cudaMemset(db, 0, 16);
    k_sub<<<128, 256>>>(dp, np, db);
    const int n = 1 << 22;
    k_packed<<<n / 256, 256>>>(n, db + 1);
    const cudaError_t e = cudaDeviceSynchronize();
    cudaMemcpy(hb, db, 16, cudaMemcpyDeviceToHost);
    printf("%s %llu %llu\n", cudaGetErrorString(e), hb[0], hb[1]);
    return e == cudaSuccess ? 0 : 1;
}
"""


def test_mixed_subtraction_and_packed_fp32_match_scalar(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "arith.cu"
    src.write_text(SOURCE)
    exe = tmp_path / "arith"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert out[0] == "no", out
    sub_bad, packed_bad = int(out[-2]), int(out[-1])
    print(f"mixed subtraction mismatches {sub_bad} of {65536 * 64}; packed FP32x2 mismatches {packed_bad} "
          f"of {3 << 22} triples")
    assert sub_bad == 0
    assert packed_bad == 0
