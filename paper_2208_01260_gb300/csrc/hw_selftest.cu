// Device self-check of the integer-pipe binary64 multiply and reciprocal (hw_fp64_int.h) against the
// FP64 pipe on the device itself (hwswe.h: hw_selftest_fp64_int).
#include <cuda_runtime.h>

#include "hw_fp64_int.h"
#include "hw_internal.h"

namespace hw {
namespace {

// splitmix64 finaliser: a counter-based generator of operand bits
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__global__ void k_selftest_mul(long long n, unsigned long long seed, unsigned long long* cnt) {
  const unsigned long long SGN_FRAC = 0x800fffffffffffffull;
  unsigned long long acc = 0, bad = 0, missed = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long c = mix64(seed ^ (3ull * i));
    unsigned long long a = mix64(c + 1), b = mix64(c + 2);
    switch ((int)(c % 7)) {
      case 1:
        a = (a & SGN_FRAC) | (unsigned long long)(1000 + (c >> 8) % 48) << 52;
        b = (b & SGN_FRAC) | (unsigned long long)(1000 + (c >> 16) % 48) << 52;
        break;
      case 2:
        a = (a & 0x800fff0000000000ull) | 1023ull << 52;
        b = (b & 0x800ffffff0000000ull) | 1023ull << 52;
        break;
      case 3:
        b = a ^ ((c >> 8) & 0xfff);
        break;
      case 4:
        if ((c >> 8) & 1) a &= 0x8000000000000000ull;
        else b &= 0x8000000000000000ull;
        break;
      case 5:
        a = (a & SGN_FRAC) | (unsigned long long)(1 + (c >> 8) % 40) << 52;
        b = (b & SGN_FRAC) | (unsigned long long)(1000 + (c >> 16) % 40) << 52;
        if ((c >> 24) & 1) a = (a & SGN_FRAC) | (unsigned long long)(2000 + (c >> 32) % 46) << 52;
        break;
      case 6:
        a = (a & SGN_FRAC) | (unsigned long long)(((c >> 8) % 3 == 0) ? 2047 : 0) << 52;
        break;
      default:
        break;
    }
    const double x = __longlong_as_double((long long)a), y = __longlong_as_double((long long)b);
    const double t = __dmul_rn(x, y);
    double r;
    if (f64_mul_int(x, y, r)) {
      ++acc;
      bad += __double_as_longlong(r) != __double_as_longlong(t);
    } else {
      const unsigned ex = (unsigned)(a >> 52) & 0x7ffu, ey = (unsigned)(b >> 52) & 0x7ffu;
      const double at = fabs(t);
      missed += (ex != 0 && ex != 0x7ff && ey != 0 && ey != 0x7ff && at >= 0x1p-1021 && at < 0x1p1022);
    }
  }
  atomicAdd(cnt, acc);
  atomicAdd(cnt + 1, bad);
  atomicAdd(cnt + 2, missed);
}

// Products by the literal constants the kernels multiply by (the folded-constant form of the integer
// multiply), bit for bit against DMUL.
__device__ __forceinline__ void const_check(double x, double c, unsigned long long& acc, unsigned long long& bad) {
  double r;
  if (f64_mul_int<true>(x, c, r)) {
    ++acc;
    bad += __double_as_longlong(r) != __double_as_longlong(__dmul_rn(x, c));
  }
}

__global__ void k_selftest_const(long long n, unsigned long long seed, unsigned long long* cnt) {
  unsigned long long acc = 0, bad = 0, missed = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long c = mix64(seed ^ (7ull * i));
    unsigned long long a = mix64(c + 1);
    if (c % 2) a = (a & 0x800fffffffffffffull) | (unsigned long long)(990 + (c >> 8) % 60) << 52;
    const double x = __longlong_as_double((long long)a);
    const_check(x, 781.0 / 20.0, acc, bad);
    const_check(x, 13.0 / 3.0, acc, bad);
    const_check(x, 781.0 / 80.0, acc, bad);
    const_check(x, 13.0 / 12.0, acc, bad);
    const_check(x, 4.0 / 3.0, acc, bad);
    const_check(x, 0.5, acc, bad);
    const_check(x, 1.0 / 6.0, acc, bad);
    const_check(x, 0.25, acc, bad);
    const_check(x, 4.0, acc, bad);
    const_check(x, 8.0, acc, bad);
  }
  atomicAdd(cnt, acc);
  atomicAdd(cnt + 1, bad);
  atomicAdd(cnt + 2, missed);
}

// Reciprocals against the correctly rounded __drcp_rn: accepted results more than one ulp away count as
// mismatches; operands with a normal reciprocal (biased exponent 1..2044) must be accepted.
__global__ void k_selftest_rcp(long long n, unsigned long long seed, unsigned long long* cnt) {
  unsigned long long acc = 0, bad = 0, missed = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long c = mix64(seed ^ (5ull * i));
    unsigned long long a = mix64(c + 1);
    if (c % 3 == 1) a = (a & 0x800fffffffffffffull) | (unsigned long long)(1000 + (c >> 8) % 48) << 52;
    if (c % 3 == 2)  // significands near 1 and near 2, all exponents of the fast path
      a = (a & 0x80000000000fffffull) | (unsigned long long)(1 + (c >> 8) % 2044) << 52 |
          (((c >> 20) & 1) ? 0ull : 0x000ffffffff00000ull);
    const double x = __longlong_as_double((long long)a);
    const unsigned ex = (unsigned)(a >> 52) & 0x7ffu;
    double r;
    if (f64_rcp_int(x, r)) {
      ++acc;
      const long long d = __double_as_longlong(r) - __double_as_longlong(__drcp_rn(x));
      bad += (d > 1 || d < -1);
    } else {
      missed += (ex >= 1 && ex <= 2044);
    }
  }
  atomicAdd(cnt, acc);
  atomicAdd(cnt + 1, bad);
  atomicAdd(cnt + 2, missed);
}

}  // namespace
}  // namespace hw

extern "C" int hw_selftest_fp64_int(int op, long long n, unsigned long long seed, long long* counts) {
  if (op < 0 || op > 2 || n < 1 || counts == nullptr) return HW_ERR_ARG;
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, 3 * sizeof(unsigned long long)) != cudaSuccess) return HW_ERR_CUDA;
  unsigned long long h[3] = {0, 0, 0};
  cudaError_t e = cudaMemset(d, 0, sizeof(h));
  if (e == cudaSuccess) {
    if (op == 0) hw::k_selftest_mul<<<1216, 256>>>(n, seed, d);
    else if (op == 1) hw::k_selftest_rcp<<<1216, 256>>>(n, seed, d);
    else hw::k_selftest_const<<<1216, 256>>>(n, seed, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return HW_ERR_CUDA;
  for (int k = 0; k < 3; ++k) counts[k] = (long long)h[k];
  return HW_OK;
}
