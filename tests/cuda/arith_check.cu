// Unit check of the library's own arithmetic building blocks (fr_arith.cuh) against CUDA's
// correctly rounded operations, on 2^20 inputs per test drawn with splitmix64 (counter-based:
// input i is splitmix64 of the counter i).  Prints one line per check: name, worst error.
//   rcp   : rcp_t(double) (hardware approximation + two Newton steps) against 1.0 / x, in ulps
//   f32   : f32_from_double_bits(x) against __double2float_rn(x), in float ulps
//   f64   : f_to_double_bits(f) against double(f), in ulps (must be 0)
//   ffrel : |hi + lo - x| / |x| of ff_from_double(x), exponents -70..120
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <cuda_runtime.h>

#include "fr_arith.cuh"

using namespace frg;

__device__ uint64_t splitmix64(uint64_t i) {
  uint64_t z = i * 0x9E3779B97F4A7C15ull + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// positive normal double with a random significand and an exponent in [emin, emax]
__device__ double draw(uint64_t i, int emin, int emax) {
  const uint64_t r = splitmix64(i);
  const int e = emin + int((r >> 52) % uint64_t(emax - emin + 1));
  const uint64_t bits = (uint64_t(e + 1023) << 52) | (r & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double((long long)bits);
}

__global__ void k_check(int64_t n, unsigned long long* worst) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  // rcp over a wide range (exponents -60..60) and the density/pressure range [1/16, 16)
  const double x = (i & 1) ? draw(uint64_t(i), -60, 60) : draw(uint64_t(i), -4, 3);
  const double r = rcp_t(x), q = 1.0 / x;
  long long d = __double_as_longlong(r) - __double_as_longlong(q);
  atomicMax(&worst[0], (unsigned long long)(d < 0 ? -d : d));
  // double -> float rounding (within the float range, either sign)
  const double y = ((i >> 1) & 1) ? -draw(uint64_t(i) + 7, -120, 120) : draw(uint64_t(i) + 7, -120, 120);
  const float a = f32_from_double_bits(y), b = __double2float_rn(y);
  int df = __float_as_int(a) - __float_as_int(b);
  atomicMax(&worst[1], (unsigned long long)(df < 0 ? -df : df));
  // float -> double widening is exact
  const double w = f_to_double_bits(b);
  long long dw = __double_as_longlong(w) - __double_as_longlong(double(b));
  atomicMax(&worst[2], (unsigned long long)(dw < 0 ? -dw : dw));
  // double -> double-word split (exponents where the low word is a normal float)
  const double z = ((i >> 1) & 1) ? -draw(uint64_t(i) + 13, -70, 120) : draw(uint64_t(i) + 13, -70, 120);
  const ff s = ff_from_double(z);
  const double rel = fabs((double(s.h) + double(s.l)) - z) / fabs(z);
  atomicMax(&worst[3], (unsigned long long)__double_as_longlong(rel));  // rel >= 0: bits order
}

int main() {
  const int64_t n = int64_t(1) << 20;
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, 4 * sizeof(unsigned long long)) != cudaSuccess) return 2;
  cudaMemset(d, 0, 4 * sizeof(unsigned long long));
  k_check<<<unsigned((n + 255) / 256), 256>>>(n, d);
  unsigned long long h[4];
  if (cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
  cudaFree(d);
  double rel;
  memcpy(&rel, &h[3], 8);
  printf("rcp %llu\nf32 %llu\nf64 %llu\nffrel %.6e\n", h[0], h[1], h[2], rel);
  return 0;
}
