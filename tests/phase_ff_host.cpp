// Host build of the complex64 tables' phase factor (wp_phase_ff.cuh: FP64 reduction of the
// argument modulo pi/2, float-float Taylor series of cosine and sine), for the CPU tests.
// The float-float arithmetic's rounded intrinsics are the IEEE single-precision operations
// (built with -ffp-contract=off, so that no product and sum fuse on the host either).
// Reads a count n and n doubles from stdin (binary); writes for each argument the float
// parts cos.hi, cos.lo, sin.hi, sin.lo.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <vector>

#include <cuda_runtime.h>  // __host__ / __device__ / __forceinline__ for a host compiler

static inline float __fadd_rn(float a, float b) { return a + b; }
static inline float __fsub_rn(float a, float b) { return a - b; }
static inline float __fmul_rn(float a, float b) { return a * b; }

#include "wp_phase_ff.cuh"

int main() {
  int64_t n = 0;
  if (fread(&n, sizeof(n), 1, stdin) != 1 || n < 0 || n > (int64_t(1) << 26)) return 2;
  std::vector<double> th((size_t)n);
  if (n && fread(th.data(), sizeof(double), (size_t)n, stdin) != (size_t)n) return 2;
  std::vector<float> out(4 * (size_t)n);
  for (int64_t i = 0; i < n; i++) {
    wp::ff c, s;
    wp::cis_ff(th[i], c, s);
    out[4 * i + 0] = c.hi;
    out[4 * i + 1] = c.lo;
    out[4 * i + 2] = s.hi;
    out[4 * i + 3] = s.lo;
  }
  if (n && fwrite(out.data(), sizeof(float), out.size(), stdout) != out.size()) return 3;
  return 0;
}
