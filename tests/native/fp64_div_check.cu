// Checks mpm::div64 / mpm::rcp64 against the IEEE float64 division on the GPU: seeded
// log-uniform operands over [1e-30, 1e30] with random signs, the fallback ranges of the
// divisor (subnormal-as-float32, beyond float32), and exact cases.  Prints the largest
// difference in ulps and exits non-zero when it exceeds one ulp.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "fp64_div.cuh"

__global__ void k_check(const double* a, const double* b, double* q, double* r, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    q[i] = mpm::div64(a[i], b[i]);
    r[i] = mpm::rcp64(b[i]);
  }
}

static uint64_t state = 0x9e3779b97f4a7c15ull;
static double unif() {  // splitmix64 -> [0, 1)
  uint64_t z = (state += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

static int64_t ulps(double x, double y) {
  int64_t ix, iy;
  std::memcpy(&ix, &x, 8);
  std::memcpy(&iy, &y, 8);
  if ((ix < 0) != (iy < 0)) return x == y ? 0 : INT64_MAX;
  return ix > iy ? ix - iy : iy - ix;
}

int main() {
  std::vector<double> a, b;
  const int nrand = 1 << 20;
  for (int i = 0; i < nrand; ++i) {
    a.push_back((unif() < 0.5 ? -1 : 1) * std::pow(10.0, -30.0 + 60.0 * unif()));
    b.push_back((unif() < 0.5 ? -1 : 1) * std::pow(10.0, -30.0 + 60.0 * unif()));
  }
  const double special_b[] = {1e-40, 5e-39, 1.17e-38, 1.2e-38, 2.35e-38, 2.36e-38, 4.2e37, 4.3e37, 8.5e37, 3.4e38,
                              3.5e38, 1e40, 1e-300, 1e300, 1.0, 2.0, 3.0, 4.0, 0.5, 7.0, 1.0 + 1e-15};
  for (double sb : special_b)
    for (double sa : {1.0, 3.0, -2.5, 1e-10, 1e10, 0.0}) {
      a.push_back(sa);
      b.push_back(sb);
    }
  const int n = (int)a.size();
  double *da, *db, *dq, *dr;
  cudaMalloc(&da, n * 8);
  cudaMalloc(&db, n * 8);
  cudaMalloc(&dq, n * 8);
  cudaMalloc(&dr, n * 8);
  cudaMemcpy(da, a.data(), n * 8, cudaMemcpyHostToDevice);
  cudaMemcpy(db, b.data(), n * 8, cudaMemcpyHostToDevice);
  k_check<<<(n + 255) / 256, 256>>>(da, db, dq, dr, n);
  std::vector<double> q(n), r(n);
  cudaMemcpy(q.data(), dq, n * 8, cudaMemcpyDeviceToHost);
  cudaMemcpy(r.data(), dr, n * 8, cudaMemcpyDeviceToHost);
  if (cudaGetLastError() != cudaSuccess) {
    std::printf("cuda error\n");
    return 2;
  }
  int64_t worst_q = 0, worst_r = 0;
  long long exact = 0;
  int iq = -1, ir = -1;
  for (int i = 0; i < n; ++i) {
    const double wq = a[i] / b[i], wr = 1.0 / b[i];
    if (std::isfinite(wq) && std::fpclassify(wq) != FP_SUBNORMAL) {
      const int64_t u = ulps(q[i], wq);
      if (u > worst_q) {
        worst_q = u;
        iq = i;
      }
      exact += u == 0;
    }
    if (std::isfinite(wr) && std::fpclassify(wr) != FP_SUBNORMAL) {
      const int64_t u = ulps(r[i], wr);
      if (u > worst_r) {
        worst_r = u;
        ir = i;
      }
    }
  }
  std::printf("n=%d max_ulp_div=%lld max_ulp_rcp=%lld exact_div=%lld\n", n, (long long)worst_q, (long long)worst_r,
              exact);
  if (iq >= 0) std::printf("worst div: %.17g / %.17g -> %.17g\n", a[iq], b[iq], q[iq]);
  if (ir >= 0) std::printf("worst rcp: 1 / %.17g -> %.17g\n", b[ir], r[ir]);
  cudaFree(da);
  cudaFree(db);
  cudaFree(dq);
  cudaFree(dr);
  return (worst_q <= 1 && worst_r <= 1) ? 0 : 1;
}
