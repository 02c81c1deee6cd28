// Checks mpm::div64 / mpm::rcp64 against the IEEE float64 division on the GPU: seeded
// log-uniform operands over [1e-30, 1e30] with random signs, the fallback ranges of the
// divisor (subnormal-as-float32, beyond float32), and exact cases.  Prints the largest
// difference in ulps and exits non-zero when it exceeds one ulp.  Also compares the
// integer-unit conversions (fp_bits.cuh) with the hardware conversions on the same device
// over the float32 normal range: bit-identical, or the program exits non-zero.
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

// conversions: hardware and integer-unit results side by side
__global__ void k_conv(const double* x, float* hw_n, float* sw_n, const float* f, double* hw_w, double* sw_w, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    hw_n[i] = __double2float_rn(x[i]);
    sw_n[i] = mpm::f64_to_f32_rn(x[i]);
    hw_w[i] = (double)f[i];
    sw_w[i] = mpm::f32_to_f64(f[i]);
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
  // conversions over the float32 normal range (both signs, seeded exponents and mantissas)
  const int nc = 1 << 20;
  std::vector<double> cx(nc);
  std::vector<float> cf(nc);
  for (int i = 0; i < nc; ++i) {
    const double m = 1.0 + unif();
    const int e = -126 + (int)(253.999 * unif());
    cx[i] = (unif() < 0.5 ? -1 : 1) * std::ldexp(m, e);
    cf[i] = (float)((unif() < 0.5 ? -1 : 1) * std::ldexp(1.0 + unif(), -126 + (int)(253.999 * unif())));
  }
  double *dcx, *dhw_w, *dsw_w;
  float *dcf, *dhw_n, *dsw_n;
  cudaMalloc(&dcx, nc * 8);
  cudaMalloc(&dhw_w, nc * 8);
  cudaMalloc(&dsw_w, nc * 8);
  cudaMalloc(&dcf, nc * 4);
  cudaMalloc(&dhw_n, nc * 4);
  cudaMalloc(&dsw_n, nc * 4);
  cudaMemcpy(dcx, cx.data(), nc * 8, cudaMemcpyHostToDevice);
  cudaMemcpy(dcf, cf.data(), nc * 4, cudaMemcpyHostToDevice);
  k_conv<<<(nc + 255) / 256, 256>>>(dcx, dhw_n, dsw_n, dcf, dhw_w, dsw_w, nc);
  std::vector<float> hw_n(nc), sw_n(nc);
  std::vector<double> hw_w(nc), sw_w(nc);
  cudaMemcpy(hw_n.data(), dhw_n, nc * 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(sw_n.data(), dsw_n, nc * 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(hw_w.data(), dhw_w, nc * 8, cudaMemcpyDeviceToHost);
  cudaMemcpy(sw_w.data(), dsw_w, nc * 8, cudaMemcpyDeviceToHost);
  if (cudaGetLastError() != cudaSuccess) {
    std::printf("cuda error\n");
    return 2;
  }
  long long conv_bad = 0;
  for (int i = 0; i < nc; ++i) {
    const bool narrow_ok = std::memcmp(&hw_n[i], &sw_n[i], 4) == 0 || std::fabs(cx[i]) >= 0x1.fffffep127;
    conv_bad += !narrow_ok || std::memcmp(&hw_w[i], &sw_w[i], 8) != 0;
  }
  cudaFree(dcx);
  cudaFree(dhw_w);
  cudaFree(dsw_w);
  cudaFree(dcf);
  cudaFree(dhw_n);
  cudaFree(dsw_n);
  std::printf("n=%d max_ulp_div=%lld max_ulp_rcp=%lld exact_div=%lld conversions=%d conversion_mismatches=%lld\n", n,
              (long long)worst_q, (long long)worst_r, exact, nc, conv_bad);
  if (iq >= 0) std::printf("worst div: %.17g / %.17g -> %.17g\n", a[iq], b[iq], q[iq]);
  if (ir >= 0) std::printf("worst rcp: 1 / %.17g -> %.17g\n", b[ir], r[ir]);
  cudaFree(da);
  cudaFree(db);
  cudaFree(dq);
  cudaFree(dr);
  return (worst_q <= 1 && worst_r <= 1 && conv_bad == 0) ? 0 : 1;
}
