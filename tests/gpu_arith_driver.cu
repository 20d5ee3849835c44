// Test driver: the Newton-Raphson inverse cube root of sve_device.cuh against
// CUDA's IEEE result, on inputs read from stdin.
// Usage: gpu_arith_driver < inputs (one double per line) > outputs
// Output per input: x, rcbrt64(x), 1/cbrt(x)
#include <cstdio>
#include <vector>

#include "../paper_1307_0491_gb300/csrc/sve_device.cuh"

__global__ void rcbrt_values(const double* x, double* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  out[2 * i + 0] = sve::rcbrt64(v);
  out[2 * i + 1] = 1.0 / cbrt(v);
}

int main() {
  std::vector<double> x;
  double v;
  while (std::scanf("%lf", &v) == 1) x.push_back(v);
  const int n = (int)x.size();
  if (n == 0) return 1;
  double *dx = nullptr, *dout = nullptr;
  if (cudaMalloc(&dx, sizeof(double) * n) != cudaSuccess) return 2;
  if (cudaMalloc(&dout, sizeof(double) * 2 * n) != cudaSuccess) return 2;
  cudaMemcpy(dx, x.data(), sizeof(double) * n, cudaMemcpyHostToDevice);
  rcbrt_values<<<(n + 255) / 256, 256>>>(dx, dout, n);
  std::vector<double> out(2 * (size_t)n);
  if (cudaMemcpy(out.data(), dout, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
  for (int i = 0; i < n; ++i)
    std::printf("%.17g %.17g %.17g\n", x[i], out[2 * i], out[2 * i + 1]);
  cudaFree(dx);
  cudaFree(dout);
  return 0;
}
