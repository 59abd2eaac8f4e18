// FP64 pipe probe (standalone, not part of libttq): cycles per FP64 fused
// multiply-add for one dependent chain per warp and for eight independent
// chains, with 1..32 warps on one SM; a chain with a single active lane; a
// 64-bit shuffle chain and an FP32 FMA chain for comparison.  The kernels'
// design (instruction counts on dependency chains, work per scheduler) rests on
// these figures.  Built and run by `python -m paper_1903_11554_gb300.probe`.
#include <cstdio>
#include <cuda_runtime.h>
__global__ void dep_chain(double *out, long long *cyc, int n, double a, double b) {
  double x = threadIdx.x * 1e-3;
  long long t0 = clock64();
  for (int i = 0; i < n; ++i) x = fma(x, a, b);
  long long t1 = clock64();
  if (threadIdx.x % 32 == 0) cyc[blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32] = t1 - t0;
  out[blockIdx.x * blockDim.x + threadIdx.x] = x;
}
// 8 independent chains per thread
__global__ void ind_chain(double *out, long long *cyc, int n, double a, double b) {
  double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  long long t0 = clock64();
  for (int i = 0; i < n; ++i) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  long long t1 = clock64();
  if (threadIdx.x % 32 == 0) cyc[blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32] = t1 - t0;
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
// one active lane doing a dependent chain (rest of the warp predicated off)
__global__ void one_lane_chain(double *out, long long *cyc, int n, double a, double b) {
  double x = threadIdx.x * 1e-3;
  long long t0 = clock64();
  if (threadIdx.x == 0) for (int i = 0; i < n; ++i) x = fma(x, a, b);
  long long t1 = clock64();
  if (threadIdx.x == 0) cyc[0] = t1 - t0;
  out[threadIdx.x] = x;
}
__global__ void shfl_chain(double *out, long long *cyc, int n) {
  double x = threadIdx.x * 1e-3;
  long long t0 = clock64();
  for (int i = 0; i < n; ++i) x = __shfl_sync(0xffffffffu, x, (threadIdx.x + 1) & 31);
  long long t1 = clock64();
  if (threadIdx.x == 0) cyc[0] = t1 - t0;
  out[threadIdx.x] = x;
}
__global__ void fp32_chain(float *out, long long *cyc, int n, float a, float b) {
  float x = threadIdx.x * 1e-3f;
  long long t0 = clock64();
  for (int i = 0; i < n; ++i) x = fmaf(x, a, b);
  long long t1 = clock64();
  if (threadIdx.x == 0) cyc[0] = t1 - t0;
  out[threadIdx.x] = x;
}
int main() {
  const int n = 4096;
  double *out; long long *cyc; float *outf;
  // sizes: up to 1 block x 1024 threads (32 warps) -> out 1024 doubles, cyc 32 entries
  cudaMalloc(&out, 1024 * sizeof(double));
  cudaMalloc(&outf, 1024 * sizeof(float));
  cudaMalloc(&cyc, 64 * sizeof(long long));
  long long h[64];
  const double a = 0.999999, b = 1e-6;
  for (int warps : {1, 2, 4, 8, 16, 32}) {
    dep_chain<<<1, 32 * warps>>>(out, cyc, n, a, b);
    cudaMemcpy(h, cyc, warps * sizeof(long long), cudaMemcpyDeviceToHost);
    long long mx = 0; for (int w = 0; w < warps; ++w) mx = h[w] > mx ? h[w] : mx;
    printf("dependent DFMA chain, %2d warps/SM: %.1f cycles per DFMA per warp\n", warps, (double)mx / n);
  }
  for (int warps : {1, 2, 4, 8, 16, 32}) {
    ind_chain<<<1, 32 * warps>>>(out, cyc, n, a, b);
    cudaMemcpy(h, cyc, warps * sizeof(long long), cudaMemcpyDeviceToHost);
    long long mx = 0; for (int w = 0; w < warps; ++w) mx = h[w] > mx ? h[w] : mx;
    printf("8 independent chains, %2d warps/SM: %.2f cycles per warp-DFMA (SM: %.2f lane-DFMA/clk)\n", warps,
           (double)mx / (8.0 * n), 8.0 * n * 32 * warps / (double)mx);
  }
  one_lane_chain<<<1, 32>>>(out, cyc, n, a, b);
  cudaMemcpy(h, cyc, sizeof(long long), cudaMemcpyDeviceToHost);
  printf("one active lane, dependent chain: %.1f cycles per DFMA\n", (double)h[0] / n);
  shfl_chain<<<1, 32>>>(out, cyc, n);
  cudaMemcpy(h, cyc, sizeof(long long), cudaMemcpyDeviceToHost);
  printf("dependent 64-bit shuffle chain: %.1f cycles per shuffle\n", (double)h[0] / n);
  fp32_chain<<<1, 32>>>(outf, cyc, n, 0.999f, 1e-3f);
  cudaMemcpy(h, cyc, sizeof(long long), cudaMemcpyDeviceToHost);
  printf("dependent FFMA chain: %.1f cycles per FFMA\n", (double)h[0] / n);
  cudaError_t e = cudaDeviceSynchronize();
  printf("status %s\n", cudaGetErrorString(e));
  return e == cudaSuccess ? 0 : 1;
}
