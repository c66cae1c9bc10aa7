// fp64_peak.cu -- measures the FP64 throughput of the GPU the benchmark runs
// on: DFMA (independent FMA chains per thread) and FP64 mma.sync (m8n8k4,
// m16n8k4, m16n8k8).  The benchmark's FP64 roofline uses the DFMA figure.
//
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fp64_peak fp64_peak.cu && ./fp64_peak
//
// Every kernel only touches registers and writes one double per thread into
// a buffer sized for the largest grid it launches.
#include <cstdio>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { \
  printf("CUDA error %s at line %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)

template <int CH>
__global__ void dfma_kernel(double* out, int iters, double a, double b) {
  double acc[CH];
#pragma unroll
  for (int i = 0; i < CH; i++) acc[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < CH; i++) acc[i] = fma(acc[i], a, b);
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < CH; i++) s += acc[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int CH>
__global__ void dmma884_kernel(double* out, int iters) {
  double a = 1.0 + threadIdx.x * 1e-6, b = 0.999;
  double c[CH][2];
#pragma unroll
  for (int i = 0; i < CH; i++) { c[i][0] = 0; c[i][1] = 0; }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < CH; i++)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                   : "+d"(c[i][0]), "+d"(c[i][1]) : "d"(a), "d"(b));
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < CH; i++) s += c[i][0] + c[i][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int CH>
__global__ void dmma1688_kernel(double* out, int iters) {
  double a0 = 1.0 + threadIdx.x * 1e-6, a1 = 0.5, a2 = 0.25, a3 = 0.125, b0 = 0.999, b1 = 0.5;
  double c[CH][4];
#pragma unroll
  for (int i = 0; i < CH; i++) { c[i][0] = 0; c[i][1] = 0; c[i][2] = 0; c[i][3] = 0; }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < CH; i++)
      asm volatile("mma.sync.aligned.m16n8k8.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                   : "+d"(c[i][0]), "+d"(c[i][1]), "+d"(c[i][2]), "+d"(c[i][3])
                   : "d"(a0), "d"(a1), "d"(a2), "d"(a3), "d"(b0), "d"(b1));
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < CH; i++) s += c[i][0] + c[i][1] + c[i][2] + c[i][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int main() {
  cudaDeviceProp p;
  CK(cudaGetDeviceProperties(&p, 0));
  const int sms = p.multiProcessorCount;
  printf("device %s, %d SMs, L2 %d bytes, cc %d.%d\n", p.name, sms, p.l2CacheSize, p.major, p.minor);
  const int max_threads = sms * 8 * 256;
  double* out;
  CK(cudaMalloc(&out, sizeof(double) * max_threads));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  auto timed = [&](auto launch, double flops, const char* name) {
    launch();
    cudaDeviceSynchronize();
    cudaEventRecord(e0);
    for (int r = 0; r < 5; r++) launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    printf("%-34s %9.3f ms/launch  %.4f TFLOP/s  (%s)\n", name, ms / 5, 5 * flops / (ms * 1e-3) / 1e12,
           cudaGetErrorString(cudaGetLastError()));
  };
  for (int bps : {1, 4, 8}) {
    const int grid = sms * bps, thr = 256, iters = 4096;
    char name[64];
    snprintf(name, sizeof(name), "DFMA, 8 chains, %d CTA/SM", bps);
    timed([&] { dfma_kernel<8><<<grid, thr>>>(out, iters, 0.9999, 1e-7); }, 2.0 * grid * thr * iters * 8, name);
  }
  {
    const int grid = sms * 4, thr = 256, iters = 1024;
    // m8n8k4: 2*8*8*4 = 512 flops per warp instruction
    timed([&] { dmma884_kernel<8><<<grid, thr>>>(out, iters); }, 512.0 * (grid * thr / 32) * iters * 8,
          "mma.sync f64 m8n8k4, 4 CTA/SM");
    // m16n8k8: 2*16*8*8 = 2048 flops per warp instruction
    timed([&] { dmma1688_kernel<4><<<grid, thr>>>(out, 512); }, 2048.0 * (grid * thr / 32) * 512 * 4,
          "mma.sync f64 m16n8k8, 4 CTA/SM");
  }
  CK(cudaGetLastError());
  CK(cudaFree(out));
  return 0;
}
