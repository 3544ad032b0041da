// Scalar (non-tensor) floating-point issue-rate microbenchmark.
//
// The source-term update is bound by scalar FP64/FP32 arithmetic, not by a
// dense contraction, so its roofline denominator is the FMA issue rate of the
// SM pipes. This program measures it: every thread runs independent FMA
// chains (enough of them to hide pipe latency) for a fixed number of steps,
// the grid fills every SM several times over, and CUDA events time it.
// One FMA counts as 2 flops. The result of each thread is written out so the
// compiler cannot drop the chains.
//
// Usage: fp_peak [reps]   -> prints one JSON line with fp64/fp32 TFLOP/s.
#include <cstdio>
#include <cstdlib>
#include <cuda_runtime.h>

#define CK(x)                                                                  \
  do {                                                                         \
    cudaError_t e_ = (x);                                                      \
    if (e_ != cudaSuccess) {                                                   \
      std::fprintf(stderr, "CUDA error %s at %s:%d\n", cudaGetErrorString(e_), \
                   __FILE__, __LINE__);                                        \
      std::exit(1);                                                            \
    }                                                                          \
  } while (0)

template <typename T, int CHAINS>
__global__ void fma_loop(T *out, int steps, T a, T b) {
  T acc[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) acc[k] = T(threadIdx.x + k);
  for (int s = 0; s < steps; ++s) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) acc[k] = fma(acc[k], a, b);
  }
  T r = 0;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) r += acc[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// The cost of one division, square root or expm1, in FMA issue slots of the
// same precision: the same independent chains, each step one such operation
// (kept bounded and normal: x -> a / x + b alternates between x and a / x;
// x -> sqrt(x) a + b tends to 1; x -> expm1(x) a + b with a = b = 1/4 to
// 0.36), timed against the FMA chains.  The counting model of the update tallies these operations by kind;
// these weights turn its tallies into issue slots.
enum Op { kDiv, kSqrt, kExpm1 };

template <typename T, int CHAINS, int OP>
__global__ void op_loop(T *out, int steps, T a, T b) {
  T acc[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) acc[k] = T(0.5) + T(0.01) * T(k) + T(1e-6) * T(threadIdx.x);
  for (int s = 0; s < steps; ++s) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) {
      if (OP == kDiv) acc[k] = a / acc[k] + b;
      else if (OP == kSqrt) acc[k] = sqrt(acc[k]) * a + b;
      else acc[k] = expm1(acc[k]) * a + b;
    }
  }
  T r = 0;
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) r += acc[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// Milliseconds of the best of reps launches of kernel(out, steps, a, b).
template <typename T, typename K>
static float best_ms(K kernel, int blocks, int threads, int steps, int reps, T a, T b) {
  T *out = nullptr;
  CK(cudaMalloc(&out, sizeof(T) * (size_t)blocks * threads));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  kernel<<<blocks, threads>>>(out, steps, a, b);  // warm-up
  CK(cudaGetLastError());
  CK(cudaDeviceSynchronize());
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    CK(cudaEventRecord(e0));
    kernel<<<blocks, threads>>>(out, steps, a, b);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) best = ms;
  }
  CK(cudaFree(out));
  CK(cudaEventDestroy(e0));
  CK(cudaEventDestroy(e1));
  return best;
}

// Issue slots of one op of each kind, relative to one FMA (the extra FMA or
// add of the sqrt and div chains taken off).
template <typename T>
static void op_costs(int blocks, int threads, int steps, int reps, double out[3]) {
  const float f = best_ms<T>(fma_loop<T, 8>, blocks, threads, steps, reps, T(0.9999999), T(1e-7));
  const float d = best_ms<T>(op_loop<T, 8, kDiv>, blocks, threads, steps, reps, T(0.25), T(0));
  const float q = best_ms<T>(op_loop<T, 8, kSqrt>, blocks, threads, steps, reps, T(1), T(0));
  const float x = best_ms<T>(op_loop<T, 8, kExpm1>, blocks, threads, steps, reps, T(0.25), T(0.25));
  out[0] = d / f - 1.0;  // a / x + b: the division and one add
  out[1] = q / f - 1.0;  // sqrt(x) a + b: the root and one FMA
  out[2] = x / f - 1.0;  // expm1(x) a + b: the function and one FMA
}

template <typename T, int CHAINS>
static double run(int blocks, int threads, int steps, int reps) {
  T *out = nullptr;
  CK(cudaMalloc(&out, sizeof(T) * (size_t)blocks * threads));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // a slightly below 1 keeps the chains finite for any step count
  const T a = T(0.9999999), b = T(1e-7);
  fma_loop<T, CHAINS><<<blocks, threads>>>(out, steps, a, b);  // warm-up
  CK(cudaGetLastError());
  CK(cudaDeviceSynchronize());
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    CK(cudaEventRecord(e0));
    fma_loop<T, CHAINS><<<blocks, threads>>>(out, steps, a, b);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) best = ms;
  }
  CK(cudaFree(out));
  CK(cudaEventDestroy(e0));
  CK(cudaEventDestroy(e1));
  const double flops = 2.0 * CHAINS * (double)steps * blocks * threads;
  return flops / (best * 1e-3) / 1e12;
}

int main(int argc, char **argv) {
  int reps = argc > 1 ? std::atoi(argv[1]) : 5;
  int dev = 0, sms = 0, clk = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev));
  const int threads = 256, blocks = sms * 8;
  double t64 = run<double, 8>(blocks, threads, 1 << 12, reps);
  double t32 = run<float, 8>(blocks, threads, 1 << 16, reps);
  double c64[3], c32[3];
  op_costs<double>(blocks, threads, 1 << 10, reps, c64);
  op_costs<float>(blocks, threads, 1 << 14, reps, c32);
  std::printf("{\"sms\": %d, \"sm_clock_khz_attr\": %d, \"fp64_fma_tflops\": %.4f, "
              "\"fp32_fma_tflops\": %.3f, \"fp64_op_slots\": {\"div\": %.2f, \"sqrt\": %.2f, "
              "\"exp\": %.2f}, \"fp32_op_slots\": {\"div\": %.2f, \"sqrt\": %.2f, \"exp\": %.2f}}\n",
              sms, clk, t64, t32, c64[0], c64[1], c64[2], c32[0], c32[1], c32[2]);
  return 0;
}
