// Kernel-class timing with CUDA events on the launching stream, launch counting,
// and an FP64 FMA throughput probe (diagnostics declared in include/pp_prof.h).
#include <vector>

#include "../../include/pp_prof.h"
#include "prof.h"

namespace pp {

namespace {
int g_kind = PP_K_NONE;
std::vector<cudaEvent_t> g_ev;   // pairs (start, stop)
size_t g_used = 0;               // events used
int64_t g_launch[PP_K_COUNT] = {0};
int64_t g_timed = 0;
constexpr size_t kMaxPairs = 1 << 16;
}  // namespace

void prof_begin(int kind, cudaStream_t st, cudaEvent_t* stop_out) {
  g_launch[kind]++;
  *stop_out = nullptr;
  if (kind != g_kind || g_used + 2 > 2 * kMaxPairs) return;
  if (g_used + 2 > g_ev.size()) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return;
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return;
    }
    g_ev.push_back(a);
    g_ev.push_back(b);
  }
  cudaEventRecord(g_ev[g_used], st);
  *stop_out = g_ev[g_used + 1];
  g_used += 2;
  g_timed++;
}

void prof_end(cudaEvent_t stop, cudaStream_t st) {
  if (stop) cudaEventRecord(stop, st);
}

__global__ void k_fma_probe(double* out, int iters) {
  double a0 = threadIdx.x * 1e-9, a1 = a0 + 1e-9, a2 = a0 + 2e-9, a3 = a0 + 3e-9;
  double a4 = a0 + 4e-9, a5 = a0 + 5e-9, a6 = a0 + 6e-9, a7 = a0 + 7e-9;
  const double b = 0.999999999, c = 1e-12;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      a0 = fma(a0, b, c);
      a1 = fma(a1, b, c);
      a2 = fma(a2, b, c);
      a3 = fma(a3, b, c);
      a4 = fma(a4, b, c);
      a5 = fma(a5, b, c);
      a6 = fma(a6, b, c);
      a7 = fma(a7, b, c);
    }
  }
  double s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (s == 12345.678) out[0] = s;  // keeps the chains alive
}

}  // namespace pp

extern "C" {

int pp_prof_select(int kind) {
  using namespace pp;
  if (kind < 0 || kind >= PP_K_COUNT) return -1;
  cudaDeviceSynchronize();
  g_kind = kind;
  g_used = 0;
  g_timed = 0;
  for (int k = 0; k < PP_K_COUNT; ++k) g_launch[k] = 0;
  return 0;
}

int pp_prof_read(int64_t* launches, double* total_ms) {
  using namespace pp;
  if (cudaDeviceSynchronize() != cudaSuccess) return -6;
  double tot = 0.0;
  for (size_t i = 0; i + 1 < g_used; i += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, g_ev[i], g_ev[i + 1]) == cudaSuccess) tot += ms;
  }
  if (launches) *launches = g_timed;
  if (total_ms) *total_ms = tot;
  return 0;
}

int pp_prof_counts(int64_t* counts) {
  using namespace pp;
  if (!counts) return -1;
  for (int k = 0; k < PP_K_COUNT; ++k) counts[k] = g_launch[k];
  return 0;
}

int pp_measure_fp64_peak(int device, double* tflops) {
  using namespace pp;
  if (!tflops) return -1;
  if (cudaSetDevice(device) != cudaSuccess) return -6;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double)) != cudaSuccess) return -6;
  const int threads = 256, blocks = sms * 8, iters = 2048;
  k_fma_probe<<<blocks, threads>>>(out, 16);  // warm-up
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a);
  k_fma_probe<<<blocks, threads>>>(out, iters);
  cudaEventRecord(b);
  cudaError_t e = cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  if (e != cudaSuccess || ms <= 0.f) return -6;
  double flops = 2.0 * 8.0 * 16.0 * iters * (double)threads * blocks;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return 0;
}

}  // extern "C"
