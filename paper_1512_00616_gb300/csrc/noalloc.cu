// pp_qoi_rate_noalloc: the instantaneous-QoI reduction of pp_qoi_rate without any device
// allocation.  Its scratch (per-element partial sums, per-block partials and the
// finishing counter) lives in one file-scope static device array, so callers that may
// not call cudaMalloc can use it.  Example callers: code running under a memory pool or
// allocator that forbids outside allocations, or code that must not allocate after
// start-up.
#include <mutex>

#include "context.h"
#include "../../include/pp.h"

namespace pp {
namespace {

constexpr int kNoAllocMaxElems = 1 << 16;                 // element capacity of the scratch
constexpr int kNoAllocPartials = 4096;                     // per-block partial sums
constexpr size_t kNoAllocWords = (size_t)kNoAllocMaxElems * 2 + kNoAllocPartials + 32;

// 1 MiB + 33 KiB of scratch per device that loads the library, kept until process exit.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocWords];

constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;  // first lookups from several host threads do not race

// Device address of the scratch array on `device` (which must be current); looked up once
// per device.  A cudaDeviceReset of that device makes the cached address stale.
int scratch_address(pp_ctx* ctx, int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return set_error(ctx, PP_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[device]) {
    double* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return set_error(ctx, PP_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_ptr[device] = p;
  }
  *out = g_scratch_ptr[device];
  return PP_OK;
}

}  // namespace
}  // namespace pp

using namespace pp;

extern "C" int pp_qoi_rate_noalloc(pp_ctx* ctx, const pp_mesh* mesh, const double* mu, int n_mu, double t,
                                   const double* u, double* out) {
  if (!ctx || !mesh || !mu || !u || !out) return set_error(ctx, PP_EINVAL, "pp_qoi_rate_noalloc: null argument");
  PP_TRY(check_mu(ctx, n_mu));
  if (mesh->ne > kNoAllocMaxElems)
    return set_error(ctx, PP_EINVAL, "pp_qoi_rate_noalloc: mesh has more than 65536 elements (scratch capacity)");
  PP_CK(cudaSetDevice(ctx->device));
  double* scratch = nullptr;
  PP_TRY(scratch_address(ctx, ctx->device, &scratch));
  double* per_elem = scratch;                                   // [ne][2]
  double* partial = scratch + (size_t)kNoAllocMaxElems * 2;     // [blocks][2]
  double* result = partial + kNoAllocPartials;                  // [2]
  unsigned* counter = reinterpret_cast<unsigned*>(result + 8);  // finishing counter, must start at zero
  PP_CK(cudaMemsetAsync(counter, 0, sizeof(unsigned), ctx->stream));
  FrameT<double> fr = frame_of(motion(ctx, mu, n_mu, t));
  PP_CK(launch_qoi(mesh->dev, ctx->tb, ctx->ph, fr, u, per_elem, ctx->stream));
  PP_CK(launch_colsum(mesh->ne, 2, per_elem, result, partial, counter, ctx->stream));
  PP_CK(cudaMemcpyAsync(out, result, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  PP_CK(cudaStreamSynchronize(ctx->stream));
  return PP_OK;
}
