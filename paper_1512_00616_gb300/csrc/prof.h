// Hooks used by the launch wrappers to time one kernel class (include/pp_prof.h).
#pragma once
#include <cuda_runtime.h>

namespace pp {
void prof_begin(int kind, cudaStream_t st, cudaEvent_t* stop_out);
void prof_end(cudaEvent_t stop, cudaStream_t st);
// algorithmic bytes of the next `launches` launches of class `kind` (counted only when
// those launches will be timed)
void prof_add_bytes(int kind, double bytes, int launches);

struct ProfScope {
  cudaEvent_t stop;
  cudaStream_t st;
  ProfScope(int kind, cudaStream_t s) : st(s) { prof_begin(kind, s, &stop); }
  ~ProfScope() { prof_end(stop, st); }
};
}  // namespace pp
