// Objects behind the C ABI handles and the host helpers shared by capi.cu and driver.cu.
#pragma once
#include "dp_internal.cuh"
#include "path.cuh"

struct dp_model {
  dpgb::DeviceModel m;
  char* ws = nullptr;  // cached scratch
  size_t ws_cap = 0;
  dpgb::DevStatus* status = nullptr;       // device
  dpgb::DevStatus* status_host = nullptr;  // pinned
  unsigned char* stage = nullptr;          // pinned staging for small per-call uploads
  size_t stage_cap = 0;
  dpgb::Prof prof;
  // set once a frame overflowed the density-sized candidate buffer: later builds use the
  // full DP_MAX_CANDIDATES buffer
  bool nl_full_cap = false;
};

struct dp_nlist {
  int device;
  int natoms, nc, ntypes;
  int* nl_j = nullptr;
  int* nl_code = nullptr;
  int* counts = nullptr;
};

namespace dpgb {

bool is_device_ptr(const void* p);
int ensure_ws(dp_model* md, size_t bytes);
int ensure_stage(dp_model* md, size_t bytes);
int read_status(dp_model* md, cudaStream_t st, int* n_overflow);
int type_starts(const int* type_host, const int* dtype_start, int N, int ntypes, cudaStream_t st, int* out);

}  // namespace dpgb
