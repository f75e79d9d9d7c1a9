// Objects behind the C ABI handles and the host helpers shared by capi.cu and driver.cu.
#pragma once
#include "dp_internal.cuh"
#include "path.cuh"

// A call sequence recorded as a CUDA graph, replayed while the calls keep the same shape.
struct DpGraph {
  std::vector<unsigned long long> sig;  // what the recorded call depended on (sizes, pointers, box)
  cudaGraphExec_t exec = nullptr;
  unsigned char* stage = nullptr;  // pinned per-call tables the graph uploads (private copy)
  size_t stage_cap = 0;
  std::vector<dpgb::Prof::Rec> prof;  // timing events recorded inside the graph
  long launches = 0;                  // kernel launches of one replay
};

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
  // per-type atom counts of the last device type array seen (checked on the device when reused)
  const int* ts_ptr = nullptr;
  int ts_n = -1;
  int ts_v[DP_MAX_TYPES + 1] = {};
  // graph of the last repeated call shape; the shape of the previous call
  DpGraph graph;
  std::vector<unsigned long long> last_sig;
  cudaStream_t cap_st = nullptr;  // capture stream (the caller's may be the legacy default stream)
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
// DP_E_ARG (with a message) when one of the n host values is NaN or infinite.
int check_finite_host(const double* x, long n);
int ensure_ws(dp_model* md, size_t bytes);
int ensure_stage(dp_model* md, size_t bytes);
int read_status(dp_model* md, cudaStream_t st, int* n_overflow);
void drop_graph(dp_model* md);
// read_status result: the per-type atom counts differ from the ones the call was set up with
constexpr int kStatusTypeChange = -1000;
int type_starts(const int* type_host, const int* dtype_start, int N, int ntypes, cudaStream_t st, int* out);

}  // namespace dpgb
