// Neighbour-list build that allocates no memory at all.
//
// Some callers cannot allocate device memory when they need a neighbour list: an MD engine
// that hands the library a pre-reserved arena and forbids any other allocation, code that
// runs while another component owns the whole device memory pool, or a driver loop that is
// being recorded into a CUDA graph (allocation calls are not allowed during capture).  This
// entry point serves them: it bins atoms into the same cell list as dp_build_nlist and forms
// the same bit-exact list, but its cell-list scratch lives in one file-scope device array of
// fixed size, and its outputs go straight into buffers the caller already owns.  The search
// itself always runs the per-atom kernel (one warp per centre atom, the full DP_MAX_CANDIDATES
// buffer): the cell-centred kernel that dp_build_nlist prefers stages a candidate stream sized
// from each frame's density and retries on the per-atom kernel when a cell overflows it, and
// this entry point has neither the room to size it nor a second pass.
//
// The array is shared by every call on a device and keeps the previous call's contents;
// everything that must start at zero (cell counters, status words) is cleared by each call.
// Calls that overlap on the GPU (different streams, or host threads without ordering) race
// on the array.
#include <mutex>

#include "dp_internal.cuh"

namespace dpgb {

namespace {

constexpr int kMaxAtoms = DP_NOALLOC_MAX_ATOMS;
constexpr int kMaxCells = DP_NOALLOC_MAX_CELLS;
constexpr long kMaxSlots = DP_NOALLOC_MAX_SLOTS;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// byte offsets of the pieces of the static scratch
// (type, cell) keys
constexpr size_t kMaxKeys = (size_t)kMaxCells * DP_MAX_TYPES;
constexpr size_t kOffCellCount = 0;
constexpr size_t kOffCellStart = kOffCellCount + align256(sizeof(int) * kMaxKeys);
constexpr size_t kOffAtomKey = kOffCellStart + align256(sizeof(int) * (kMaxKeys + 1));
constexpr size_t kOffAtomL = kOffAtomKey + align256(sizeof(int2) * kMaxAtoms);
constexpr size_t kOffAtomM = kOffAtomL + align256(sizeof(float4) * kMaxAtoms);
constexpr size_t kOffSortedL = kOffAtomM + align256(sizeof(int4) * kMaxAtoms);
constexpr size_t kOffSortedM = kOffSortedL + align256(sizeof(float4) * kMaxAtoms);
constexpr size_t kOffCode = kOffSortedM + align256(sizeof(int4) * kMaxAtoms);
constexpr size_t kOffCounts = kOffCode + align256(sizeof(int) * kMaxSlots);
constexpr size_t kOffStatus = kOffCounts + align256(sizeof(int) * DP_MAX_TYPES * kMaxAtoms);
constexpr size_t kOffBbox = kOffStatus + align256(sizeof(DevStatus));
constexpr size_t kOffGeom = kOffBbox + align256(sizeof(double) * 6);
constexpr size_t kScratchBytes = kOffGeom + align256(sizeof(NlGeom));

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_dev[kMaxDevices] = {};
void* g_scratch_ctx[kMaxDevices] = {};  // the context the cached address belongs to
std::mutex g_scratch_mu;

typedef int (*CtxGetCurrentFn)(void**);
CtxGetCurrentFn g_ctx_get = nullptr;

// The current driver context (null if it cannot be read): a device reset or a destroyed primary
// context gives a new one, in which the array has to be looked up again.
void* current_context() {
  if (!g_ctx_get) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return nullptr;
    }
    g_ctx_get = reinterpret_cast<CtxGetCurrentFn>(fn);
  }
  void* ctx = nullptr;
  return g_ctx_get(&ctx) == 0 ? ctx : nullptr;
}

// Device address of the static scratch on the current device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up once per device (again when
// the device's context has changed since, or when the context cannot be identified).
int scratch_on_current_device(char** out) {
  int dev = 0;
  DP_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device index beyond the no-allocation entry point's table");
    return DP_E_ARG;
  }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  void* ctx = current_context();  // null before the runtime has made a context current: look up
  if (!g_scratch_dev[dev] || !ctx || ctx != g_scratch_ctx[dev]) {
    void* p = nullptr;
    DP_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_dev[dev] = p;
    g_scratch_ctx[dev] = ctx;
  }
  *out = static_cast<char*>(g_scratch_dev[dev]);
  return DP_OK;
}

__global__ void k_unpack_shift(const int* __restrict__ code, long n, int* __restrict__ shift) {
  const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  int a, b, c;
  unpack_shift(code[k], a, b, c);
  shift[3 * k] = a;
  shift[3 * k + 1] = b;
  shift[3 * k + 2] = c;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace dpgb

using namespace dpgb;

extern "C" int dp_build_nlist_noalloc(const dp_model_config* cfg, int natoms, const double* coord, const int* type,
                                      const double* box, int* nl_j, int* nl_shift, int* n_overflow, void* stream) {
  if (!cfg || !coord || !type || !nl_j || !nl_shift || natoms < 1) {
    set_error("invalid argument");
    return DP_E_ARG;
  }
  if (cfg->ntypes < 1 || cfg->ntypes > DP_MAX_TYPES || !(cfg->rcut > 0)) {
    set_error("invalid model configuration");
    return DP_E_ARG;
  }
  // a hybrid descriptor's list: the larger cutoff and, per type, the larger sel of its parts
  const dp_model_config lcfg = list_config(*cfg);
  cfg = &lcfg;
  long nc = 0;
  for (int t = 0; t < cfg->ntypes; ++t) {
    if (cfg->sel[t] < 1) {
      set_error("invalid model configuration");
      return DP_E_ARG;
    }
    nc += cfg->sel[t];
  }
  if (natoms > kMaxAtoms || (long)natoms * nc > kMaxSlots) {
    set_error("frame too large for the no-allocation neighbour list: at most " + std::to_string(kMaxAtoms) +
              " atoms and " + std::to_string(kMaxSlots) + " neighbour slots (natoms x sum(sel))");
    return DP_E_ARG;
  }
  if (!on_device(coord) || !on_device(type) || !on_device(nl_j) || !on_device(nl_shift)) {
    set_error("dp_build_nlist_noalloc takes device pointers only");
    return DP_E_ARG;
  }
  char* s = nullptr;
  int rc = scratch_on_current_device(&s);
  if (rc != DP_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int* cell_count = reinterpret_cast<int*>(s + kOffCellCount);
  int* cell_start = reinterpret_cast<int*>(s + kOffCellStart);
  int2* atom_key = reinterpret_cast<int2*>(s + kOffAtomKey);
  float4* atom_l = reinterpret_cast<float4*>(s + kOffAtomL);
  int4* atom_m = reinterpret_cast<int4*>(s + kOffAtomM);
  float4* sorted_l = reinterpret_cast<float4*>(s + kOffSortedL);
  int4* sorted_m = reinterpret_cast<int4*>(s + kOffSortedM);
  int* code = reinterpret_cast<int*>(s + kOffCode);
  int* counts = reinterpret_cast<int*>(s + kOffCounts);
  DevStatus* status = reinterpret_cast<DevStatus*>(s + kOffStatus);
  double* bbox = reinterpret_cast<double*>(s + kOffBbox);
  NlGeom* geom = reinterpret_cast<NlGeom*>(s + kOffGeom);

  double lohi[6] = {0, 0, 0, 0, 0, 0};
  if (!box) {
    DP_CUDA_TRY(launch_bbox(coord, natoms, bbox, st));
    DP_CUDA_TRY(cudaMemcpyAsync(lohi, bbox, sizeof(lohi), cudaMemcpyDeviceToHost, st));
    DP_CUDA_TRY(cudaStreamSynchronize(st));
  }
  NlGeom g;
  rc = host_geometry(*cfg, natoms, box, lohi, g);
  if (rc != DP_OK) return rc;
  g.cap = DP_MAX_CANDIDATES;  // one pass, never a retry
  if ((long)g.ncell[0] * g.ncell[1] * g.ncell[2] > kMaxCells) {
    set_error("cell grid larger than the no-allocation limit of " + std::to_string(kMaxCells) + " cells");
    return DP_E_ARG;
  }
  DP_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(DevStatus), st));
  DP_CUDA_TRY(cudaMemcpyAsync(geom, &g, sizeof(NlGeom), cudaMemcpyHostToDevice, st));
  const NlLaunch L{natoms, g.ncell[0] * g.ncell[1] * g.ncell[2], g.cap, geom, nullptr, nullptr, 1,
                   (2 * g.K[0] + 1) * (2 * g.K[1] + 1) * (2 * g.K[2] + 1), 0};
  const NlScratch sc{cell_count, cell_start, atom_key, atom_l, atom_m, sorted_l, sorted_m};
  DP_CUDA_TRY(launch_nlist_build(L, cfg->ntypes, coord, type, sc, nl_j, code, counts, status, st));
  const long n = (long)natoms * nc;
  k_unpack_shift<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(code, n, nl_shift);
  DP_CUDA_TRY(cudaGetLastError());
  DevStatus hs;
  DP_CUDA_TRY(cudaMemcpyAsync(&hs, status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
  DP_CUDA_TRY(cudaStreamSynchronize(st));
  if (n_overflow) *n_overflow = hs.sel_overflow;
  if (hs.bad_coord) {
    set_error("non-finite coordinate (NaN or Inf): the list is not valid");
    return DP_E_ARG;
  }
  if (hs.bad_type) {
    set_error("atom type outside [0, ntypes)");
    return DP_E_ARG;
  }
  if (hs.capacity == 2) {
    set_error("periodic image index beyond +-511 cells: coordinates too far outside the box");
    return DP_E_ARG;
  }
  if (hs.capacity) {
    set_error("more than DP_MAX_CANDIDATES atoms within r_c of one atom");
    return DP_E_CAPACITY;
  }
  if (hs.sel_overflow) {
    set_error("neighbour count exceeded sel for " + std::to_string(hs.sel_overflow) + " (atom, type) blocks");
    return DP_E_SEL_OVERFLOW;
  }
  return DP_OK;
}
