// Types shared by the per-frame path kernels and their host orchestration.
#pragma once
#include <algorithm>

#include "dp_internal.cuh"

namespace dpgb {

struct PathConst {
  int natoms, nc, M, A, ntypes, type_one_side;
  int sel[DP_MAX_TYPES];
  int sel_off[DP_MAX_TYPES + 1];
  double h[9];
  int periodic;
  double rs, rc;
  double near2;  // unused (kept for layout)
  const double* tshift;  // device [frames][27][3]: t(n) for n in {-1,0,1}^3, or null
  int nframes;
  const int* atom_frame;  // device [natoms] frame of each atom, or null (one frame)
  const double* boxes;    // device [frames][9] cell rows, or null (one frame: h)
  int Dw;                 // width of D (row stride of D and dE/dD)
  // descriptor part (Sec. II.A.1) whose slots the fields above describe: its kind, its block of
  // D, and where its slots sit in the neighbour list (slot q of type block t reads list slot
  // lsel_off[t] + q of a row of lnc entries); a listed pair with r^2 >= rc2 is padding for it
  int kind;
  int doff;
  int lnc;
  int lsel_off[DP_MAX_TYPES + 1];
  double rc2;
};

// The PathConst of one part of a model, from the model-level one (list geometry).
inline PathConst part_pc(const PathConst& pc, const PartDesc& P) {
  PathConst q = pc;
  q.kind = P.kind;
  q.nc = P.nc;
  for (int t = 0; t < pc.ntypes; ++t) q.sel[t] = P.sel[t];
  for (int t = 0; t <= pc.ntypes; ++t) q.sel_off[t] = P.sel_off[t];
  q.rc = P.rc;
  q.rs = P.rs;
  q.rc2 = P.rc * P.rc;
  q.M = P.M;
  q.A = P.A;
  q.doff = P.doff;
  return q;
}

// se_e3 parts run on the fused pair kernel (path.cu): embedding widths up to 32 and all of the
// part's nets in shared memory.
bool e3_supported(const PartDesc& P, int precision);

// Per-kernel CUDA-event timing and launch counting.  Every kernel launch of the path sits in
// a ProfScope; when timing is on, start/stop events are recorded on the launch stream around
// it and folded into per-name totals once the call has synchronised.
struct Prof {
  bool timing = false;
  long launches = 0;
  struct Rec {
    int id;
    cudaEvent_t a, b;
  };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  std::vector<std::string> names;
  std::vector<double> total_ms;
  std::vector<long> count;
  std::vector<double> work;  // tensor-core FLOPs the scope's kernels reported issuing (0: not counted)
  int id_of(const char* name) {
    for (size_t k = 0; k < names.size(); ++k)
      if (names[k] == name) return (int)k;
    names.push_back(name);
    total_ms.push_back(0.0);
    count.push_back(0);
    work.push_back(0.0);
    return (int)names.size() - 1;
  }
  cudaEvent_t ev() {
    if (pool.empty()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      return e;
    }
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  // Fold finished events into the totals (call after the stream synchronised).
  void collect() {
    for (const Rec& r : pending) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
        total_ms[r.id] += ms;
        count[r.id] += 1;
      }
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    pending.clear();
    cudaGetLastError();
  }
  // Fold the timings of events recorded inside a graph replay (the events stay with the graph).
  void collect_from(const std::vector<Rec>& recs) {
    for (const Rec& r : recs) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
        total_ms[r.id] += ms;
        count[r.id] += 1;
      }
    }
    cudaGetLastError();
  }
  void reset() {
    collect();
    for (auto& t : total_ms) t = 0.0;
    for (auto& c : count) c = 0;
    for (auto& w : work) w = 0.0;
    launches = 0;
  }
  ~Prof() {
    for (auto& r : pending) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    for (auto& e : pool) cudaEventDestroy(e);
  }
};

struct ProfScope {
  Prof* p;
  cudaStream_t st;
  int id = -1;
  cudaEvent_t a{}, b{};
  ProfScope(Prof* prof, const char* name, cudaStream_t s, int nlaunch = 1) : p(prof), st(s) {
    if (!p) return;
    p->launches += nlaunch;
    if (p->timing) {
      id = p->id_of(name);
      a = p->ev();
      b = p->ev();
      record(a);
    }
  }
  // Inside a stream capture the record must be external, so that it becomes a graph node that
  // records on every replay (a plain record would only order the capture).
  void record(cudaEvent_t e) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs == cudaStreamCaptureStatusActive)
      cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else
      cudaEventRecord(e, st);
  }
  ~ProfScope() {
    if (p && p->timing) {
      record(b);
      p->pending.push_back(Prof::Rec{id, a, b});
    }
  }
};

struct PathIO {
  Prof* prof;  // may be null
  const double* coord;  // device [N][3]
  const int* type;      // device [N]
  const int* perm;      // device [N] sorted position -> atom
  const int* nl_j;      // device [N][Nc]
  const int* nl_code;   // device [N][Nc]
  int type_start[DP_MAX_TYPES + 1];  // host copy
  double* energy;       // device [1]
  double* force;        // device [N][3], zeroed by the caller
  double* virial;       // device [9]
  double* atom_energy;  // device [N] (always written, input order)
  double* atom_virial;  // device [N][9] per-atom virial (input order)
  DevStatus* status;    // device status words
  double* epart;        // device scratch for per-block energy partials [ceil(N/256)]
  // from the list build of this call (null with an external list): per atom (input order) its
  // cell-local FP32 position and its image / packed cell coordinates, and each frame's geometry
  const float4* atom_l;
  const int4* atom_m;
  const NlGeom* geoms;
  // from the cell-centred list build of this call (else null): [N][Nc] in sorted atom order, each
  // listed pair's FP32 displacement and, in w, 1 (FP32 usable), 0 (exact FP64 needed), -1 (padding)
  const float4* disp;
};

struct __align__(32) D4 {
  double x, y, z, w;
};
struct __align__(16) F4 {
  float x, y, z, w;
};
template <class R>
struct Vec4;
template <>
struct Vec4<double> {
  typedef D4 T;
  __device__ static D4 make(double a, double b, double c, double d) { return D4{a, b, c, d}; }
};
template <>
struct Vec4<float> {
  typedef F4 T;
  __device__ static F4 make(float a, float b, float c, float d) { return F4{a, b, c, d}; }
};

__device__ __forceinline__ double tanh_r(double z) { return tanh(z); }
__device__ __forceinline__ float tanh_r(float z) { return tanhf(z); }

constexpr int kMaxNets = DP_MAX_TYPES * DP_MAX_TYPES;

template <class R>
struct NetPtrs {
  const R* w0[kMaxNets];
  const R* b0[kMaxNets];
};

// Bump allocator over one cached device buffer (256-byte aligned pieces).
struct Arena {
  char* base = nullptr;
  size_t cap = 0, used = 0;
  bool fail = false;
  bool measure = false;  // when true only counts bytes
  template <class T>
  T* get(long n) {
    size_t bytes = ((size_t)(n > 0 ? n : 1) * sizeof(T) + 255) & ~(size_t)255;
    size_t at = used;
    used += bytes;
    if (measure) return reinterpret_cast<T*>(static_cast<uintptr_t>(256));
    if (used > cap) {
      fail = true;
      return nullptr;
    }
    return reinterpret_cast<T*>(base + at);
  }
  bool ok() const { return !fail; }
};

template <class R>
int run_fitting(const DeviceModel& m, const PathConst& pc, const R* params, const R* D, const PathIO& io, Arena& ar,
                cudaStream_t st, const R** gD_out);
cudaError_t launch_sum_rows(const double* in, long n, int w, double* out, cudaStream_t st);
// Per-atom energies given as nparts FP32 partial sums [nparts][n] (sorted order), summed in a
// fixed order, to input order in FP64.
cudaError_t launch_energy_f32(const float* Eparts, int nparts, const int* perm, int n, double* atom_e,
                              cudaStream_t st);
// t(n) for n in {-1,0,1}^3 into out [27][3] (device)
cudaError_t launch_shift_table(const PathConst& pc, double* out, cudaStream_t st);

template <class R>
int run_generic(const DeviceModel& m, const PathConst& pc, const R* params, const PathIO& io, Arena& ar,
                cudaStream_t st);

// Uncompressed path with the embedding and fitting GEMMs on the tensor cores (emb_tc.cu): BF16 or
// TF32 operands by the model's precision.
bool tc_uncompressed_supported(const DeviceModel& m);
int tc_uncompressed_prepare(DeviceModel& m, const double* params_host);
int run_tc_uncompressed(const DeviceModel& m, const PathConst& pc, const PathIO& io, Arena& ar, cudaStream_t st);

}  // namespace dpgb
