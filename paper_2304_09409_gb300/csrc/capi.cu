// C ABI of libdpgb: model and neighbour-list objects, scratch management, and the
// per-frame driver that chains the kernels of the se_e2_a path.
#include <algorithm>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "capi_internal.cuh"
#include "dp_internal.cuh"
#include "fit_tc.cuh"
#include "path.cuh"
#include "table.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace dpgb {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }

// error word of the stand-alone tensor-core GEMM entry point
__device__ int g_gemm_err;

namespace {

// One mbarrier that expects one arrival nobody makes; thread 0 waits on it through the bounded
// wait of the tensor-core kernels, which gives up after `limit` polls and raises *err.
__global__ void k_wait_selftest(long limit, int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    ptx::mbar_init(&bar, 1);
    ptx::mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) ptx::mbar_wait_limit(&bar, 0, err, limit);
  __syncthreads();
}

__global__ void k_narrow(const double* __restrict__ x, long n, float* __restrict__ y) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) y[e] = (float)x[e];
}

int skip_kind(int n_in, int n_out) { return n_out == n_in ? 1 : (n_out == 2 * n_in ? 2 : 0); }

bool is_hybrid(const dp_model_config& c) {
  return c.descriptor == DP_DESC_HYBRID_R || c.descriptor == DP_DESC_HYBRID_E3;
}

int check_config(const dp_model_config* c) {
  if (!c) return DP_E_ARG;
  if (c->ntypes < 1 || c->ntypes > DP_MAX_TYPES) return DP_E_ARG;
  if (c->n_embed < 1 || c->n_embed > DP_MAX_LAYERS || c->n_fit < 0 || c->n_fit > DP_MAX_LAYERS) return DP_E_ARG;
  for (int t = 0; t < c->ntypes; ++t)
    if (c->sel[t] < 1) return DP_E_ARG;
  for (int l = 0; l < c->n_embed; ++l)
    if (c->embed[l] < 1) return DP_E_ARG;
  for (int l = 0; l < c->n_fit; ++l)
    if (c->fit[l] < 1) return DP_E_ARG;
  if (c->descriptor < DP_DESC_SE_E2_A || c->descriptor > DP_DESC_HYBRID_E3) return DP_E_ARG;
  const bool first_a = c->descriptor != DP_DESC_SE_E2_R && c->descriptor != DP_DESC_SE_E3;
  if (first_a && (c->axis < 1 || c->axis > c->embed[c->n_embed - 1])) return DP_E_ARG;
  if (!(c->rcut > 0) || !(c->rcut_smth >= 0) || !(c->rcut_smth < c->rcut)) return DP_E_ARG;
  if (is_hybrid(*c)) {
    if (c->n_embed_2 < 1 || c->n_embed_2 > DP_MAX_LAYERS) return DP_E_ARG;
    for (int l = 0; l < c->n_embed_2; ++l)
      if (c->embed_2[l] < 1) return DP_E_ARG;
    for (int t = 0; t < c->ntypes; ++t)
      if (c->sel_2[t] < 1) return DP_E_ARG;
    if (!(c->rcut_2 > 0) || !(c->rcut_smth_2 >= 0) || !(c->rcut_smth_2 < c->rcut_2)) return DP_E_ARG;
  }
  return DP_OK;
}

// The parts of a descriptor (Sec. II.A.1), their nets' parameter layout from `off` on, and
// their blocks of D (Dw receives the width of D).
std::vector<PartDesc> make_parts(const dp_model_config& c, long& off, int& Dw) {
  std::vector<PartDesc> parts;
  auto add = [&](int kind, double rc, double rs, const int* sel, int nl, const int* widths) {
    PartDesc P;
    P.kind = kind;
    P.rc = rc;
    P.rs = rs;
    P.nc = 0;
    for (int t = 0; t < c.ntypes; ++t) {
      P.sel[t] = sel[t];
      P.sel_off[t] = P.nc;
      P.nc += sel[t];
    }
    P.sel_off[c.ntypes] = P.nc;
    P.M = widths[nl - 1];
    P.A = kind == PART_A ? c.axis : 0;
    P.nl = nl;
    // se_e3 nets are indexed by the two neighbours' types; two-body nets by (a_i, a_j) or a_j
    P.n_nets = (kind == PART_E3 || !c.type_one_side) ? c.ntypes * c.ntypes : c.ntypes;
    P.w_off = off;
    for (int n = 0; n < P.n_nets; ++n) {
      int prev = 1;
      for (int l = 0; l < nl; ++l) {
        P.emb.push_back(LayerDesc{prev, widths[l], off, skip_kind(prev, widths[l]), 1});
        off += (long)prev * widths[l] + widths[l];
        prev = widths[l];
      }
    }
    P.per_net = (off - P.w_off) / P.n_nets;
    P.doff = Dw;
    Dw += kind == PART_A ? P.M * P.A : P.M;
    parts.push_back(P);
  };
  Dw = 0;
  const int d = c.descriptor;
  const int k1 = d == DP_DESC_SE_E2_R ? PART_R : (d == DP_DESC_SE_E3 ? PART_E3 : PART_A);
  add(k1, c.rcut, c.rcut_smth, c.sel, c.n_embed, c.embed);
  if (is_hybrid(c))
    add(d == DP_DESC_HYBRID_R ? PART_R : PART_E3, c.rcut_2, c.rcut_smth_2, c.sel_2, c.n_embed_2, c.embed_2);
  return parts;
}

// Parameter layout: the parts' embedding nets, then the fitting nets by type.
long layout(const dp_model_config& c, std::vector<PartDesc>* parts_out, std::vector<LayerDesc>* fit, int* Dw_out) {
  long off = 0;
  int Dw = 0;
  std::vector<PartDesc> parts = make_parts(c, off, Dw);
  for (int t = 0; t < c.ntypes; ++t) {
    int prev = Dw;
    for (int l = 0; l <= c.n_fit; ++l) {
      const bool last = (l == c.n_fit);
      const int no = last ? 1 : c.fit[l];
      LayerDesc L{prev, no, off, last ? 0 : skip_kind(prev, no), last ? 0 : 1};
      if (fit) fit->push_back(L);
      off += (long)prev * no + no;
      prev = no;
    }
  }
  if (parts_out) *parts_out = parts;
  if (Dw_out) *Dw_out = Dw;
  return off;
}

}  // namespace

dp_model_config list_config(const dp_model_config& c) {
  dp_model_config l = c;
  if (is_hybrid(c)) {
    l.rcut = std::max(c.rcut, c.rcut_2);
    for (int t = 0; t < c.ntypes; ++t) l.sel[t] = std::max(c.sel[t], c.sel_2[t]);
  }
  return l;
}

int check_finite_host(const double* x, long n) {
  for (long k = 0; k < n; ++k)
    if (!std::isfinite(x[k])) {
      set_error("non-finite coordinate (NaN or Inf) at atom " + std::to_string(k / 3));
      return DP_E_ARG;
    }
  return DP_OK;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void drop_graph(dp_model* md) {
  DpGraph& g = md->graph;
  if (g.exec) cudaGraphExecDestroy(g.exec);
  g.exec = nullptr;
  for (auto& r : g.prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g.prof.clear();
  g.sig.clear();
  g.launches = 0;
}

int ensure_ws(dp_model* md, size_t bytes) {
  if (bytes <= md->ws_cap) return DP_OK;
  drop_graph(md);  // a recorded graph points into the old scratch
  if (md->ws) {
    DP_CUDA_TRY(cudaDeviceSynchronize());
    cudaFree(md->ws);
    md->ws = nullptr;
    md->ws_cap = 0;
  }
  size_t cap = bytes + bytes / 8 + (1 << 20);
  DP_CUDA_TRY(cudaMalloc(&md->ws, cap));
  md->ws_cap = cap;
  return DP_OK;
}

int read_status(dp_model* md, cudaStream_t st, int* n_overflow) {
  DP_CUDA_TRY(cudaMemcpyAsync(md->status_host, md->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
  DP_CUDA_TRY(cudaStreamSynchronize(st));
  md->prof.collect();
  const DevStatus s = *md->status_host;
  if (md->prof.timing && md->m.mom_npass) {  // issued MMA work of the moment kernels
    // one block: 128 accumulator rows x 64 x the padded width M, times the passes
    const double per = 2.0 * 128.0 * 64.0 * md->m.mom_npad * md->m.mom_npass;
    if (s.mma_blocks[0]) md->prof.work[md->prof.id_of("mom_fwd")] += per * s.mma_blocks[0];
    if (s.mma_blocks[1]) md->prof.work[md->prof.id_of("mom_bwd")] += per * s.mma_blocks[1];
  }
  if (n_overflow) *n_overflow = s.sel_overflow;
  if (s.bad_coord) {
    set_error("non-finite coordinate (NaN or Inf): results of this call are not valid");
    return DP_E_ARG;
  }
  if (s.bad_type) {
    set_error("atom type outside [0, ntypes)");
    return DP_E_ARG;
  }
  if (s.type_change) return kStatusTypeChange;
  if (s.capacity == 2) {
    set_error("periodic image index beyond +-511 cells: coordinates too far outside the box");
    return DP_E_ARG;
  }
  if (s.capacity) {
    set_error("more than DP_MAX_CANDIDATES atoms within r_c of one atom");
    return DP_E_CAPACITY;
  }
  if (s.sel_overflow) {
    set_error("neighbour count exceeded sel for " + std::to_string(s.sel_overflow) + " (atom, type) blocks");
    return DP_E_SEL_OVERFLOW;
  }
  if (s.timeout) {
    set_error("a bounded wait inside a tensor-core kernel gave up; results are invalid");
    return DP_E_TIMEOUT;
  }
  if (s.table_range) {
    set_error("compressed model: s outside the tabulated range (last piece extrapolated)");
    return DP_E_RANGE;
  }
  return DP_OK;
}

// Host-side per-type atom counts when types are on the host; else read back.
int type_starts(const int* type_host, const int* dtype_start, int N, int ntypes, cudaStream_t st, int* out) {
  if (type_host) {
    std::vector<int> cnt(ntypes, 0);
    for (int i = 0; i < N; ++i) {
      if (type_host[i] < 0 || type_host[i] >= ntypes) {
        set_error("atom type outside [0, ntypes)");
        return DP_E_ARG;
      }
      cnt[type_host[i]]++;
    }
    out[0] = 0;
    for (int t = 0; t < ntypes; ++t) out[t + 1] = out[t] + cnt[t];
    return DP_OK;
  }
  DP_CUDA_TRY(cudaMemcpyAsync(out, dtype_start, sizeof(int) * (ntypes + 1), cudaMemcpyDeviceToHost, st));
  DP_CUDA_TRY(cudaStreamSynchronize(st));
  if (out[ntypes] != N) {
    set_error("atom type outside [0, ntypes)");
    return DP_E_ARG;
  }
  return DP_OK;
}

int ensure_stage(dp_model* md, size_t bytes) {
  if (bytes <= md->stage_cap) return DP_OK;
  if (md->stage) cudaFreeHost(md->stage);
  md->stage = nullptr;
  md->stage_cap = 0;
  const size_t cap = bytes + bytes / 4 + 4096;
  DP_CUDA_TRY(cudaMallocHost(&md->stage, cap));
  md->stage_cap = cap;
  return DP_OK;
}

}  // namespace dpgb

using namespace dpgb;

extern "C" {

int dp_last_error(char* buf, int len) {
  if (buf && len > 0) {
    const size_t n = std::min(g_err.size(), (size_t)len - 1);
    std::memcpy(buf, g_err.data(), n);
    buf[n] = 0;
  }
  return (int)g_err.size();
}

int dp_wait_selftest(long spin_limit, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  int* err = nullptr;
  DP_CUDA_TRY(cudaMalloc(&err, sizeof(int)));
  int herr = -1;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 32, 0, st>>>(spin_limit > 0 ? spin_limit : ptx::kSpin, err);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(err);
  if (e != cudaSuccess) {
    set_error(std::string("wait self-test: ") + cudaGetErrorString(e));
    return DP_E_CUDA;
  }
  if (herr) {
    set_error("wait self-test: the bounded wait gave up, as intended");
    return DP_E_TIMEOUT;
  }
  return DP_OK;
}

long dp_model_n_params(const dp_model_config* cfg) {
  if (check_config(cfg) != DP_OK) return -1;
  return layout(*cfg, nullptr, nullptr, nullptr);
}

int dp_model_create(const dp_model_config* cfg, const double* params, long n_params, int device, int precision,
                    int compressed, dp_model** out) {
  if (!out || !params) {
    set_error("null argument");
    return DP_E_ARG;
  }
  *out = nullptr;
  if (check_config(cfg) != DP_OK) {
    set_error("invalid model configuration");
    return DP_E_ARG;
  }
  if (precision < DP_PREC_FP64 || precision > DP_PREC_BF16) {
    set_error("unknown precision");
    return DP_E_ARG;
  }
  dp_model* md = new dp_model();
  DeviceModel& m = md->m;
  m.cfg = *cfg;
  m.device = device;
  m.precision = precision;
  m.compressed = compressed ? 1 : 0;
  m.n_params = layout(*cfg, &m.parts, &m.fit, &m.Dw);
  m.emb = m.parts[0].emb;
  m.lcfg = list_config(*cfg);
  m.n_fit_layers = cfg->n_fit + 1;
  if (n_params != m.n_params) {
    set_error("n_params does not match the configuration (" + std::to_string(m.n_params) + " expected)");
    delete md;
    return DP_E_ARG;
  }
  m.nc = 0;
  for (int t = 0; t < cfg->ntypes; ++t) {
    m.sel_off[t] = m.nc;
    m.nc += m.lcfg.sel[t];
  }
  m.sel_off[cfg->ntypes] = m.nc;
  m.M = m.parts[0].M;
  m.A = m.parts[0].A;
  m.n_embed_nets = m.parts[0].n_nets;
  const bool one_part = cfg->descriptor == DP_DESC_SE_E2_R || cfg->descriptor == DP_DESC_SE_E3;
  if (cfg->descriptor != DP_DESC_SE_E2_A && (precision > DP_PREC_FP32 || (compressed && !one_part))) {
    set_error("se_e2_r and se_e3 models run in FP64 or FP32, compressed or not; hybrids uncompressed");
    delete md;
    return DP_E_UNSUPPORTED;
  }
  for (const PartDesc& P : m.parts)
    if (P.kind == PART_E3 && !e3_supported(P, precision)) {
      set_error("se_e3 embedding widths above 32, or nets too large for shared memory");
      delete md;
      return DP_E_UNSUPPORTED;
    }
  if (precision == DP_PREC_TF32 && compressed) {
    set_error("TF32 applies to the network GEMMs of the uncompressed model");
    delete md;
    return DP_E_UNSUPPORTED;
  }
  const bool tc_uncompressed = !compressed && (precision == DP_PREC_TF32 || precision == DP_PREC_BF16);
  if (tc_uncompressed && !tc_uncompressed_supported(m)) {
    set_error("tensor-core network GEMMs need widths <= 256, at most 8 (centre, neighbour) type pairs, "
              "M * M_< a multiple of 16, two or more embedding layers and a hidden fitting layer");
    delete md;
    return DP_E_UNSUPPORTED;
  }
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    set_error(std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    delete md;
    return DP_E_CUDA;
  }
  std::vector<float> p32(params, params + n_params);
  e = cudaMalloc(&m.p64, sizeof(double) * n_params);
  if (e == cudaSuccess) e = cudaMalloc(&m.p32, sizeof(float) * n_params);
  if (e == cudaSuccess) e = cudaMemcpy(m.p64, params, sizeof(double) * n_params, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m.p32, p32.data(), sizeof(float) * n_params, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&md->status, sizeof(DevStatus));
  if (e == cudaSuccess) e = cudaMallocHost(&md->status_host, sizeof(DevStatus));
  if (e != cudaSuccess) {
    set_error(std::string("model upload: ") + cudaGetErrorString(e));
    dp_free_model(md);
    return e == cudaErrorMemoryAllocation ? DP_E_OOM : DP_E_CUDA;
  }
  if (compressed) {
    int rc = build_tables(m);
    if (rc != DP_OK) {
      dp_free_model(md);
      return rc;
    }
  }
  for (int t = 0; t < cfg->ntypes; ++t) {
    const LayerDesc& Lo = m.fit[(size_t)t * m.n_fit_layers + m.n_fit_layers - 1];
    m.fit_out_bias[t] = (float)params[Lo.w_off + Lo.n_in];
  }
  if (tc_uncompressed) {
    int rc = tc_uncompressed_prepare(m, params);
    if (rc != DP_OK) {
      dp_free_model(md);
      return rc;
    }
  }
  if (precision == DP_PREC_BF16 && compressed) {
    int rc = prepare_fit_bf16(m, params);
    if (rc != DP_OK) {
      dp_free_model(md);
      return rc;
    }
  }
  // FP32 compressed models run the fitting net on split BF16 operands (three tensor-core passes,
  // about 16 significant bits per operand) where its shapes fit the tensor-core kernels
  if (precision == DP_PREC_FP32 && compressed && fit_tc_supported(m)) {
    int rc = prepare_fit_bf16(m, params, true);
    if (rc != DP_OK) {
      dp_free_model(md);
      return rc;
    }
  }
  *out = md;
  return DP_OK;
}

int dp_model_set_params(dp_model* md, const double* params, long n_params, void* stream) {
  if (!md || !params || n_params != md->m.n_params) {
    set_error("invalid argument (params must hold exactly the model's n_params values)");
    return DP_E_ARG;
  }
  DeviceModel& m = md->m;
  if (m.compressed) {
    set_error("compressed models hold tabulated nets: create a new model to change parameters");
    return DP_E_UNSUPPORTED;
  }
  DP_CUDA_TRY(cudaSetDevice(m.device));
  cudaStream_t st = (cudaStream_t)stream;
  const cudaMemcpyKind kind = is_device_ptr(params) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  DP_CUDA_TRY(cudaMemcpyAsync(m.p64, params, sizeof(double) * n_params, kind, st));
  k_narrow<<<(unsigned)((n_params + 255) / 256), 256, 0, st>>>(m.p64, n_params, m.p32);
  DP_CUDA_TRY(cudaGetLastError());
  DP_CUDA_TRY(cudaStreamSynchronize(st));
  return DP_OK;
}

int dp_init_model(const char* path, int device, int precision, int compressed, dp_model** out) {
  if (!path || !out) {
    set_error("null argument");
    return DP_E_ARG;
  }
  FILE* f = std::fopen(path, "rb");
  if (!f) {
    set_error(std::string("cannot open ") + path);
    return DP_E_ARG;
  }
  char magic[8];
  dp_model_config cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  long long n = 0;
  bool ok = std::fread(magic, 1, 8, f) == 8;
  // version 1 files hold the struct up to type_one_side (se_e2_a models)
  const bool v1 = ok && std::memcmp(magic, "DPGBW001", 8) == 0;
  ok = ok && (v1 || std::memcmp(magic, "DPGBW002", 8) == 0);
  const size_t cfg_bytes = v1 ? offsetof(dp_model_config, descriptor) : sizeof(cfg);
  ok = ok && std::fread(&cfg, 1, cfg_bytes, f) == cfg_bytes && std::fread(&n, sizeof(n), 1, f) == 1 && n > 0 &&
       n < (1LL << 34);
  std::vector<double> p;
  if (ok) {
    p.resize((size_t)n);
    ok = std::fread(p.data(), sizeof(double), (size_t)n, f) == (size_t)n;
  }
  std::fclose(f);
  if (!ok) {
    set_error(std::string("malformed weight file ") + path);
    return DP_E_ARG;
  }
  return dp_model_create(&cfg, p.data(), (long)n, device, precision, compressed, out);
}

int dp_gemm_bf16(int rows, int K, int N, const void* A, const void* Bt, float* C, void* stream) {
  if (rows < 1 || K < 8 || K % 8 || N < 1 || !is_device_ptr(A) || !is_device_ptr(Bt) || !is_device_ptr(C)) {
    set_error("dp_gemm_bf16: device pointers, rows >= 1, K a multiple of 8, N >= 1");
    return DP_E_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int* err = nullptr;
  DP_CUDA_TRY(cudaGetSymbolAddress((void**)&err, g_gemm_err));
  TcArgs a;
  std::memset(&a, 0, sizeof(a));
  a.ntypes = 1;
  a.row_start[1] = rows;
  a.tile_start[1] = (rows + 127) / 128;
  a.K = K;
  a.N = N;
  a.BN = tc_pick_bn(N, a.tile_start[1]);
  a.out_f32 = C;
  a.err = err;
  CUtensorMap ta;
  TcMaps tb;
  int rc = make_tmap_bf16(&ta, A, rows, K, 128);
  if (rc == DP_OK) rc = make_tmap_bf16(&tb.m[0], Bt, N, K, a.BN);
  if (rc != DP_OK) return rc;
  DP_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
  DP_CUDA_TRY(launch_tc_gemm(TC_EPI_PLAIN, ta, tb, a, st));
  int herr = 0;
  DP_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  DP_CUDA_TRY(cudaStreamSynchronize(st));
  if (herr) {
    set_error("tensor-core GEMM: a bounded pipeline wait timed out");
    return DP_E_TIMEOUT;
  }
  return DP_OK;
}

int dp_model_export_table(const dp_model* md, double* out, int* n_intervals) {
  if (!md || !out || !md->m.compressed) {
    set_error("invalid argument or model not compressed");
    return DP_E_ARG;
  }
  DP_CUDA_TRY(cudaSetDevice(md->m.device));
  if (n_intervals) *n_intervals = md->m.tab.n1 + md->m.tab.n2;
  return export_tables(md->m, out);
}

int dp_profile_enable(dp_model* md, int on) {
  if (!md) return DP_E_ARG;
  md->prof.collect();
  md->prof.timing = on != 0;
  return DP_OK;
}

int dp_profile_reset(dp_model* md) {
  if (!md) return DP_E_ARG;
  md->prof.reset();
  return DP_OK;
}

int dp_profile_count(const dp_model* md) { return md ? (int)md->prof.names.size() : 0; }

int dp_profile_read(const dp_model* md, int k, char* name, int name_len, double* total_ms, long* count) {
  if (!md || k < 0 || k >= (int)md->prof.names.size()) return DP_E_ARG;
  if (name && name_len > 0) {
    std::strncpy(name, md->prof.names[k].c_str(), (size_t)name_len - 1);
    name[name_len - 1] = 0;
  }
  if (total_ms) *total_ms = md->prof.total_ms[k];
  if (count) *count = md->prof.count[k];
  return DP_OK;
}

long dp_launch_count(const dp_model* md) { return md ? md->prof.launches : -1; }

int dp_profile_work(const dp_model* md, int k, double* flop) {
  if (!md || !flop || k < 0 || k >= (int)md->prof.names.size()) return DP_E_ARG;
  *flop = md->prof.work[k];
  return DP_OK;
}

int dp_free_model(dp_model* md) {
  if (!md) return DP_OK;
  cudaSetDevice(md->m.device);
  cudaFree(md->m.p64);
  cudaFree(md->m.p32);
  cudaFree(md->m.tab64);
  cudaFree(md->m.tab32);
  cudaFree(md->m.mom_tab);
  cudaFree(md->m.fit_wt_bf16);
  cudaFree(md->m.fit_w_bf16);
  cudaFree(md->m.fit_wt_bf16_lo);
  cudaFree(md->m.fit_w_bf16_lo);
  cudaFree(md->m.tc_wt);
  cudaFree(md->m.tc_w);
  cudaFree(md->ws);
  cudaFree(md->status);
  if (md->status_host) cudaFreeHost(md->status_host);
  if (md->stage) cudaFreeHost(md->stage);
  drop_graph(md);
  if (md->graph.stage) cudaFreeHost(md->graph.stage);
  if (md->cap_st) cudaStreamDestroy(md->cap_st);
  delete md;
  return DP_OK;
}

int dp_nlist_export(const dp_nlist* nl, int* nl_j, int* nl_shift) {
  if (!nl || !nl_j || !nl_shift) {
    set_error("invalid argument");
    return DP_E_ARG;
  }
  DP_CUDA_TRY(cudaSetDevice(nl->device));
  const size_t n = (size_t)nl->natoms * nl->nc;
  std::vector<int> code(n);
  DP_CUDA_TRY(cudaMemcpy(nl_j, nl->nl_j, sizeof(int) * n, cudaMemcpyDeviceToHost));
  DP_CUDA_TRY(cudaMemcpy(code.data(), nl->nl_code, sizeof(int) * n, cudaMemcpyDeviceToHost));
  for (size_t k = 0; k < n; ++k) unpack_shift(code[k], nl_shift[3 * k], nl_shift[3 * k + 1], nl_shift[3 * k + 2]);
  return DP_OK;
}

int dp_free_nlist(dp_nlist* nl) {
  if (!nl) return DP_OK;
  cudaSetDevice(nl->device);
  cudaFree(nl->nl_j);
  cudaFree(nl->nl_code);
  cudaFree(nl->counts);
  delete nl;
  return DP_OK;
}

}  // extern "C"
