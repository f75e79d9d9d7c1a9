// C ABI of libdpgb: model and neighbour-list objects, scratch management, and the
// per-frame driver that chains the kernels of the se_e2_a path.
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "dp_internal.cuh"
#include "fit_tc.cuh"
#include "path.cuh"
#include "table.cuh"
#include "tc_gemm.cuh"

struct dp_model {
  dpgb::DeviceModel m;
  char* ws = nullptr;  // cached scratch
  size_t ws_cap = 0;
  dpgb::DevStatus* status = nullptr;  // device
  dpgb::DevStatus* status_host = nullptr;  // pinned
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

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }

// error word of the stand-alone tensor-core GEMM entry point
__device__ int g_gemm_err;

namespace {

int skip_kind(int n_in, int n_out) { return n_out == n_in ? 1 : (n_out == 2 * n_in ? 2 : 0); }

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
  if (c->axis < 1 || c->axis > c->embed[c->n_embed - 1]) return DP_E_ARG;
  if (!(c->rcut > 0) || !(c->rcut_smth >= 0) || !(c->rcut_smth < c->rcut)) return DP_E_ARG;
  return DP_OK;
}

long layout(const dp_model_config& c, std::vector<LayerDesc>* emb, std::vector<LayerDesc>* fit) {
  const int nets = c.type_one_side ? c.ntypes : c.ntypes * c.ntypes;
  long off = 0;
  for (int n = 0; n < nets; ++n) {
    int prev = 1;
    for (int l = 0; l < c.n_embed; ++l) {
      LayerDesc L{prev, c.embed[l], off, skip_kind(prev, c.embed[l]), 1};
      if (emb) emb->push_back(L);
      off += (long)prev * c.embed[l] + c.embed[l];
      prev = c.embed[l];
    }
  }
  const int M = c.embed[c.n_embed - 1];
  for (int t = 0; t < c.ntypes; ++t) {
    int prev = M * c.axis;
    for (int l = 0; l <= c.n_fit; ++l) {
      const bool last = (l == c.n_fit);
      const int no = last ? 1 : c.fit[l];
      LayerDesc L{prev, no, off, last ? 0 : skip_kind(prev, no), last ? 0 : 1};
      if (fit) fit->push_back(L);
      off += (long)prev * no + no;
      prev = no;
    }
  }
  return off;
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

int ensure_ws(dp_model* md, size_t bytes) {
  if (bytes <= md->ws_cap) return DP_OK;
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

struct FrameBufs {
  double* coord;
  int* type;
  int* nl_j;
  int* nl_code;
  int* counts;
  int* cell_count;
  int* cell_start;
  int* cell_cursor;
  int* cell_atoms;
  int* atom_cell;
  int* atom_img;
  float4* atom_wf;
  int* perm;
  int* type_start;
  double* energy;
  double* force;
  double* virial;
  double* atom_energy;
  double* bbox;
  double* tshift;
  double* epart;
};

// Carve the per-call buffers that precede the path scratch.
void carve(Arena& ar, const DeviceModel& m, int N, const NlGeom* g, bool own_nlist, bool copy_coord,
           bool copy_type, bool host_force, bool host_ae, FrameBufs& b) {
  std::memset(&b, 0, sizeof(b));
  const long nc = m.nc;
  if (copy_coord) b.coord = ar.get<double>(3L * N);
  if (copy_type) b.type = ar.get<int>(N);
  if (own_nlist) {
    const int ncells = g->ncell[0] * g->ncell[1] * g->ncell[2];
    b.nl_j = ar.get<int>(N * nc);
    b.nl_code = ar.get<int>(N * nc);
    b.counts = ar.get<int>((long)N * m.cfg.ntypes);
    b.cell_count = ar.get<int>(ncells);
    b.cell_start = ar.get<int>(ncells + 1);
    b.cell_cursor = ar.get<int>(ncells);
    b.cell_atoms = ar.get<int>(N);
    b.atom_cell = ar.get<int>(N);
    b.atom_img = ar.get<int>(3L * N);
    b.atom_wf = ar.get<float4>(N);
  }
  b.perm = ar.get<int>(N);
  b.type_start = ar.get<int>(DP_MAX_TYPES + 1);
  b.energy = ar.get<double>(1);
  b.virial = ar.get<double>(9);
  if (host_force) b.force = ar.get<double>(3L * N);
  if (host_ae) b.atom_energy = ar.get<double>(N);
  b.bbox = ar.get<double>(6);
  b.tshift = ar.get<double>(81);
  b.epart = ar.get<double>((N + 255) / 256);
}

int read_status(dp_model* md, cudaStream_t st, int* n_overflow) {
  DP_CUDA_TRY(cudaMemcpyAsync(md->status_host, md->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st));
  DP_CUDA_TRY(cudaStreamSynchronize(st));
  md->prof.collect();
  const DevStatus s = *md->status_host;
  if (n_overflow) *n_overflow = s.sel_overflow;
  if (s.bad_type) {
    set_error("atom type outside [0, ntypes)");
    return DP_E_ARG;
  }
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
  if (s.table_range) {
    set_error("compressed model: s outside the tabulated range (last piece extrapolated)");
    return DP_E_RANGE;
  }
  return DP_OK;
}

// Geometry for this frame (open boundary needs the bounding box of the coordinates).
int frame_geometry(dp_model* md, int N, const double* dcoord, const double* box, double* dbbox, cudaStream_t st,
                   NlGeom& g) {
  double lohi[6] = {0, 0, 0, 0, 0, 0};
  if (!box) {
    {
      ProfScope _ps(&md->prof, "bbox", st);
      DP_CUDA_TRY(launch_bbox(dcoord, N, dbbox, st));
    }
    DP_CUDA_TRY(cudaMemcpyAsync(lohi, dbbox, sizeof(lohi), cudaMemcpyDeviceToHost, st));
    DP_CUDA_TRY(cudaStreamSynchronize(st));
  }
  const int rc = host_geometry(md->m.cfg, N, box, lohi, g);
  if (md->nl_full_cap) g.cap = DP_MAX_CANDIDATES;
  return rc;
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

}  // namespace
}  // namespace dpgb

using namespace dpgb;

extern "C" {

const char* dp_last_error(void) { return g_err.c_str(); }

long dp_model_n_params(const dp_model_config* cfg) {
  if (check_config(cfg) != DP_OK) return -1;
  return layout(*cfg, nullptr, nullptr);
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
  m.n_params = layout(*cfg, &m.emb, &m.fit);
  m.n_fit_layers = cfg->n_fit + 1;
  if (n_params != m.n_params) {
    set_error("n_params does not match the configuration (" + std::to_string(m.n_params) + " expected)");
    delete md;
    return DP_E_ARG;
  }
  m.nc = 0;
  for (int t = 0; t < cfg->ntypes; ++t) {
    m.sel_off[t] = m.nc;
    m.nc += cfg->sel[t];
  }
  m.sel_off[cfg->ntypes] = m.nc;
  m.M = cfg->embed[cfg->n_embed - 1];
  m.A = cfg->axis;
  m.n_embed_nets = cfg->type_one_side ? cfg->ntypes : cfg->ntypes * cfg->ntypes;
  if (precision == DP_PREC_TF32 || (precision == DP_PREC_BF16 && !compressed)) {
    set_error("this precision needs the compressed embedding (BF16) or is not available (TF32)");
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
  if (precision == DP_PREC_BF16) {
    int rc = prepare_fit_bf16(m, params);
    if (rc != DP_OK) {
      dp_free_model(md);
      return rc;
    }
  }
  *out = md;
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
  long long n = 0;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "DPGBW001", 8) == 0 &&
            std::fread(&cfg, sizeof(cfg), 1, f) == 1 && std::fread(&n, sizeof(n), 1, f) == 1 && n > 0 &&
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
  a.BN = tc_pick_bn(N, a.tile_start[1], false);
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

int dp_free_model(dp_model* md) {
  if (!md) return DP_OK;
  cudaSetDevice(md->m.device);
  cudaFree(md->m.p64);
  cudaFree(md->m.p32);
  cudaFree(md->m.tab64);
  cudaFree(md->m.tab32);
  cudaFree(md->m.fit_wt_bf16);
  cudaFree(md->m.fit_w_bf16);
  cudaFree(md->ws);
  cudaFree(md->status);
  if (md->status_host) cudaFreeHost(md->status_host);
  delete md;
  return DP_OK;
}

int dp_build_nlist(dp_model* md, int N, const double* coord, const int* type, const double* box, dp_nlist** out,
                   int* n_overflow, void* stream) {
  if (!md || !coord || !type || !out || N < 1) {
    set_error("invalid argument");
    return DP_E_ARG;
  }
  *out = nullptr;
  DP_CUDA_TRY(cudaSetDevice(md->m.device));
  cudaStream_t st = (cudaStream_t)stream;
  const bool copy_coord = !is_device_ptr(coord), copy_type = !is_device_ptr(type);
  // first pass: sizes (geometry needs device coordinates only for open boundaries)
  Arena pre;
  pre.measure = true;
  FrameBufs b;
  NlGeom g;
  std::memset(&g, 0, sizeof(g));
  g.ncell[0] = g.ncell[1] = g.ncell[2] = 256;  // upper bound for sizing
  carve(pre, md->m, N, &g, true, copy_coord, copy_type, false, false, b);
  int rc = ensure_ws(md, pre.used);
  if (rc != DP_OK) return rc;
  Arena ar;
  ar.base = md->ws;
  ar.cap = md->ws_cap;
  carve(ar, md->m, N, &g, true, copy_coord, copy_type, false, false, b);
  const double* dcoord = copy_coord ? b.coord : coord;
  const int* dtype = copy_type ? b.type : type;
  if (copy_coord) DP_CUDA_TRY(cudaMemcpyAsync(b.coord, coord, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, st));
  if (copy_type) DP_CUDA_TRY(cudaMemcpyAsync(b.type, type, sizeof(int) * N, cudaMemcpyHostToDevice, st));
  rc = frame_geometry(md, N, dcoord, box, b.bbox, st, g);
  if (rc != DP_OK) return rc;
  dp_nlist* nl = new dp_nlist();
  nl->device = md->m.device;
  nl->natoms = N;
  nl->nc = md->m.nc;
  nl->ntypes = md->m.cfg.ntypes;
  cudaError_t e = cudaMalloc(&nl->nl_j, sizeof(int) * (size_t)N * nl->nc);
  if (e == cudaSuccess) e = cudaMalloc(&nl->nl_code, sizeof(int) * (size_t)N * nl->nc);
  if (e == cudaSuccess) e = cudaMalloc(&nl->counts, sizeof(int) * (size_t)N * nl->ntypes);
  if (e != cudaSuccess) {
    set_error(std::string("nlist allocation: ") + cudaGetErrorString(e));
    dp_free_nlist(nl);
    return DP_E_OOM;
  }
  DP_CUDA_TRY(cudaMemsetAsync(md->status, 0, sizeof(DevStatus), st));
  {
    ProfScope _ps(&md->prof, "nlist", st, 4);
    DP_CUDA_TRY(launch_nlist_build(g, dcoord, dtype, b.cell_count, b.cell_start, b.cell_cursor, b.cell_atoms,
                                   b.atom_cell, b.atom_img, b.atom_wf, nl->nl_j, nl->nl_code, nl->counts, md->status,
                                   st));
  }
  rc = read_status(md, st, n_overflow);
  if (rc != DP_OK && rc != DP_E_SEL_OVERFLOW) {
    dp_free_nlist(nl);
    if (rc == DP_E_CAPACITY && !md->nl_full_cap) {
      md->nl_full_cap = true;  // retry once with the full candidate buffer
      return dp_build_nlist(md, N, coord, type, box, out, n_overflow, stream);
    }
    return rc;
  }
  *out = nl;
  return rc;
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

int dp_compute(dp_model* md, dp_nlist* nlist, int N, const double* coord, const int* type, const double* box,
               double* energy, double* force, double* virial, double* atom_energy, void* stream) {
  if (!md || !coord || !type || !energy || !force || !virial || N < 1) {
    set_error("invalid argument");
    return DP_E_ARG;
  }
  if (nlist && (nlist->natoms != N || nlist->nc != md->m.nc || nlist->device != md->m.device)) {
    set_error("neighbour list does not match this frame/model");
    return DP_E_ARG;
  }
  DP_CUDA_TRY(cudaSetDevice(md->m.device));
  cudaStream_t st = (cudaStream_t)stream;
  const DeviceModel& m = md->m;
  const bool copy_coord = !is_device_ptr(coord), copy_type = !is_device_ptr(type);
  const bool host_e = !is_device_ptr(energy), host_f = !is_device_ptr(force), host_v = !is_device_ptr(virial);
  const bool host_ae = atom_energy && !is_device_ptr(atom_energy);
  const bool own_nlist = (nlist == nullptr);
  const bool fp64 = (m.precision == DP_PREC_FP64);
  // sizing pass
  NlGeom g;
  std::memset(&g, 0, sizeof(g));
  g.ncell[0] = g.ncell[1] = g.ncell[2] = 256;
  PathConst pc;
  std::memset(&pc, 0, sizeof(pc));
  pc.natoms = N;
  pc.nc = m.nc;
  pc.M = m.M;
  pc.A = m.A;
  pc.ntypes = m.cfg.ntypes;
  pc.type_one_side = m.cfg.type_one_side;
  for (int t = 0; t < m.cfg.ntypes; ++t) pc.sel[t] = m.cfg.sel[t];
  for (int t = 0; t <= m.cfg.ntypes; ++t) pc.sel_off[t] = m.sel_off[t];
  pc.rs = m.cfg.rcut_smth;
  pc.rc = m.cfg.rcut;
  {
    const double rn = m.cfg.rcut - 1.0 > 0.0 ? m.cfg.rcut - 1.0 : 0.0;
    pc.near2 = rn * rn;
  }
  PathIO io;
  std::memset(&io, 0, sizeof(io));
  Arena pre;
  pre.measure = true;
  FrameBufs b;
  carve(pre, m, N, &g, own_nlist, copy_coord, copy_type, host_f, host_ae, b);
  int rc = m.compressed ? run_compressed(m, pc, io, pre, st)
                        : (fp64 ? run_generic<double>(m, pc, m.p64, io, pre, st)
                                : run_generic<float>(m, pc, m.p32, io, pre, st));
  if (rc != DP_OK) return rc;
  rc = ensure_ws(md, pre.used);
  if (rc != DP_OK) return rc;
  Arena ar;
  ar.base = md->ws;
  ar.cap = md->ws_cap;
  carve(ar, m, N, &g, own_nlist, copy_coord, copy_type, host_f, host_ae, b);
  const double* dcoord = copy_coord ? b.coord : coord;
  const int* dtype = copy_type ? b.type : type;
  if (copy_coord) DP_CUDA_TRY(cudaMemcpyAsync(b.coord, coord, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, st));
  if (copy_type) DP_CUDA_TRY(cudaMemcpyAsync(b.type, type, sizeof(int) * N, cudaMemcpyHostToDevice, st));
  DP_CUDA_TRY(cudaMemsetAsync(md->status, 0, sizeof(DevStatus), st));
  rc = frame_geometry(md, N, dcoord, box, b.bbox, st, g);
  if (rc != DP_OK) return rc;
  if (own_nlist) {
    ProfScope _ps(&md->prof, "nlist", st, 4);
    DP_CUDA_TRY(launch_nlist_build(g, dcoord, dtype, b.cell_count, b.cell_start, b.cell_cursor, b.cell_atoms,
                                   b.atom_cell, b.atom_img, b.atom_wf, b.nl_j, b.nl_code, b.counts, md->status, st));
  }
  {
    ProfScope _ps(&md->prof, "type_perm", st);
    DP_CUDA_TRY(launch_type_perm(dtype, N, m.cfg.ntypes, b.perm, b.type_start, &md->status->bad_type, st));
  }
  rc = type_starts(copy_type ? type : nullptr, b.type_start, N, m.cfg.ntypes, st, io.type_start);
  if (rc != DP_OK) return rc;
  for (int k = 0; k < 9; ++k) pc.h[k] = g.h[k];
  pc.periodic = g.periodic;
  if (g.periodic) {
    pc.tshift = b.tshift;
    ProfScope _ps(&md->prof, "shift_table", st);
    DP_CUDA_TRY(launch_shift_table(pc, b.tshift, st));
  }
  io.coord = dcoord;
  io.type = dtype;
  io.perm = b.perm;
  io.nl_j = own_nlist ? b.nl_j : nlist->nl_j;
  io.nl_code = own_nlist ? b.nl_code : nlist->nl_code;
  io.energy = host_e ? b.energy : energy;
  io.virial = host_v ? b.virial : virial;
  io.force = host_f ? b.force : force;
  io.atom_energy = atom_energy ? (host_ae ? b.atom_energy : atom_energy) : nullptr;
  io.status = md->status;
  io.epart = b.epart;
  io.prof = &md->prof;
  DP_CUDA_TRY(cudaMemsetAsync(io.force, 0, sizeof(double) * 3 * N, st));
  rc = m.compressed ? run_compressed(m, pc, io, ar, st)
                    : (fp64 ? run_generic<double>(m, pc, m.p64, io, ar, st)
                            : run_generic<float>(m, pc, m.p32, io, ar, st));
  if (rc != DP_OK) return rc;
  if (host_e) DP_CUDA_TRY(cudaMemcpyAsync(energy, io.energy, sizeof(double), cudaMemcpyDeviceToHost, st));
  if (host_v) DP_CUDA_TRY(cudaMemcpyAsync(virial, io.virial, sizeof(double) * 9, cudaMemcpyDeviceToHost, st));
  if (host_f) DP_CUDA_TRY(cudaMemcpyAsync(force, io.force, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, st));
  if (host_ae)
    DP_CUDA_TRY(cudaMemcpyAsync(atom_energy, io.atom_energy, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
  rc = read_status(md, st, nullptr);
  if (rc == DP_E_CAPACITY && own_nlist && !md->nl_full_cap) {
    md->nl_full_cap = true;  // retry once with the full candidate buffer
    return dp_compute(md, nlist, N, coord, type, box, energy, force, virial, atom_energy, stream);
  }
  return rc;
}

}  // extern "C"
