// Host driver of the path over one or more frames of one model: dp_compute (one frame),
// dp_compute_batch (many frames with their own cells and atom counts, evaluated together by
// the same kernels), and dp_build_nlist.
//
// Frames are concatenated; every per-atom kernel is frame-agnostic except for the frame's
// cell (neighbour search, image shifts), which it reads from small per-frame tables uploaded
// once per call from pinned host memory.  Per-frame energy and virial are FP64 sums of the
// per-atom values over fixed 512-atom chunks (deterministic order), then over each frame's
// chunks.
#include <algorithm>
#include <cstring>
#include <vector>

#include "capi_internal.cuh"
#include "grad.cuh"
#include "table.cuh"

namespace dpgb {

namespace {

constexpr int kChunk = 128;  // atoms per fixed-order partial sum of the per-frame energy and virial

__global__ void k_atom_frame(const int* __restrict__ frame_start, int F, int N, int* __restrict__ atom_frame) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int lo = 0, hi = F - 1;  // last frame f with frame_start[f] <= i
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (frame_start[mid] <= i)
      lo = mid;
    else
      hi = mid - 1;
  }
  atom_frame[i] = lo;
}

__global__ void k_shift_tables(const double* __restrict__ boxes, double* __restrict__ out) {
  const int f = blockIdx.x, q = threadIdx.x;
  if (q >= 27) return;
  const double* h = boxes + 9L * f;
  const int n0 = q / 9 - 1, n1 = (q / 3) % 3 - 1, n2 = q % 3 - 1;
  for (int a = 0; a < 3; ++a)
    out[81L * f + q * 3 + a] = __dadd_rn(__dadd_rn(__dmul_rn((double)n0, h[a]), __dmul_rn((double)n1, h[3 + a])),
                                         __dmul_rn((double)n2, h[6 + a]));
}

// Per-chunk sums of atom energies and atom virials (10 values), fixed order; the block that
// finishes a frame's last chunk then forms the frame's sums from the chunk partials, thread k
// adding chunks k, k + 128, ... of the frame and a fixed tree over the threads (the order depends
// on the frame alone, not on the batch or on which block finished last).  fcount[f] counts the
// finished chunks of frame f; it is zero on entry and left zero.
__global__ void __launch_bounds__(kChunk)
    k_chunk_sums(const int* __restrict__ chunk, const double* __restrict__ ae, const double* __restrict__ av,
                 double* __restrict__ cpart, const int* __restrict__ frame_chunk, int nframes, int* __restrict__ fcount,
                 double* __restrict__ energy, double* __restrict__ virial) {
  static_assert(kChunk == 128, "four warps per chunk block");
  __shared__ double red[4][10];
  __shared__ int s_last;
  const int c = blockIdx.x;
  const int beg = chunk[2 * c], end = chunk[2 * c + 1];
  double acc[10];
#pragma unroll
  for (int q = 0; q < 10; ++q) acc[q] = 0.0;
  for (int i = beg + threadIdx.x; i < end; i += blockDim.x) {
    acc[0] += ae[i];
#pragma unroll
    for (int q = 0; q < 9; ++q) acc[1 + q] += av[9L * i + q];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 10; ++q) {
    double x = acc[q];
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    if (lane == 0) red[w][q] = x;
  }
  __syncthreads();
  int f = 0;  // frame of this chunk
  {
    int lo = 0, hi = nframes - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (frame_chunk[mid] <= c) lo = mid; else hi = mid - 1;
    }
    f = lo;
  }
  const int c0 = frame_chunk[f], c1 = frame_chunk[f + 1];
  if (threadIdx.x < 10) {
    double x = 0.0;
    for (int k = 0; k < 4; ++k) x += red[k][threadIdx.x];
    cpart[10L * c + threadIdx.x] = x;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&fcount[f], 1) == c1 - c0 - 1;
  __syncthreads();
  if (!s_last) return;  // block-uniform
  __threadfence();
  const int tid = threadIdx.x;
#pragma unroll
  for (int q = 0; q < 10; ++q) acc[q] = 0.0;
  for (int cc = c0 + tid; cc < c1; cc += kChunk)
#pragma unroll
    for (int q = 0; q < 10; ++q) acc[q] += __ldcg(cpart + 10L * cc + q);
#pragma unroll
  for (int q = 0; q < 10; ++q) {
    double x = acc[q];
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    if (lane == 0) red[w][q] = x;
  }
  __syncthreads();
  if (tid < 10) {
    const double x = (red[0][tid] + red[1][tid]) + (red[2][tid] + red[3][tid]);
    if (tid == 0)
      energy[f] = x;
    else
      virial[9L * f + tid - 1] = x;
  }
  if (tid == 0) fcount[f] = 0;
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// Per-frame tables, laid out identically in pinned staging and on the device.
struct FrameTables {
  int F = 0, N = 0, C = 0;
  int ncells = 0, cap = 0, periodic = 1;
  std::vector<int> start, cell_off, chunk, frame_chunk;
  std::vector<NlGeom> geoms;
  std::vector<double> boxes;
  size_t off_geoms = 0, off_celloff = 0, off_start = 0, off_chunk = 0, off_fchunk = 0, off_boxes = 0, bytes = 0;

  void layout() {
    size_t o = 0;
    off_geoms = o;
    o += a256(sizeof(NlGeom) * F);
    off_celloff = o;
    o += a256(sizeof(int) * (F + 1));
    off_start = o;
    o += a256(sizeof(int) * (F + 1));
    off_chunk = o;
    o += a256(sizeof(int) * 2 * C);
    off_fchunk = o;
    o += a256(sizeof(int) * (F + 1));
    off_boxes = o;
    o += a256(sizeof(double) * 9 * F);
    bytes = o;
  }
  int max_noff() const {
    int m = 0;
    for (const NlGeom& g : geoms) m = std::max(m, (2 * g.K[0] + 1) * (2 * g.K[1] + 1) * (2 * g.K[2] + 1));
    return m;
  }
  // Largest mean candidate stream of one cell, frame by frame: atoms per cell times the cells
  // of its stencil.
  int max_stream() const {
    double m = 0.0;
    for (int f = 0; f < F; ++f) {
      const NlGeom& g = geoms[f];
      const double per_cell = (double)(start[f + 1] - start[f]) / std::max(1, g.ncell[0] * g.ncell[1] * g.ncell[2]);
      m = std::max(m, per_cell * (2 * g.K[0] + 1) * (2 * g.K[1] + 1) * (2 * g.K[2] + 1));
    }
    return (int)std::ceil(m);
  }
  void pack(unsigned char* p) const {
    std::memcpy(p + off_geoms, geoms.data(), sizeof(NlGeom) * F);
    std::memcpy(p + off_celloff, cell_off.data(), sizeof(int) * (F + 1));
    std::memcpy(p + off_start, start.data(), sizeof(int) * (F + 1));
    std::memcpy(p + off_chunk, chunk.data(), sizeof(int) * 2 * C);
    std::memcpy(p + off_fchunk, frame_chunk.data(), sizeof(int) * (F + 1));
    std::memcpy(p + off_boxes, boxes.data(), sizeof(double) * 9 * F);
  }
};

int build_tables_host(dp_model* md, int F, const int* natoms, const double* boxes, const double* lohi,
                      FrameTables& T) {
  T.F = F;
  T.start.assign(F + 1, 0);
  for (int f = 0; f < F; ++f) {
    if (natoms[f] < 1) {
      set_error("every frame needs at least one atom");
      return DP_E_ARG;
    }
    T.start[f + 1] = T.start[f] + natoms[f];
  }
  T.N = T.start[F];
  T.periodic = boxes ? 1 : 0;
  T.geoms.resize(F);
  T.cell_off.assign(F + 1, 0);
  T.boxes.assign(9 * (size_t)F, 0.0);
  T.cap = 0;
  for (int f = 0; f < F; ++f) {
    const int rc = host_geometry(md->m.lcfg, natoms[f], boxes ? boxes + 9 * f : nullptr, lohi, T.geoms[f]);
    if (rc != DP_OK) return rc;
    NlGeom& g = T.geoms[f];
    if (md->nl_full_cap) g.cap = DP_MAX_CANDIDATES;
    T.cap = std::max(T.cap, g.cap);
    T.cell_off[f + 1] = T.cell_off[f] + g.ncell[0] * g.ncell[1] * g.ncell[2];
    if (boxes)
      for (int k = 0; k < 9; ++k) T.boxes[9 * f + k] = boxes[9 * f + k];
  }
  T.ncells = T.cell_off[F];
  T.chunk.clear();
  T.frame_chunk.assign(F + 1, 0);
  for (int f = 0; f < F; ++f) {
    for (int b = T.start[f]; b < T.start[f + 1]; b += kChunk) {
      T.chunk.push_back(b);
      T.chunk.push_back(std::min(b + kChunk, T.start[f + 1]));
    }
    T.frame_chunk[f + 1] = (int)T.chunk.size() / 2;
  }
  T.C = (int)T.chunk.size() / 2;
  T.layout();
  return DP_OK;
}

struct Bufs {
  double* coord;
  int* type;
  int *nl_j, *nl_code, *counts;
  int *cell_count, *cell_start;
  int2* atom_key;
  float4 *atom_l, *sorted_l, *disp;
  int4 *atom_m, *sorted_m;
  unsigned char* ftab;
  int* atom_frame;
  double* tshift;
  int *perm, *type_start;
  double *energy, *virial, *force, *atom_energy, *atom_virial, *cpart, *epart;
  int* fcount;  // finished chunks per frame (k_chunk_sums)
};

void carve(Arena& ar, const DeviceModel& m, const FrameTables& T, bool own_nlist, bool copy_coord, bool copy_type,
           bool host_e, bool host_v, bool host_f, bool dev_ae, Bufs& b) {
  std::memset(&b, 0, sizeof(b));
  const long N = T.N, nc = m.nc;
  if (copy_coord) b.coord = ar.get<double>(3 * N);
  if (copy_type) b.type = ar.get<int>(N);
  if (own_nlist) {
    b.nl_j = ar.get<int>(N * nc);
    b.nl_code = ar.get<int>(N * nc);
    b.counts = ar.get<int>(N * m.cfg.ntypes);
    const long nkeys = (long)T.ncells * m.cfg.ntypes;
    b.cell_count = ar.get<int>(nkeys);
    b.cell_start = ar.get<int>(nkeys + 1);
    b.atom_key = ar.get<int2>(N);
    b.atom_l = ar.get<float4>(N);
    b.atom_m = ar.get<int4>(N);
    b.sorted_l = ar.get<float4>(N);
    b.sorted_m = ar.get<int4>(N);
    if (m.compressed && m.mom_npass == 1) b.disp = ar.get<float4>(N * nc);  // mixed mode's FP32 displacements
  }
  b.ftab = ar.get<unsigned char>((long)T.bytes);
  if (T.F > 1) b.atom_frame = ar.get<int>(N);
  b.tshift = ar.get<double>(81L * T.F);
  b.perm = ar.get<int>(N);
  b.type_start = ar.get<int>(DP_MAX_TYPES + 1);
  if (host_e) b.energy = ar.get<double>(T.F);
  if (host_v) b.virial = ar.get<double>(9L * T.F);
  if (host_f) b.force = ar.get<double>(3 * N);
  if (!dev_ae) b.atom_energy = ar.get<double>(N);
  b.atom_virial = ar.get<double>(9 * N);
  b.cpart = ar.get<double>(10L * T.C);
  b.fcount = ar.get<int>(T.F);
  b.epart = ar.get<double>((N + 255) / 256);
}

int host_bbox(const double* coord, int N, double* lohi) {
  for (int a = 0; a < 3; ++a) {
    lohi[a] = 1e300;
    lohi[3 + a] = -1e300;
  }
  for (int i = 0; i < N; ++i)
    for (int a = 0; a < 3; ++a) {
      lohi[a] = std::min(lohi[a], coord[3 * i + a]);
      lohi[3 + a] = std::max(lohi[3 + a], coord[3 * i + a]);
    }
  return DP_OK;
}

// Bounding box of device coordinates (open boundaries), read back once.
int device_bbox(dp_model* md, const double* dcoord, int N, cudaStream_t st, double* lohi) {
  double* d = nullptr;
  DP_CUDA_TRY(cudaMallocAsync(&d, sizeof(double) * 6, st));
  {
    ProfScope _ps(&md->prof, "bbox", st);
    DP_CUDA_TRY(launch_bbox(dcoord, N, d, st));
  }
  DP_CUDA_TRY(cudaMemcpyAsync(lohi, d, sizeof(double) * 6, cudaMemcpyDeviceToHost, st));
  DP_CUDA_TRY(cudaFreeAsync(d, st));
  DP_CUDA_TRY(cudaStreamSynchronize(st));
  return DP_OK;
}

PathConst make_pc(const DeviceModel& m, int N) {
  PathConst pc;
  std::memset(&pc, 0, sizeof(pc));
  pc.natoms = N;
  pc.nc = m.nc;
  pc.M = m.M;
  pc.A = m.A;
  pc.Dw = m.Dw;
  pc.doff = 0;
  pc.kind = m.parts[0].kind;
  pc.ntypes = m.cfg.ntypes;
  pc.type_one_side = m.cfg.type_one_side;
  // list geometry (for a one-part model, the part's own)
  for (int t = 0; t < m.cfg.ntypes; ++t) pc.sel[t] = m.lcfg.sel[t];
  for (int t = 0; t <= m.cfg.ntypes; ++t) pc.sel_off[t] = pc.lsel_off[t] = m.sel_off[t];
  pc.lnc = m.nc;
  pc.rs = m.parts[0].rs;
  pc.rc = m.lcfg.rcut;
  pc.rc2 = m.lcfg.rcut * m.lcfg.rcut;
  return pc;
}

int run_path(const DeviceModel& m, const PathConst& pc, const PathIO& io, Arena& ar, cudaStream_t st) {
  if (m.compressed && m.cfg.descriptor == DP_DESC_SE_E2_A) return run_compressed(m, pc, io, ar, st);
  if (m.precision == DP_PREC_TF32 || m.precision == DP_PREC_BF16) return run_tc_uncompressed(m, pc, io, ar, st);
  if (m.precision == DP_PREC_FP64) return run_generic<double>(m, pc, m.p64, io, ar, st);
  return run_generic<float>(m, pc, m.p32, io, ar, st);
}

// Parameter-gradient request: dPhi/dtheta for Phi = sum_f g_energy[f] E_f + sum_i g_force[i] . F_i.
struct GradReq {
  const double* g_energy;  // [F] host or device
  const double* g_force;   // [N][3] host or device
  const double* g_virial;  // [F][9] host or device, or null
  double* grad;            // [n_params] host or device
};

// The whole path over F frames.  nlist (F == 1 only) replaces the internal list build.  With
// gr set, the call computes the parameter gradient instead of energy / force / virial.
int run_frames(dp_model* md, dp_nlist* nlist, int F, const int* natoms, const double* coord, const int* type,
               const double* boxes, double* energy, double* force, double* virial, double* atom_energy,
               cudaStream_t st, const GradReq* gr = nullptr) {
  const DeviceModel& m = md->m;
  DP_CUDA_TRY(cudaSetDevice(m.device));
  const bool copy_coord = !is_device_ptr(coord), copy_type = !is_device_ptr(type);
  const bool host_e = !is_device_ptr(energy), host_f = !is_device_ptr(force), host_v = !is_device_ptr(virial);
  const bool dev_ae = atom_energy && is_device_ptr(atom_energy);
  const bool own_nlist = (nlist == nullptr);
  int Ntot = 0;
  for (int f = 0; f < F; ++f) Ntot += natoms[f];
  if (copy_coord) {  // host coordinates are checked before any work is queued
    const int rc0 = check_finite_host(coord, 3L * Ntot);
    if (rc0 != DP_OK) return rc0;
  }
  // open boundaries (one frame): the cell grid needs the bounding box first
  double lohi[6] = {0, 0, 0, 0, 0, 0};
  if (!boxes) {
    if (F != 1) {
      set_error("batches of frames need periodic cells");
      return DP_E_UNSUPPORTED;
    }
    const int rc = copy_coord ? host_bbox(coord, Ntot, lohi) : device_bbox(md, coord, Ntot, st, lohi);
    if (rc != DP_OK) return rc;
  }
  FrameTables T;
  int rc = build_tables_host(md, F, natoms, boxes, lohi, T);
  if (rc != DP_OK) return rc;
  const int N = T.N;
  PathConst pc = make_pc(m, N);
  PathIO io;
  std::memset(&io, 0, sizeof(io));
  // sizing pass, then the real carve
  Arena pre;
  pre.measure = true;
  Bufs b;
  carve(pre, m, T, own_nlist, copy_coord, copy_type, host_e, host_v, host_f, dev_ae, b);
  // gradient mode: device copies of the seeds and of the result where the caller's are host arrays
  const bool g_a_host = gr && !is_device_ptr(gr->g_energy), g_w_host = gr && !is_device_ptr(gr->g_force),
             g_v_host = gr && gr->g_virial && !is_device_ptr(gr->g_virial),
             g_out_host = gr && !is_device_ptr(gr->grad);
  double *d_ga = nullptr, *d_gw = nullptr, *d_gv = nullptr, *d_gout = nullptr;
  auto carve_grad = [&](Arena& a) {
    d_ga = g_a_host ? a.get<double>(F) : const_cast<double*>(gr ? gr->g_energy : nullptr);
    d_gw = g_w_host ? a.get<double>(3L * N) : const_cast<double*>(gr ? gr->g_force : nullptr);
    d_gv = g_v_host ? a.get<double>(9L * F) : const_cast<double*>(gr ? gr->g_virial : nullptr);
    d_gout = g_out_host ? a.get<double>(m.n_params) : (gr ? gr->grad : nullptr);
  };
  carve_grad(pre);
  rc = gr ? run_param_grad(m, pc, io, nullptr, nullptr, nullptr, -1.0, nullptr, pre, st) : run_path(m, pc, io, pre, st);
  if (rc != DP_OK) return rc;
  rc = ensure_ws(md, pre.used);
  if (rc == DP_OK) rc = ensure_stage(md, T.bytes);
  if (rc != DP_OK) return rc;
  Arena ar;
  ar.base = md->ws;
  ar.cap = md->ws_cap;
  carve(ar, m, T, own_nlist, copy_coord, copy_type, host_e, host_v, host_f, dev_ae, b);
  carve_grad(ar);
  const double* dcoord = copy_coord ? b.coord : coord;
  const int* dtype = copy_type ? b.type : type;

  // per-type starts of the type-sorted order: counted here for host types, the counts of the
  // last call for the same device array (checked on the device), else read back mid-call
  TypeStartCheck chk;
  std::memset(&chk, 0, sizeof(chk));
  bool ts_known = false;
  if (copy_type) {
    rc = type_starts(type, nullptr, N, m.cfg.ntypes, st, io.type_start);
    if (rc != DP_OK) return rc;
    ts_known = true;
  } else if (md->ts_ptr == type && md->ts_n == N) {
    for (int t = 0; t <= m.cfg.ntypes; ++t) io.type_start[t] = md->ts_v[t];
    ts_known = true;
  }
  if (ts_known) {
    chk.on = 1;
    for (int t = 0; t <= m.cfg.ntypes; ++t) chk.v[t] = io.type_start[t];
  }

  // All device work of the call, in stream order on s (tables uploaded from `stage`); the
  // path's scratch is carved afresh from the same arena position every time.
  const size_t ar_used0 = ar.used;
  auto enqueue = [&](cudaStream_t s, unsigned char* stage) -> int {
    ar.used = ar_used0;
    ar.fail = false;
    if (copy_coord) DP_CUDA_TRY(cudaMemcpyAsync(b.coord, coord, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, s));
    if (copy_type) DP_CUDA_TRY(cudaMemcpyAsync(b.type, type, sizeof(int) * N, cudaMemcpyHostToDevice, s));
    if (g_a_host) DP_CUDA_TRY(cudaMemcpyAsync(d_ga, gr->g_energy, sizeof(double) * F, cudaMemcpyHostToDevice, s));
    if (g_w_host) DP_CUDA_TRY(cudaMemcpyAsync(d_gw, gr->g_force, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, s));
    if (g_v_host) DP_CUDA_TRY(cudaMemcpyAsync(d_gv, gr->g_virial, sizeof(double) * 9 * F, cudaMemcpyHostToDevice, s));
    T.pack(stage);
    DP_CUDA_TRY(cudaMemcpyAsync(b.ftab, stage, T.bytes, cudaMemcpyHostToDevice, s));
    const NlGeom* d_geoms = reinterpret_cast<const NlGeom*>(b.ftab + T.off_geoms);
    const int* d_celloff = reinterpret_cast<const int*>(b.ftab + T.off_celloff);
    const int* d_start = reinterpret_cast<const int*>(b.ftab + T.off_start);
    const int* d_chunk = reinterpret_cast<const int*>(b.ftab + T.off_chunk);
    const int* d_fchunk = reinterpret_cast<const int*>(b.ftab + T.off_fchunk);
    const double* d_boxes = reinterpret_cast<const double*>(b.ftab + T.off_boxes);
    DP_CUDA_TRY(cudaMemsetAsync(md->status, 0, sizeof(DevStatus), s));
    if (F > 1) {
      ProfScope _ps(&md->prof, "atom_frame", s);
      k_atom_frame<<<(N + 255) / 256, 256, 0, s>>>(d_start, F, N, b.atom_frame);
    }
    if (own_nlist) {
      // the list build's (type, cell) order is the path's type-sorted order, and its first
      // launch also forms the image translations
      NlLaunch L{N, T.ncells, T.cap, d_geoms, b.atom_frame, F > 1 ? d_celloff : nullptr, F, T.max_noff(),
                 T.max_stream()};
      NlExtras ex{b.perm, b.type_start, chk, d_boxes, T.periodic ? F : 0, T.periodic ? b.tshift : nullptr, b.disp,
                  false};
      ProfScope _ps(&md->prof, "nlist", s, nlist_launches(L, m.cfg.ntypes));
      const NlScratch sc{b.cell_count, b.cell_start, b.atom_key, b.atom_l, b.atom_m, b.sorted_l, b.sorted_m};
      DP_CUDA_TRY(launch_nlist_build(L, m.cfg.ntypes, dcoord, dtype, sc, b.nl_j, b.nl_code, b.counts, md->status, s,
                                     &ex));
      io.disp = ex.disp_written ? b.disp : nullptr;
    } else {
      ProfScope _ps(&md->prof, "type_perm", s);
      DP_CUDA_TRY(launch_type_perm(dtype, N, m.cfg.ntypes, b.perm, b.type_start, md->status, chk, s));
    }
    if (!ts_known) {  // first call on this device type array: read the counts back (synchronises)
      int r = type_starts(nullptr, b.type_start, N, m.cfg.ntypes, s, io.type_start);
      if (r != DP_OK) return r;
      md->ts_ptr = type;
      md->ts_n = N;
      for (int t = 0; t <= m.cfg.ntypes; ++t) md->ts_v[t] = io.type_start[t];
    }
    pc.nframes = F;
    pc.periodic = T.periodic;
    pc.atom_frame = b.atom_frame;
    pc.boxes = F > 1 ? d_boxes : nullptr;
    for (int k = 0; k < 9; ++k) pc.h[k] = T.geoms[0].h[k];
    if (T.periodic) {
      pc.tshift = b.tshift;
      if (!own_nlist) {
        ProfScope _ps(&md->prof, "shift_table", s);
        k_shift_tables<<<F, 32, 0, s>>>(d_boxes, b.tshift);
      }
    }
    io.prof = &md->prof;
    io.coord = dcoord;
    io.type = dtype;
    io.perm = b.perm;
    io.nl_j = own_nlist ? b.nl_j : nlist->nl_j;
    io.nl_code = own_nlist ? b.nl_code : nlist->nl_code;
    io.force = host_f ? b.force : force;
    io.atom_energy = dev_ae ? atom_energy : b.atom_energy;
    io.atom_virial = b.atom_virial;
    io.status = md->status;
    io.epart = b.epart;
    io.atom_l = own_nlist ? b.atom_l : nullptr;
    io.atom_m = own_nlist ? b.atom_m : nullptr;
    io.geoms = own_nlist ? d_geoms : nullptr;
    if (gr) {
      {
        ProfScope _ps(&md->prof, "param_grad", s);
        int r = run_param_grad(m, pc, io, d_gw, d_ga, d_gv, -1.0, d_gout, ar, s);
        if (r != DP_OK) return r;
      }
      if (g_out_host)
        DP_CUDA_TRY(cudaMemcpyAsync(gr->grad, d_gout, sizeof(double) * m.n_params, cudaMemcpyDeviceToHost, s));
      return DP_OK;
    }
    DP_CUDA_TRY(cudaMemsetAsync(io.force, 0, sizeof(double) * 3 * N, s));
    DP_CUDA_TRY(cudaMemsetAsync(b.fcount, 0, sizeof(int) * F, s));
    if (!m.compressed) DP_CUDA_TRY(cudaMemsetAsync(io.atom_virial, 0, sizeof(double) * 9 * N, s));
    int r = run_path(m, pc, io, ar, s);
    if (r != DP_OK) return r;
    double* d_energy = host_e ? b.energy : energy;
    double* d_virial = host_v ? b.virial : virial;
    {
      ProfScope _ps(&md->prof, "frame_sums", s);
      k_chunk_sums<<<T.C, kChunk, 0, s>>>(d_chunk, io.atom_energy, io.atom_virial, b.cpart, d_fchunk, F, b.fcount,
                                          d_energy, d_virial);
    }
    DP_CUDA_TRY(cudaGetLastError());
    if (host_e) DP_CUDA_TRY(cudaMemcpyAsync(energy, d_energy, sizeof(double) * F, cudaMemcpyDeviceToHost, s));
    if (host_v) DP_CUDA_TRY(cudaMemcpyAsync(virial, d_virial, sizeof(double) * 9 * F, cudaMemcpyDeviceToHost, s));
    if (host_f) DP_CUDA_TRY(cudaMemcpyAsync(force, io.force, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, s));
    if (atom_energy && !dev_ae)
      DP_CUDA_TRY(cudaMemcpyAsync(atom_energy, io.atom_energy, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
    return DP_OK;
  };

  // After the call: a changed type count or an overflowing candidate buffer re-runs it.
  auto finish = [&](int r) -> int {
    if (r == kStatusTypeChange) {
      md->ts_ptr = nullptr;
      md->ts_n = -1;
      drop_graph(md);
      return run_frames(md, nlist, F, natoms, coord, type, boxes, energy, force, virial, atom_energy, st, gr);
    }
    if (r == DP_E_CAPACITY && own_nlist && !md->nl_full_cap) {
      md->nl_full_cap = true;  // retry once with the full candidate buffer
      drop_graph(md);
      return run_frames(md, nlist, F, natoms, coord, type, boxes, energy, force, virial, atom_energy, st, gr);
    }
    return r;
  };

  // Repeated call shapes (same sizes, buffers and cell) replay one CUDA graph of the whole call:
  // recorded on the second call of a shape, replayed from the third.  Host buffers must be
  // pinned (the graph's copies read them at replay).
  std::vector<unsigned long long> sig;
  bool graphable = !gr && ts_known && boxes;
  auto pinned_or_device = [](const void* p) {
    if (!p) return true;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged || a.type == cudaMemoryTypeHost;
  };
  if (graphable)
    graphable = pinned_or_device(coord) && pinned_or_device(type) && pinned_or_device(energy) &&
                pinned_or_device(force) && pinned_or_device(virial) && pinned_or_device(atom_energy);
  if (graphable) {
    auto put = [&](const void* p) { sig.push_back((unsigned long long)(uintptr_t)p); };
    sig.push_back((unsigned long long)F);
    for (int f = 0; f < F; ++f) sig.push_back((unsigned long long)natoms[f]);
    put(coord); put(type); put(energy); put(force); put(virial); put(atom_energy); put(nlist); put(md->ws);
    for (int k = 0; k < 9 * F; ++k) {
      unsigned long long u;
      std::memcpy(&u, boxes + k, 8);
      sig.push_back(u);
    }
    for (int t = 0; t <= m.cfg.ntypes; ++t) sig.push_back((unsigned long long)(unsigned)chk.v[t]);
    sig.push_back((unsigned long long)md->nl_full_cap | ((unsigned long long)md->prof.timing << 1));
    sig.push_back((unsigned long long)(copy_coord | (copy_type << 1) | (host_e << 2) | (host_v << 3) |
                                       (host_f << 4) | (dev_ae << 5)));
  }
  DpGraph& G = md->graph;
  if (graphable && G.exec && G.sig == sig) {  // replay
    DP_CUDA_TRY(cudaGraphLaunch(G.exec, st));
    md->prof.launches += G.launches;
    int r = read_status(md, st, nullptr);
    if (md->prof.timing) md->prof.collect_from(G.prof);
    return finish(r);
  }
  if (graphable && sig == md->last_sig) {  // second call of this shape: record it
    drop_graph(md);
    if (!md->cap_st) DP_CUDA_TRY(cudaStreamCreateWithFlags(&md->cap_st, cudaStreamNonBlocking));
    if (G.stage_cap < T.bytes) {
      if (G.stage) cudaFreeHost(G.stage);
      G.stage = nullptr;
      G.stage_cap = 0;
      DP_CUDA_TRY(cudaMallocHost(&G.stage, T.bytes + 4096));
      G.stage_cap = T.bytes + 4096;
    }
    const long l0 = md->prof.launches;
    const size_t p0 = md->prof.pending.size();
    DP_CUDA_TRY(cudaStreamBeginCapture(md->cap_st, cudaStreamCaptureModeRelaxed));
    int r = enqueue(md->cap_st, G.stage);
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(md->cap_st, &graph);
    cudaError_t ie = cudaErrorUnknown;
    if (r == DP_OK && ce == cudaSuccess && graph) ie = cudaGraphInstantiate(&G.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    // timing events recorded during capture belong to the graph now
    G.prof.assign(md->prof.pending.begin() + (long)p0, md->prof.pending.end());
    md->prof.pending.resize(p0);
    G.launches = md->prof.launches - l0;
    md->prof.launches = l0;
    if (r == DP_OK && ie == cudaSuccess) {
      G.sig = sig;
      DP_CUDA_TRY(cudaGraphLaunch(G.exec, st));
      md->prof.launches += G.launches;
      int r2 = read_status(md, st, nullptr);
      if (md->prof.timing) md->prof.collect_from(G.prof);
      return finish(r2);
    }
    drop_graph(md);  // recording failed: run the call directly (and do not try this shape again)
    md->last_sig.clear();
    rc = ensure_stage(md, T.bytes);
    if (rc != DP_OK) return rc;
    rc = enqueue(st, md->stage);
    if (rc != DP_OK) return rc;
    return finish(read_status(md, st, nullptr));
  }
  md->last_sig = sig;
  rc = enqueue(st, md->stage);
  if (rc != DP_OK) return rc;
  return finish(read_status(md, st, nullptr));
}

}  // namespace
}  // namespace dpgb

using namespace dpgb;

extern "C" {

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
  return run_frames(md, nlist, 1, &N, coord, type, box, energy, force, virial, atom_energy, (cudaStream_t)stream);
}

int dp_compute_batch(dp_model** models, int nmodels, int nframes, const int* natoms, const int* frame_model,
                     const double* coord, const int* type, const double* boxes, double* energy, double* force,
                     double* virial, double* atom_energy, void* stream) {
  if (!models || nmodels < 1 || nframes < 1 || !natoms || !coord || !type || !boxes || !energy || !force ||
      !virial || (nmodels > 1 && !frame_model)) {
    set_error("invalid argument");
    return DP_E_ARG;
  }
  for (int k = 0; k < nmodels; ++k)
    if (!models[k] || models[k]->m.device != models[0]->m.device) {
      set_error("dp_compute_batch: every model must exist and live on the same device");
      return DP_E_ARG;
    }
  for (int f = 0; f < nframes; ++f)
    if (natoms[f] < 1 || (frame_model && (frame_model[f] < 0 || frame_model[f] >= nmodels))) {
      set_error("dp_compute_batch: every frame needs at least one atom and a model index in [0, nmodels)");
      return DP_E_ARG;
    }
  // consecutive frames of the same model run as one pass of that model's kernels, all in stream
  // order; the first error ends the call, warnings (sel overflow, table range) are carried on
  int warn = DP_OK;
  long a0 = 0;
  for (int f0 = 0; f0 < nframes;) {
    const int k = frame_model ? frame_model[f0] : 0;
    int f1 = f0 + 1;
    long na = natoms[f0];
    while (f1 < nframes && (frame_model ? frame_model[f1] : 0) == k) na += natoms[f1++];
    const int rc = run_frames(models[k], nullptr, f1 - f0, natoms + f0, coord + 3 * a0, type + a0, boxes + 9L * f0,
                              energy + f0, force + 3 * a0, virial + 9L * f0, atom_energy ? atom_energy + a0 : nullptr,
                              (cudaStream_t)stream);
    if (rc != DP_OK && rc != DP_E_SEL_OVERFLOW && rc != DP_E_RANGE) return rc;
    if (rc != DP_OK && warn == DP_OK) warn = rc;
    a0 += na;
    f0 = f1;
  }
  return warn;
}

int dp_param_grad(dp_model* md, int nframes, const int* natoms, const double* coord, const int* type,
                  const double* boxes, const double* g_energy, const double* g_force, const double* g_virial,
                  double* grad, void* stream) {
  if (!md || nframes < 1 || !natoms || !coord || !type || !g_energy || !g_force || !grad) {
    set_error("invalid argument");
    return DP_E_ARG;
  }
  if (!boxes && nframes != 1) {
    set_error("batches of frames need periodic cells");
    return DP_E_UNSUPPORTED;
  }
  if (g_virial && !boxes) {
    set_error("a virial seed needs periodic cells");
    return DP_E_ARG;
  }
  if (md->m.cfg.descriptor != DP_DESC_SE_E2_A) {
    set_error("parameter gradients are implemented for se_e2_a models");
    return DP_E_UNSUPPORTED;
  }
  const GradReq gr{g_energy, g_force, g_virial, grad};
  return run_frames(md, nullptr, nframes, natoms, coord, type, boxes, nullptr, nullptr, nullptr, nullptr,
                    (cudaStream_t)stream, &gr);
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
  const DeviceModel& m = md->m;
  const bool copy_coord = !is_device_ptr(coord), copy_type = !is_device_ptr(type);
  if (copy_coord) {
    const int rc0 = check_finite_host(coord, 3L * N);
    if (rc0 != DP_OK) return rc0;
  }
  double lohi[6] = {0, 0, 0, 0, 0, 0};
  if (!box) {
    const int rc = copy_coord ? host_bbox(coord, N, lohi) : device_bbox(md, coord, N, st, lohi);
    if (rc != DP_OK) return rc;
  }
  FrameTables T;
  int rc = build_tables_host(md, 1, &N, box, lohi, T);
  if (rc != DP_OK) return rc;
  Arena pre;
  pre.measure = true;
  Bufs b;
  carve(pre, m, T, true, copy_coord, copy_type, false, false, false, false, b);
  rc = ensure_ws(md, pre.used);
  if (rc == DP_OK) rc = ensure_stage(md, T.bytes);
  if (rc != DP_OK) return rc;
  Arena ar;
  ar.base = md->ws;
  ar.cap = md->ws_cap;
  carve(ar, m, T, true, copy_coord, copy_type, false, false, false, false, b);
  const double* dcoord = copy_coord ? b.coord : coord;
  const int* dtype = copy_type ? b.type : type;
  if (copy_coord) DP_CUDA_TRY(cudaMemcpyAsync(b.coord, coord, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, st));
  if (copy_type) DP_CUDA_TRY(cudaMemcpyAsync(b.type, type, sizeof(int) * N, cudaMemcpyHostToDevice, st));
  T.pack(md->stage);
  DP_CUDA_TRY(cudaMemcpyAsync(b.ftab, md->stage, T.bytes, cudaMemcpyHostToDevice, st));
  dp_nlist* nl = new dp_nlist();
  nl->device = m.device;
  nl->natoms = N;
  nl->nc = m.nc;
  nl->ntypes = m.cfg.ntypes;
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
    NlLaunch L{N, T.ncells, T.cap, reinterpret_cast<const NlGeom*>(b.ftab + T.off_geoms), nullptr, nullptr, 1,
               T.max_noff(), T.max_stream()};
    ProfScope _ps(&md->prof, "nlist", st, nlist_launches(L, m.cfg.ntypes));
    const NlScratch sc{b.cell_count, b.cell_start, b.atom_key, b.atom_l, b.atom_m, b.sorted_l, b.sorted_m};
    DP_CUDA_TRY(launch_nlist_build(L, m.cfg.ntypes, dcoord, dtype, sc, nl->nl_j, nl->nl_code, nl->counts, md->status,
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

}  // extern "C"
