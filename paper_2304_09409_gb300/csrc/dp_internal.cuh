// Internal declarations shared by the CUDA translation units of libdpgb.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dpgb.h"

namespace dpgb {

// ------------------------------------------------------------------------------------------
// Geometry of one neighbour-list build (host-computed launch configuration)
// ------------------------------------------------------------------------------------------
struct NlGeom {
  int natoms, ntypes, nc;
  int sel[DP_MAX_TYPES];
  int sel_off[DP_MAX_TYPES + 1];
  int periodic;
  double h[9];       // cell rows h0, h1, h2 (periodic)
  double inv[9];     // inverse of h (periodic)
  double origin[3];  // open boundary: fractional = (x - origin) / ext
  double ext[3];
  double rext[3];    // open boundary: 1 / ext
  double rn[3];      // 1 / ncell
  float hc[9];       // edge vectors of one cell, h_e / ncell_e (diag(ext / ncell) when open), FP32
  float r_n2c, r_n12c;  // 1 / (2K_2 + 1), 1 / ((2K_1 + 1)(2K_2 + 1)): decoding a surrounding-cell index
  int ncell[3];
  int K[3];          // virtual-cell search half-width per axis
  double rc2;        // r_c^2 (exact membership test)
  // FP32 screening of the cell-local distance (error below eps in r^2, bounded on the host):
  float rc2_in;      // r2_32 < rc2_in: certainly inside (rc2_in <= rc2 - eps)
  float rc2_out;     // r2_32 > rc2_out: certainly outside (rc2_out >= rc2 + eps)
  float tie_w;       // FP32 keys further apart than tie_w are ordered as their FP64 values
  int cap;           // candidate buffer per centre atom (rounded up to 128..DP_MAX_CANDIDATES)
};

// Image shift (n0, n1, n2) packed as 10-bit offsets; |n| < 512.
__host__ __device__ inline int pack_shift(int n0, int n1, int n2) {
  return ((n0 + 512) << 20) | ((n1 + 512) << 10) | (n2 + 512);
}
__host__ __device__ inline void unpack_shift(int code, int& n0, int& n1, int& n2) {
  n0 = ((code >> 20) & 1023) - 512;
  n1 = ((code >> 10) & 1023) - 512;
  n2 = (code & 1023) - 512;
}

// Pair displacement (x_j + t) - x_i with t = n0 h0 + n1 h1 + n2 h2, evaluated left to right
// with explicitly rounded FP64 operations (never contracted into FMA), so every kernel that
// needs r_ij reproduces the neighbour builder's value bit for bit.
__device__ __forceinline__ void pair_disp_exact(const double* __restrict__ xi, const double* __restrict__ xj,
                                                int n0, int n1, int n2, const double* h, int periodic,
                                                double& d0, double& d1, double& d2) {
  double d[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double t = 0.0;
    if (periodic)
      t = __dadd_rn(__dadd_rn(__dmul_rn((double)n0, h[0 * 3 + a]), __dmul_rn((double)n1, h[1 * 3 + a])),
                    __dmul_rn((double)n2, h[2 * 3 + a]));
    d[a] = __dsub_rn(__dadd_rn(xj[a], t), xi[a]);
  }
  d0 = d[0];
  d1 = d[1];
  d2 = d[2];
}
__device__ __forceinline__ double norm2_exact(double d0, double d1, double d2) {
  return __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
}

// ------------------------------------------------------------------------------------------
// Model as held on the device
// ------------------------------------------------------------------------------------------
struct LayerDesc {
  int n_in, n_out;
  long w_off;  // offset of W [n_in][n_out] in the parameter arrays; b follows W
  int skip;    // 0 none, 1 +x, 2 +{x,x}
  int tanh_act;
};

// One descriptor part (Sec. II.A.1): its own cutoffs, sel and embedding nets, writing the
// block [doff, doff + width) of D.  A model has one part, or two for a hybrid.
enum PartKind { PART_A = 0, PART_R = 1, PART_E3 = 2 };
struct PartDesc {
  int kind;
  double rc, rs;
  int sel[DP_MAX_TYPES];
  int sel_off[DP_MAX_TYPES + 1];
  int nc;
  int M, A;      // output width of its nets; M_< (se_e2_a parts)
  int doff;      // first column of its block of D
  int nl;        // embedding layers
  int n_nets;    // N_t^2, or N_t (two-body nets with type_one_side)
  long w_off;    // offset of its first net's parameters
  long per_net;  // parameters of one net
  std::vector<LayerDesc> emb;  // per net * nl + layer
};

struct TableDesc {
  double s0, stride1, stride2;
  int n1, n2;
};

struct DeviceModel {
  dp_model_config cfg;
  int device;
  int precision;
  int compressed;
  int nc, M, A, n_embed_nets;
  int Dw;  // width of D (the fitting net's input)
  // neighbour-list geometry (nc, sel_off, lcfg.rcut, lcfg.sel): for a hybrid, the larger cutoff
  // and per type the larger sel of its parts; for one part, the part's own
  int sel_off[DP_MAX_TYPES + 1];
  dp_model_config lcfg;
  std::vector<PartDesc> parts;
  std::vector<LayerDesc> emb;  // first part's nets, per net * n_embed + layer
  std::vector<LayerDesc> fit;  // per type * n_fit_layers + layer
  int n_fit_layers;
  long n_params;
  double* p64 = nullptr;  // device FP64 parameters
  float* p32 = nullptr;   // device FP32 copy
  TableDesc tab{};
  double* tab64 = nullptr;  // [nets][lc][M][6]
  float* tab32 = nullptr;
  // BF16 operands of the tensor-core fitting net: per (type, hidden layer) W^T [n_out][n_in]
  // (forward) and W [n_in][n_out] (backward), at fit_bf16_off[type * n_fit + layer].
  void* fit_wt_bf16 = nullptr;
  void* fit_w_bf16 = nullptr;
  // low halves W - bf16(W) of the same operands (split three-pass products of the FP32 mode)
  void* fit_wt_bf16_lo = nullptr;
  void* fit_w_bf16_lo = nullptr;
  float fit_out_bias[DP_MAX_TYPES] = {};  // bias of the final linear layer, per type
  std::vector<long> fit_bf16_off;
  // tensor maps of those operands, keyed by (type, layer, direction, box rows)
  mutable std::vector<std::pair<long, std::vector<unsigned char>>> tmap_cache;
  // uncompressed tensor-core path (emb_tc.cu): per layer, forward W^T [n_out][pad16(n_in)] and
  // backward W [n_in][pad16(n_out)] operands in BF16 or FP32 (TF32 mode); embedding layers l >= 1
  // of every net, then the hidden fitting layers of every type, at tc_off
  void* tc_wt = nullptr;
  void* tc_w = nullptr;
  std::vector<long> tc_off;
  // interval-moment operands of the compressed embedding on the tensor cores (mom.cu)
  int mom_npass = 0;  // 0 none; 1 FP16 single pass; 3 BF16 high/low, three passes
  int mom_npad = 0, mom_lcp = 0;
  void* mom_tab = nullptr;               // forward and backward coefficient tables
  std::vector<unsigned char> mom_maps;   // four CUtensorMaps: forward hi/lo, backward hi/lo
};

// ------------------------------------------------------------------------------------------
// Error state and helpers (capi.cu)
// ------------------------------------------------------------------------------------------
void set_error(const std::string& msg);
// The configuration the neighbour list is built with: the larger cutoff and, per type, the larger
// sel of a hybrid's parts (a one-part configuration unchanged).
dp_model_config list_config(const dp_model_config& c);
#define DP_CUDA_TRY(expr)                                                                   \
  do {                                                                                      \
    cudaError_t _e = (expr);                                                                \
    if (_e != cudaSuccess) {                                                                \
      dpgb::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));                  \
      return _e == cudaErrorMemoryAllocation ? DP_E_OOM : DP_E_CUDA;                        \
    }                                                                                       \
  } while (0)

// Device status words written by kernels.
struct DevStatus {
  int sel_overflow;   // number of (atom, type) blocks beyond sel
  int capacity;       // an atom had more than DP_MAX_CANDIDATES candidates
  int table_range;    // compressed: an s outside the table
  int bad_type;       // a type outside [0, ntypes)
  int timeout;        // a bounded wait of a tensor-core kernel gave up
  int type_change;    // the per-type atom counts differ from the ones the call was set up with
  int bad_coord;      // a coordinate was NaN or infinite (the atom was binned as if at the origin)
  unsigned int mma_blocks[2];  // tensor-core blocks the moment kernels issued (forward, backward)
};

// Per-type starts of the type-sorted atom order that a call was set up with (checked on the
// device against the counts of the types actually given).
struct TypeStartCheck {
  int on;
  int v[DP_MAX_TYPES + 1];
};

// Let `kernel` take up to the device's opt-in shared memory per block.  Every caller sets the
// same value, so launches from several host threads never see the limit lowered under them
// (the shared memory a block actually gets is the launch's own request).
// Streaming multiprocessors of the current device (read once per device).
inline int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (cached[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    cached[dev] = n;
  }
  return cached[dev];
}

template <class K>
inline cudaError_t allow_max_smem(K kernel) {
  int dev = 0, mx = 0;
  cudaFuncAttributes fa;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
  if (e == cudaSuccess)  // the opt-in limit covers static and dynamic shared memory together
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - (int)fa.sharedSizeBytes);
  return e;
}

// ------------------------------------------------------------------------------------------
// Launchers (nlist.cu)
// ------------------------------------------------------------------------------------------
int host_geometry(const dp_model_config& cfg, int natoms, const double* box_host, const double* bbox_lohi,
                  NlGeom& g);
cudaError_t launch_bbox(const double* coord, int natoms, double* out_lohi /*device [6]*/, cudaStream_t st);
// One neighbour-list build over one or more frames of the same model.
struct NlLaunch {
  int natoms;             // atoms of all frames
  int ncells_total;       // cells of all frames
  int cap;                // candidate buffer per atom (max over frames)
  const NlGeom* geoms;    // device [frames]
  const int* atom_frame;  // device [natoms] frame of each atom, or null (one frame)
  const int* cell_off;    // device [frames + 1] first cell of each frame, or null (one frame)
  int nframes;            // frames in the launch
  int max_noff;           // largest (2K_0+1)(2K_1+1)(2K_2+1) over the frames
  int max_stream;         // largest mean candidate stream of one cell over the frames (0: unknown)
};
// What a path call also takes from the list build: the (type, cell) order of the atoms as its
// type-sorted order (perm [natoms], type_start [ntypes + 1], checked against chk) and the 27
// image translations of every frame (tshift [nframes][27][3] from boxes [nframes][9]).
struct NlExtras {
  int* perm;
  int* type_start;
  TypeStartCheck chk;
  const double* boxes;
  int nframes;
  double* tshift;
  // optional [natoms][nc] in sorted order: each listed pair's FP32 displacement (l_j + o) - l_i
  // and, in w, 1 when its FP32 r^2 is certainly inside r_c, 0 when only the exact FP64 test
  // decided, -1 for padding; written only by the cell-centred search (disp_written says so)
  float4* disp;
  bool disp_written;
};
// Cell arrays are indexed by (type, cell): cell_count [ntypes * ncells_total], cell_start
// [ntypes * ncells_total + 1]; per atom its key and rank within the key (atom_key, int2), its
// entry in input order (atom_l, atom_m) and in sorted order (sorted_l, sorted_m) [natoms].
struct NlScratch {
  int* cell_count;
  int* cell_start;
  int2* atom_key;
  float4* atom_l;
  int4* atom_m;
  float4* sorted_l;
  int4* sorted_m;
};
// Kernel launches one launch_nlist_build makes (the key scan is folded into the fill for few keys).
int nlist_launches(const NlLaunch& L, int ntypes);
cudaError_t launch_nlist_build(const NlLaunch& L, int ntypes, const double* coord, const int* type,
                               const NlScratch& sc, int* nl_j, int* nl_code, int* counts, DevStatus* status,
                               cudaStream_t st, NlExtras* ex = nullptr);
cudaError_t launch_type_perm(const int* type, int natoms, int ntypes, int* perm, int* type_start, DevStatus* status,
                             const TypeStartCheck& chk,
                             cudaStream_t st);

// ------------------------------------------------------------------------------------------
// Generic (CUDA-core) path, templated on the network scalar (dense.cu / path.cu)
// ------------------------------------------------------------------------------------------
struct RowMap {
  int kind;  // 0: rows r0 + r ; 1: slots (p0 + r / nk) * nc + k0 + r % nk
  long r0;
  int p0, nk, k0, nc;
  int nrows;
  // slot rows: the environment rows ([rows][4], the layer's element type) -- a row whose s is zero
  // (padding) is left unwritten, and a tile of such rows only is skipped; null: every row
  const void* zrow = nullptr;
};

template <class R>
cudaError_t launch_dense_fwd(const RowMap& rm, const R* X, int n_in, const R* W, const R* b, int n_out, int skip,
                             int tanh_act, R* Y, R* Tact, cudaStream_t st);
template <class R>
cudaError_t launch_dense_bwd(const RowMap& rm, const R* GY, const R* Tact, int n_in, const R* W, int n_out,
                             int skip, R* GX, cudaStream_t st);

}  // namespace dpgb
