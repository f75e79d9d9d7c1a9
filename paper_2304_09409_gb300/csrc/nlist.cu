// Cell-list neighbour search with a fixed per-type sel (Sec. II.A.1 per-type blocks padded
// to N_c^{a_j}; Sec. III.B.1 ordering by type, distance, index).
//
// GB300 design: atoms are binned into cells at least r_c wide (fractional coordinates in
// FP64, any rounding is harmless because binning only bounds the search).  One warp owns
// one centre atom: it walks the (2K+1)^3 virtual cells around it, tests each candidate
// first with an FP32 distance in wrapped fractional coordinates (loose cutoff), and only
// survivors pay for the exact FP64 displacement that defines membership and order.  The
// accepted entries are kept in shared memory and ranked within their type by the exact
// total order (r^2 bits, j, image code); rank < sel[t] gives the slot directly, so no
// sort pass and no global scratch beyond the cell list is needed.
#include <cstdio>

#include "dp_internal.cuh"

namespace dpgb {

namespace {

constexpr int kWarpsPerBlock = 4;
constexpr int kQueue = 64;  // prefilter survivors waiting for the exact test (per warp)

__device__ __forceinline__ int floordiv(int a, int b) { return (a >= 0) ? a / b : -((-a + b - 1) / b); }

__global__ void k_bbox(const double* __restrict__ coord, int n, double* __restrict__ out) {
  __shared__ double s[6][32];
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    for (int a = 0; a < 3; ++a) {
      double v = coord[3 * i + a];
      lo[a] = fmin(lo[a], v);
      hi[a] = fmax(hi[a], v);
    }
  for (int off = 16; off > 0; off >>= 1)
    for (int a = 0; a < 3; ++a) {
      lo[a] = fmin(lo[a], __shfl_down_sync(0xffffffffu, lo[a], off));
      hi[a] = fmax(hi[a], __shfl_down_sync(0xffffffffu, hi[a], off));
    }
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
    for (int a = 0; a < 3; ++a) { s[a][w] = lo[a]; s[3 + a][w] = hi[a]; }
  __syncthreads();
  if (threadIdx.x == 0) {
    int nw = blockDim.x >> 5;
    for (int a = 0; a < 3; ++a) {
      double L = s[a][0], H = s[3 + a][0];
      for (int k = 1; k < nw; ++k) { L = fmin(L, s[a][k]); H = fmax(H, s[3 + a][k]); }
      out[a] = L;
      out[3 + a] = H;
    }
  }
}

__global__ void k_bin(const NlGeom* __restrict__ G, const int* __restrict__ atom_frame,
                      const int* __restrict__ cell_off, int natoms, const double* __restrict__ coord,
                      int* __restrict__ cell_count, int* __restrict__ atom_cell, int* __restrict__ atom_img,
                      float4* __restrict__ atom_wf) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= natoms) return;
  const int fr = atom_frame ? atom_frame[i] : 0;
  const NlGeom& g = G[fr];
  double x[3] = {coord[3 * i], coord[3 * i + 1], coord[3 * i + 2]};
  int c[3], m[3];
  float w[3];
  for (int d = 0; d < 3; ++d) {
    double f;
    if (g.periodic)
      f = x[0] * g.inv[0 * 3 + d] + x[1] * g.inv[1 * 3 + d] + x[2] * g.inv[2 * 3 + d];
    else
      f = (x[d] - g.origin[d]) / g.ext[d];
    double fl = g.periodic ? floor(f) : 0.0;
    double wd = f - fl;
    if (g.periodic && wd >= 1.0) { wd = 0.0; fl += 1.0; }
    if (wd < 0.0) wd = 0.0;
    m[d] = (int)fl;
    int cd = (int)(wd * g.ncell[d]);
    c[d] = cd < 0 ? 0 : (cd >= g.ncell[d] ? g.ncell[d] - 1 : cd);
    w[d] = (float)wd;
  }
  int flat = (cell_off ? cell_off[fr] : 0) + (c[0] * g.ncell[1] + c[1]) * g.ncell[2] + c[2];
  atom_cell[i] = flat;
  atom_img[3 * i] = m[0];
  atom_img[3 * i + 1] = m[1];
  atom_img[3 * i + 2] = m[2];
  atom_wf[i] = make_float4(w[0], w[1], w[2], 0.f);
  atomicAdd(cell_count + flat, 1);
}

// Exclusive scan of n ints by one block (n is the number of cells: small).
__global__ void k_scan_excl(const int* __restrict__ in, int n, int* __restrict__ out, int* __restrict__ out2) {
  __shared__ int wsum[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += blockDim.x) {
    int idx = base + threadIdx.x;
    int v = idx < n ? in[idx] : 0;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
    for (int off = 1; off < 32; off <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
      int s = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
      for (int off = 1; off < 32; off <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, s, off);
        if (lane >= off) s += t;
      }
      wsum[lane] = s;  // inclusive over warps
    }
    __syncthreads();
    int before = (w > 0 ? wsum[w - 1] : 0) + carry;
    if (idx < n) {
      out[idx] = before + incl - v;
      if (out2) out2[idx] = before + incl - v;
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = before + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = carry;
}

__global__ void k_fill(int natoms, const int* __restrict__ atom_cell, int* __restrict__ cursor,
                       int* __restrict__ cell_atoms) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= natoms) return;
  int pos = atomicAdd(cursor + atom_cell[i], 1);
  cell_atoms[pos] = i;
}

struct KeyLess {
  __device__ static bool less(unsigned long long ra, int ja, int ca, unsigned long long rb, int jb, int cb) {
    if (ra != rb) return ra < rb;
    if (ja != jb) return ja < jb;
    return (unsigned)ca < (unsigned)cb;
  }
};

template <int CAP>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_nlist(const NlGeom* __restrict__ G, const int* __restrict__ atom_frame, const int* __restrict__ cell_off,
            int natoms, const double* __restrict__ coord, const int* __restrict__ type,
            const int* __restrict__ cell_start, const int* __restrict__ cell_atoms, const int* __restrict__ atom_cell,
            const int* __restrict__ atom_img, const float4* __restrict__ atom_wf, int* __restrict__ nl_j,
            int* __restrict__ nl_code, int* __restrict__ counts, DevStatus* __restrict__ st) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned long long* k_r2 = reinterpret_cast<unsigned long long*>(smem) + (size_t)warp * CAP;
  int* k_j = reinterpret_cast<int*>(smem + (size_t)kWarpsPerBlock * CAP * 8) + (size_t)warp * CAP;
  int* k_code = reinterpret_cast<int*>(smem + (size_t)kWarpsPerBlock * CAP * 12) + (size_t)warp * CAP;
  unsigned char* k_t = smem + (size_t)kWarpsPerBlock * CAP * 16 + (size_t)warp * CAP;

  const int w = blockIdx.x * kWarpsPerBlock + warp;
  if (w >= natoms) return;  // warp-uniform
  // consecutive warps take atoms of the same cell, so their candidates share the L1 cache
  const int i = cell_atoms[w];
  const int fr = atom_frame ? atom_frame[i] : 0;
  const NlGeom& g = G[fr];
  const int coff = cell_off ? cell_off[fr] : 0;

  const double xi[3] = {coord[3 * i], coord[3 * i + 1], coord[3 * i + 2]};
  const int mi0 = atom_img[3 * i], mi1 = atom_img[3 * i + 1], mi2 = atom_img[3 * i + 2];
  const float4 wi = atom_wf[i];
  const int ci = atom_cell[i] - coff;
  const int c2 = ci % g.ncell[2];
  const int c1 = (ci / g.ncell[2]) % g.ncell[1];
  const int c0 = ci / (g.ncell[2] * g.ncell[1]);
  int cnt = 0;
  bool bad_shift = false;
  // survivors of the FP32 prefilter wait in a per-warp queue, so the exact FP64 test always
  // runs on full warps (GB300's FP64 pipe is narrow)
  int* q_j = reinterpret_cast<int*>(smem + (size_t)kWarpsPerBlock * CAP * 17) + (size_t)warp * 2 * kQueue;
  int* q_c = q_j + kQueue;
  int qn = 0;
  auto drain = [&](int take) {
    bool acc = false;
    unsigned long long r2bits = 0ull;
    int j = -1, code = 0;
    if (lane < take) {
      j = q_j[lane];
      code = q_c[lane];
      int n0, n1, n2;
      unpack_shift(code, n0, n1, n2);
      const double* xj = coord + 3 * j;
      double dx, dy, dz;
      if ((n0 | n1 | n2) == 0) {  // same image: (x_j + 0) - x_i needs no shift term
        dx = __dsub_rn(xj[0], xi[0]);
        dy = __dsub_rn(xj[1], xi[1]);
        dz = __dsub_rn(xj[2], xi[2]);
      } else {
        pair_disp_exact(xi, xj, n0, n1, n2, g.h, g.periodic, dx, dy, dz);
      }
      const double r2 = norm2_exact(dx, dy, dz);
      if (r2 < g.rc2) {
        acc = true;
        r2bits = (unsigned long long)__double_as_longlong(r2);
      }
    }
    const unsigned mask = __ballot_sync(0xffffffffu, acc);
    if (acc) {
      const int pos = cnt + __popc(mask & ((1u << lane) - 1u));
      if (pos < CAP) {
        k_r2[pos] = r2bits;
        k_j[pos] = j;
        k_code[pos] = code;
        k_t[pos] = (unsigned char)type[j];
      }
    }
    cnt += __popc(mask);
    // move the entries beyond the first `take` to the front of the queue
    __syncwarp();
    const int rest = qn - take;
    int mj = 0, mc = 0;
    if (lane < rest) {
      mj = q_j[take + lane];
      mc = q_c[take + lane];
    }
    __syncwarp();
    if (lane < rest) {
      q_j[lane] = mj;
      q_c[lane] = mc;
    }
    __syncwarp();
    qn = rest;
  };

  for (int d0 = -g.K[0]; d0 <= g.K[0]; ++d0)
    for (int d1 = -g.K[1]; d1 <= g.K[1]; ++d1)
      for (int d2 = -g.K[2]; d2 <= g.K[2]; ++d2) {
        int v0 = c0 + d0, v1 = c1 + d1, v2 = c2 + d2;
        int W0 = 0, W1 = 0, W2 = 0;
        if (g.periodic) {
          W0 = floordiv(v0, g.ncell[0]);
          W1 = floordiv(v1, g.ncell[1]);
          W2 = floordiv(v2, g.ncell[2]);
          v0 -= W0 * g.ncell[0];
          v1 -= W1 * g.ncell[1];
          v2 -= W2 * g.ncell[2];
        } else if (v0 < 0 || v1 < 0 || v2 < 0 || v0 >= g.ncell[0] || v1 >= g.ncell[1] || v2 >= g.ncell[2]) {
          continue;
        }
        const int cell = coff + (v0 * g.ncell[1] + v1) * g.ncell[2] + v2;
        const int beg = cell_start[cell], end = cell_start[cell + 1];
        for (int base = beg; base < end; base += 32) {
          const int idx = base + lane;
          bool pass = false;
          int j = -1, code = 0;
          if (idx < end) {
            j = cell_atoms[idx];
            const float4 wj = atom_wf[j];
            // FP32 prefilter in wrapped fractional coordinates
            float f0 = (wj.x + (float)W0) - wi.x, f1 = (wj.y + (float)W1) - wi.y, f2 = (wj.z + (float)W2) - wi.z;
            float e0, e1, e2;
            if (g.periodic) {
              e0 = f0 * g.hf[0] + f1 * g.hf[3] + f2 * g.hf[6];
              e1 = f0 * g.hf[1] + f1 * g.hf[4] + f2 * g.hf[7];
              e2 = f0 * g.hf[2] + f1 * g.hf[5] + f2 * g.hf[8];
            } else {
              e0 = f0 * g.hf[0];
              e1 = f1 * g.hf[4];
              e2 = f2 * g.hf[8];
            }
            if (e0 * e0 + e1 * e1 + e2 * e2 < g.rc2_loose) {
              int n0 = 0, n1 = 0, n2 = 0;
              if (g.periodic) {
                n0 = W0 - atom_img[3 * j] + mi0;
                n1 = W1 - atom_img[3 * j + 1] + mi1;
                n2 = W2 - atom_img[3 * j + 2] + mi2;
              }
              if (n0 <= -512 || n0 >= 512 || n1 <= -512 || n1 >= 512 || n2 <= -512 || n2 >= 512) {
                bad_shift = true;
              } else if (!(j == i && n0 == 0 && n1 == 0 && n2 == 0)) {
                pass = true;
                code = pack_shift(n0, n1, n2);
              }
            }
          }
          const unsigned mask = __ballot_sync(0xffffffffu, pass);
          if (pass) {
            const int pos = qn + __popc(mask & ((1u << lane) - 1u));
            q_j[pos] = j;
            q_c[pos] = code;
          }
          qn += __popc(mask);
          __syncwarp();
          if (qn >= 32) drain(32);
        }
      }
  if (qn > 0) drain(qn);
  if (__any_sync(0xffffffffu, bad_shift) && lane == 0) atomicExch(&st->capacity, 2);
  if (cnt > CAP) {
    if (lane == 0) atomicExch(&st->capacity, 1);
    cnt = CAP;
  }
  __syncwarp();
  // rank of each entry among entries of the same type under the exact total order
  for (int e = lane; e < cnt; e += 32) {
    const unsigned long long re = k_r2[e];
    const int je = k_j[e], ce = k_code[e];
    const int te = k_t[e];
    int rank = 0;
    for (int f = 0; f < cnt; ++f)
      if (k_t[f] == te && KeyLess::less(k_r2[f], k_j[f], k_code[f], re, je, ce)) ++rank;
    if (rank < g.sel[te]) {
      const long slot = (long)i * g.nc + g.sel_off[te] + rank;
      nl_j[slot] = je;
      nl_code[slot] = ce;
    }
  }
  // per-type counts, padding and overflow accounting
  for (int t = 0; t < g.ntypes; ++t) {
    int c = 0;
    for (int e = lane; e < cnt; e += 32) c += (k_t[e] == t);
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    for (int q = c + lane; q < g.sel[t]; q += 32) {
      const long slot = (long)i * g.nc + g.sel_off[t] + q;
      nl_j[slot] = -1;
      nl_code[slot] = pack_shift(0, 0, 0);
    }
    if (lane == 0) {
      if (counts) counts[(long)i * g.ntypes + t] = c;
      if (c > g.sel[t]) atomicAdd(&st->sel_overflow, 1);
    }
  }
}

// Stable partition of atoms by type (one block, one pass): each thread takes a contiguous
// chunk of atoms, counts per type, and a block-wide exclusive scan of the counts gives every
// thread its output offset per type.  perm[p] = atom index, type_start[t].
__global__ void __launch_bounds__(1024)
    k_type_perm(const int* __restrict__ type, int n, int ntypes, int* __restrict__ perm, int* __restrict__ type_start,
                int* __restrict__ bad_type) {
  __shared__ int wtot[32][DP_MAX_TYPES];
  __shared__ int tstart[DP_MAX_TYPES + 1];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int lo = tid * per, hi = min(n, lo + per);
  int cnt[DP_MAX_TYPES], incl[DP_MAX_TYPES];
#pragma unroll
  for (int t = 0; t < DP_MAX_TYPES; ++t) cnt[t] = 0;
  bool bad = false;
  for (int i = lo; i < hi; ++i) {
    const int t = type[i];
    if (t < 0 || t >= ntypes) bad = true;
#pragma unroll
    for (int q = 0; q < DP_MAX_TYPES; ++q) cnt[q] += (t == q);
  }
#pragma unroll
  for (int t = 0; t < DP_MAX_TYPES; ++t) {
    int v = cnt[t];
    for (int off = 1; off < 32; off <<= 1) {
      const int x = __shfl_up_sync(0xffffffffu, v, off);
      if (lane >= off) v += x;
    }
    incl[t] = v;
    if (lane == 31) wtot[w][t] = v;
  }
  __syncthreads();
  if (tid < ntypes) {  // exclusive offsets of the warps, per type
    int acc = 0;
    for (int k = 0; k < nw; ++k) {
      const int x = wtot[k][tid];
      wtot[k][tid] = acc;
      acc += x;
    }
    tstart[tid + 1] = acc;  // total of type tid for now
  }
  __syncthreads();
  if (tid == 0) {
    tstart[0] = 0;
    for (int t = 0; t < ntypes; ++t) tstart[t + 1] += tstart[t];
  }
  __syncthreads();
  int off[DP_MAX_TYPES];
#pragma unroll
  for (int t = 0; t < DP_MAX_TYPES; ++t) off[t] = (t < ntypes) ? tstart[t] + wtot[w][t] + incl[t] - cnt[t] : 0;
  for (int i = lo; i < hi; ++i) {
    const int t = type[i];
#pragma unroll
    for (int q = 0; q < DP_MAX_TYPES; ++q)
      if (t == q && q < ntypes) perm[off[q]++] = i;
  }
  if (bad) atomicExch(bad_type, 1);
  if (tid <= ntypes) type_start[tid] = tstart[tid];
}

}  // namespace

int host_geometry(const dp_model_config& cfg, int natoms, const double* box, const double* lohi, NlGeom& g) {
  std::memset(&g, 0, sizeof(g));
  g.natoms = natoms;
  g.ntypes = cfg.ntypes;
  int off = 0;
  for (int t = 0; t < cfg.ntypes; ++t) {
    g.sel[t] = cfg.sel[t];
    g.sel_off[t] = off;
    off += cfg.sel[t];
  }
  g.sel_off[cfg.ntypes] = off;
  g.nc = off;
  const double rc = cfg.rcut;
  g.rc2 = rc * rc;
  g.rc2_loose = (float)((rc + 1e-3) * (rc + 1e-3));
  const double cellmin = rc * (1.0 + 1e-9) + 1e-9;
  if (box) {
    g.periodic = 1;
    const double* h = box;
    for (int k = 0; k < 9; ++k) { g.h[k] = h[k]; g.hf[k] = (float)h[k]; }
    double c00 = h[4] * h[8] - h[5] * h[7], c01 = h[5] * h[6] - h[3] * h[8], c02 = h[3] * h[7] - h[4] * h[6];
    double det = h[0] * c00 + h[1] * c01 + h[2] * c02;
    if (!(std::fabs(det) > 1e-12)) {
      set_error("box is singular");
      return DP_E_ARG;
    }
    g.inv[0] = c00 / det; g.inv[1] = (h[2] * h[7] - h[1] * h[8]) / det; g.inv[2] = (h[1] * h[5] - h[2] * h[4]) / det;
    g.inv[3] = c01 / det; g.inv[4] = (h[0] * h[8] - h[2] * h[6]) / det; g.inv[5] = (h[2] * h[3] - h[0] * h[5]) / det;
    g.inv[6] = c02 / det; g.inv[7] = (h[1] * h[6] - h[0] * h[7]) / det; g.inv[8] = (h[0] * h[4] - h[1] * h[3]) / det;
    const double vol = std::fabs(det);
    long total = 1;
    for (int d = 0; d < 3; ++d) {
      const double* u = h + 3 * ((d + 1) % 3);
      const double* v = h + 3 * ((d + 2) % 3);
      double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
      double width = vol / std::sqrt(cx * cx + cy * cy + cz * cz);
      int n = (int)std::floor(width / cellmin);
      if (n < 1) n = 1;
      if (n > 256) n = 256;
      g.ncell[d] = n;
      g.K[d] = (int)std::ceil(cellmin * n / width);
      if (g.K[d] < 1) g.K[d] = 1;
      if (g.K[d] > 64) {
        set_error("cell narrower than r_c/64: too many periodic images");
        return DP_E_ARG;
      }
      total *= n;
    }
    (void)total;
    // candidate buffer: twice the mean neighbour count of this density, plus a margin
    const double expect = natoms / vol * (4.0 / 3.0) * 3.141592653589793 * rc * rc * rc;
    g.cap = (int)(2.0 * expect + 32.0);
  } else {
    g.periodic = 0;
    for (int d = 0; d < 3; ++d) {
      double lo = lohi[d], hi = lohi[3 + d];
      g.origin[d] = lo - 0.5;
      g.ext[d] = (hi - lo) + 1.0;
      int n = (int)std::floor(g.ext[d] / cellmin);
      if (n < 1) n = 1;
      if (n > 256) n = 256;
      g.ncell[d] = n;
      g.K[d] = 1;
    }
    g.cap = DP_MAX_CANDIDATES;  // clusters: no meaningful density
    g.hf[0] = (float)g.ext[0];
    g.hf[4] = (float)g.ext[1];
    g.hf[8] = (float)g.ext[2];
  }
  return DP_OK;
}

cudaError_t launch_bbox(const double* coord, int natoms, double* out_lohi, cudaStream_t st) {
  k_bbox<<<1, 1024, 0, st>>>(coord, natoms, out_lohi);
  return cudaGetLastError();
}

cudaError_t launch_nlist_build(const NlLaunch& L, const double* coord, const int* type, int* cell_count,
                               int* cell_start, int* cell_cursor, int* cell_atoms, int* atom_cell, int* atom_img,
                               float4* atom_wf, int* nl_j, int* nl_code, int* counts, DevStatus* status,
                               cudaStream_t st) {
  const int ncells = L.ncells_total;
  cudaError_t e = cudaMemsetAsync(cell_count, 0, sizeof(int) * ncells, st);
  if (e != cudaSuccess) return e;
  const int nb = (L.natoms + 255) / 256;
  k_bin<<<nb, 256, 0, st>>>(L.geoms, L.atom_frame, L.cell_off, L.natoms, coord, cell_count, atom_cell, atom_img,
                            atom_wf);
  k_scan_excl<<<1, 1024, 0, st>>>(cell_count, ncells, cell_start, cell_cursor);
  k_fill<<<nb, 256, 0, st>>>(L.natoms, atom_cell, cell_cursor, cell_atoms);
  const int cap = L.cap <= 128 ? 128 : (L.cap <= 256 ? 256 : (L.cap <= 512 ? 512 : 1024));
  const size_t smem = (size_t)kWarpsPerBlock * cap * 17 + (size_t)kWarpsPerBlock * 2 * kQueue * sizeof(int);
  const unsigned blocks = (L.natoms + kWarpsPerBlock - 1) / kWarpsPerBlock;
#define DPGB_NL_LAUNCH(C)                                                                                   \
  do {                                                                                                      \
    e = cudaFuncSetAttribute(k_nlist<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);           \
    if (e != cudaSuccess) return e;                                                                         \
    k_nlist<C><<<blocks, kWarpsPerBlock * 32, smem, st>>>(L.geoms, L.atom_frame, L.cell_off, L.natoms, coord, \
                                                         type, cell_start, cell_atoms, atom_cell, atom_img,   \
                                                         atom_wf, nl_j, nl_code, counts, status);             \
  } while (0)
  if (cap == 128)
    DPGB_NL_LAUNCH(128);
  else if (cap == 256)
    DPGB_NL_LAUNCH(256);
  else if (cap == 512)
    DPGB_NL_LAUNCH(512);
  else
    DPGB_NL_LAUNCH(1024);
#undef DPGB_NL_LAUNCH
  return cudaGetLastError();
}

cudaError_t launch_type_perm(const int* type, int natoms, int ntypes, int* perm, int* type_start, int* bad_type,
                             cudaStream_t st) {
  k_type_perm<<<1, 1024, 0, st>>>(type, natoms, ntypes, perm, type_start, bad_type);
  return cudaGetLastError();
}

}  // namespace dpgb
