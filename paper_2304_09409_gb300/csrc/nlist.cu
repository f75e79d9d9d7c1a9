// Cell-list neighbour search with a fixed per-type sel (Sec. II.A.1 per-type blocks padded
// to N_c^{a_j}; Sec. III.B.1 ordering by type, distance, index).
//
// GB300 design.  Atoms are binned into cells at least r_c wide and sorted by (type, cell), so
// that the atoms of one type in one cell are contiguous.  Each sorted entry carries the
// atom's position relative to the corner of its cell in FP32 (cell-local coordinates, small
// numbers, so FP32 keeps them to ~1e-6 A) and its index.  One warp owns one centre atom and,
// for each neighbour type, streams the concatenated candidates of the (2K+1)^3 surrounding
// cells in full 32-lane batches.  The displacement is l_j - l_i + (cell offset) in FP32, with
// an error bound on r^2 computed on the host from the cell geometry; candidates that the bound
// cannot place on one side of r_c (a vanishing fraction) take the exact FP64 test that defines
// membership.  The accepted entries of each type are ranked under the exact total order
// (r^2, j, image code): FP32 keys further apart than twice the bound decide directly, and only
// pairs inside that window compare their exact FP64 r^2.  rank < sel[t] gives the slot, so no
// sort pass and no global scratch beyond the cell arrays is needed.
#include <algorithm>
#include <cstdio>

#include "dp_internal.cuh"

namespace dpgb {

namespace {

constexpr int kNlWarps = 4;  // centre atoms (warps) per block
constexpr int kNlEntryBytes = 12;  // shared bytes per accepted entry

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

// Cell of an atom, its periodic image index m (x = wrapped + m h) and its position relative to
// the corner of its cell, all from FP64 fractional coordinates.
struct Binned {
  int c[3], m[3];
  double l[3];
};
__device__ __forceinline__ Binned bin_atom(const NlGeom& g, const double* x) {
  Binned b;
  double s[3];
  for (int d = 0; d < 3; ++d) {
    double f;
    if (g.periodic)
      f = x[0] * g.inv[0 * 3 + d] + x[1] * g.inv[1 * 3 + d] + x[2] * g.inv[2 * 3 + d];
    else
      f = (x[d] - g.origin[d]) * g.rext[d];
    double fl = g.periodic ? floor(f) : 0.0;
    double wd = f - fl;
    if (g.periodic && wd >= 1.0) { wd = 0.0; fl += 1.0; }
    if (wd < 0.0) wd = 0.0;
    b.m[d] = (int)fl;
    int cd = (int)(wd * g.ncell[d]);
    b.c[d] = cd < 0 ? 0 : (cd >= g.ncell[d] ? g.ncell[d] - 1 : cd);
    s[d] = (double)b.m[d] + (double)b.c[d] * g.rn[d];
  }
  for (int d = 0; d < 3; ++d) {
    if (g.periodic)
      b.l[d] = x[d] - (s[0] * g.h[0 * 3 + d] + s[1] * g.h[1 * 3 + d] + s[2] * g.h[2 * 3 + d]);
    else
      b.l[d] = x[d] - (g.origin[d] + s[d] * g.ext[d]);
  }
  return b;
}

// Key (type, cell) of every atom, its rank among the atoms of that key (the count so far) and
// its sorted entry (cell-local FP32 position with the atom index; image index m with the packed
// cell coordinates).  When asked, the same launch also forms the 27 image translations
// t(n) = n0 h0 + n1 h1 + n2 h2, n in {-1,0,1}^3, of every frame (rounded as the exact
// displacement rounds them).
__global__ void k_bin(const NlGeom* __restrict__ G, const int* __restrict__ atom_frame,
                      const int* __restrict__ cell_off, int natoms, int ncells_total, int ntypes,
                      const double* __restrict__ coord, const int* __restrict__ type, int* __restrict__ cell_count,
                      int2* __restrict__ atom_key, float4* __restrict__ atom_l, int4* __restrict__ atom_m,
                      DevStatus* __restrict__ st, const double* __restrict__ boxes, int nframes,
                      double* __restrict__ tshift) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (tshift)
    for (int k = i; k < 27 * nframes; k += gridDim.x * blockDim.x) {
      const int f = k / 27, q = k - 27 * f;
      const double* h = boxes + 9L * f;
      const int n0 = q / 9 - 1, n1 = (q / 3) % 3 - 1, n2 = q % 3 - 1;
      for (int a = 0; a < 3; ++a)
        tshift[81L * f + q * 3 + a] = __dadd_rn(
            __dadd_rn(__dmul_rn((double)n0, h[a]), __dmul_rn((double)n1, h[3 + a])), __dmul_rn((double)n2, h[6 + a]));
    }
  if (i >= natoms) return;
  const int fr = atom_frame ? atom_frame[i] : 0;
  const NlGeom& g = G[fr];
  double x[3] = {coord[3 * i], coord[3 * i + 1], coord[3 * i + 2]};
  if (!isfinite(x[0]) || !isfinite(x[1]) || !isfinite(x[2])) {
    // reported (the call fails with DP_E_ARG); binned as if at the origin so that every index
    // derived from the position stays inside its buffer
    atomicExch(&st->bad_coord, 1);
    x[0] = x[1] = x[2] = 0.0;
  }
  const Binned b = bin_atom(g, x);
  const int t = type[i];
  if (t < 0 || t >= ntypes) {  // reported; the atom takes part in no list
    atom_key[i] = make_int2(-1, 0);
    atomicExch(&st->bad_type, 1);
    return;
  }
  const int key = t * ncells_total + (cell_off ? cell_off[fr] : 0) + (b.c[0] * g.ncell[1] + b.c[1]) * g.ncell[2] + b.c[2];
  atom_key[i] = make_int2(key, atomicAdd(cell_count + key, 1));
  atom_l[i] = make_float4((float)b.l[0], (float)b.l[1], (float)b.l[2], __int_as_float(i));
  atom_m[i] = make_int4(b.m[0], b.m[1], b.m[2], (b.c[0] << 20) | (b.c[1] << 10) | b.c[2]);
}

// Exclusive scan of n ints by one block.
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

// Exclusive scan of the key counts into shared memory by one block (a few thousand keys: every
// block of the fill forms it itself instead of waiting for a separate scan launch).
__device__ __forceinline__ void block_scan_counts(const int* __restrict__ in, int n, int* s_out) {
  __shared__ int wsum[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  for (int base = 0; base < n; base += blockDim.x) {
    const int idx = base + threadIdx.x;
    const int v = idx < n ? in[idx] : 0;
    int incl = v;
    for (int off = 1; off < 32; off <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
      int x = lane < nw ? wsum[lane] : 0;
      for (int off = 1; off < 32; off <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += t;
      }
      wsum[lane] = x;
    }
    __syncthreads();
    const int before = (w > 0 ? wsum[w - 1] : 0) + carry;
    if (idx < n) s_out[idx] = before + incl - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = before + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) s_out[n] = carry;
  __syncthreads();
}

// Sorted entries as below, with the key starts formed in shared memory by every block (block 0
// also writes them out for the search).
__global__ void k_fill_scan(int natoms, const int* __restrict__ cell_count, int nkeys, int* __restrict__ cell_start,
                            const int2* __restrict__ atom_key, const float4* __restrict__ atom_l,
                            const int4* __restrict__ atom_m, float4* __restrict__ sorted_l, int4* __restrict__ sorted_m,
                            int* __restrict__ perm, int* __restrict__ type_start, int ncells_total, int ntypes,
                            DevStatus* __restrict__ st, const TypeStartCheck chk) {
  extern __shared__ int s_start[];  // [nkeys + 1]
  block_scan_counts(cell_count, nkeys, s_start);
  if (blockIdx.x == 0)
    for (int k = threadIdx.x; k <= nkeys; k += blockDim.x) cell_start[k] = s_start[k];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (perm && i <= ntypes) {
    const int v = s_start[i * ncells_total];
    type_start[i] = v;
    if (chk.on && v != chk.v[i]) atomicExch(&st->type_change, 1);
  }
  if (i >= natoms) return;
  const int2 kr = atom_key[i];
  if (kr.x < 0) return;
  const int pos = s_start[kr.x] + kr.y;
  if (perm) perm[pos] = i;
  sorted_l[pos] = atom_l[i];
  sorted_m[pos] = atom_m[i];
}

// Sorted entries (scattered from the per-atom ones: key start + rank).  When asked, the sorted
// order also serves as the type-sorted order of the path (perm, per-type starts), with the starts
// checked against the ones the call was set up with.
__global__ void k_fill(int natoms, const int2* __restrict__ atom_key, const float4* __restrict__ atom_l,
                       const int4* __restrict__ atom_m, float4* __restrict__ sorted_l, int4* __restrict__ sorted_m,
                       int* __restrict__ perm, int* __restrict__ type_start, const int* __restrict__ cell_start,
                       int ncells_total, int ntypes, DevStatus* __restrict__ st, const TypeStartCheck chk) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (perm && i <= ntypes) {
    const int v = cell_start[i * ncells_total];
    type_start[i] = v;
    if (chk.on && v != chk.v[i]) atomicExch(&st->type_change, 1);
  }
  if (i >= natoms) return;
  const int2 kr = atom_key[i];
  if (kr.x < 0) return;
  const int pos = cell_start[kr.x] + kr.y;
  if (perm) perm[pos] = i;
  sorted_l[pos] = atom_l[i];
  sorted_m[pos] = atom_m[i];
}

// Small integers to and from FP32 through the bit pattern (exact for |v| < 2^22): no
// conversion instructions, which issue on a narrow pipe on this part.
__device__ __forceinline__ float small_int_to_float(int v) {
  return __int_as_float(0x4B400000 + v) - 12582912.0f;
}
__device__ __forceinline__ int small_float_to_int(float f) {  // nearest integer, |f| < 2^22
  return __float_as_int(__fadd_rn(f, 12582912.0f)) - 0x4B400000;
}
// floor(o / m) for 0 <= o < 2^21 from r = fl(1/m): x = (o + 1/2)/m lies at least 1/(2m) away
// from an integer, further than the error of fma(o + 1/2, r, -1/2) (relative 2^-23 of x), so
// rounding x - 1/2 to the nearest integer gives floor(x).
__device__ __forceinline__ int div_small(int o, float r) {
  return small_float_to_int(fmaf(small_int_to_float(o) + 0.5f, r, -0.5f));
}

// One surrounding cell of the centre's cell, as staged for the batch walk.
struct NbCell {
  float o0, o1, o2;  // FP32 offset of the cell's corner from the centre cell's corner (image included)
  int beg;           // first sorted entry of the cell (this type)
  int pex;           // position of that entry in the concatenated candidate stream
  int wcode;         // periodic wrap W of the cell, packed as an image code
  int wzero;         // W == 0 (the centre's own image of its cell)
  int pad;
};

// Neighbour index j and image code n = W + m_i - m_j of a sorted entry seen through a cell of
// wrap code wcode; false when n leaves the packable range.
__device__ __forceinline__ bool entry_code(const float4* __restrict__ sorted_l, const int4* __restrict__ sorted_m,
                                           int idx, int wcode, const int4& mi, int& j, int& code) {
  j = __float_as_int(__ldg(&sorted_l[idx].w));
  const int4 mj = __ldg(sorted_m + idx);
  int w0, w1, w2;
  unpack_shift(wcode, w0, w1, w2);
  const int n0 = w0 + mi.x - mj.x, n1 = w1 + mi.y - mj.y, n2 = w2 + mi.z - mj.z;
  code = 0;
  if (n0 <= -512 || n0 >= 512 || n1 <= -512 || n1 >= 512 || n2 <= -512 || n2 >= 512) return false;
  code = pack_shift(n0, n1, n2);
  return true;
}

__device__ __forceinline__ double exact_r2(const NlGeom& g, const double* xi, const double* __restrict__ coord, int j,
                                           int code) {
  const double* xj = coord + 3 * j;
  double d0, d1, d2;
  if (code == pack_shift(0, 0, 0)) {  // same image: (x_j + 0) - x_i is x_j - x_i
    d0 = __dsub_rn(xj[0], xi[0]);
    d1 = __dsub_rn(xj[1], xi[1]);
    d2 = __dsub_rn(xj[2], xi[2]);
  } else {
    int n0, n1, n2;
    unpack_shift(code, n0, n1, n2);
    pair_disp_exact(xi, xj, n0, n1, n2, g.h, g.periodic, d0, d1, d2);
  }
  return norm2_exact(d0, d1, d2);
}

// Rank of each accepted entry of one type among the entries of that type under the exact
// total order (r^2 in FP64, then j, then the image code), and its slot in the list.  FP32 keys
// further apart than tw order their entries directly; an entry with other keys inside its
// window computes the exact r^2 of itself and of those partners (rare: O-H bonds, lattice
// shells) and compares.  The keys [gs, ge) are padded with +inf to ge4 (a multiple of 4).
// wcode_of maps the stored e_w to the wrap code of the cell the entry was seen through.
template <class WcodeOf>
__device__ __forceinline__ void rank_group(const NlGeom& g, int tj, int i, const double* xi,
                                           const double* __restrict__ coord, const float4* __restrict__ sorted_l,
                                           const int4* __restrict__ sorted_m, const int4& mi, const float* e_key,
                                           const int* e_idx, const int* e_w, int gs, int ge, int ge4, float tw,
                                           WcodeOf wcode_of, int lane, bool& bad_shift, int* __restrict__ nl_j,
                                           int* __restrict__ nl_code) {
  for (int e0 = gs; e0 < ge; e0 += 32) {
    const int e = e0 + lane;
    if (e >= ge) continue;
    const float ke = e_key[e];
    const float lo_t = ke - tw, hi_t = ke + tw;
    int lo = 0, hi = 0;  // certainly smaller; certainly larger
    for (int f = gs; f < ge4; f += 4) {
      const float4 k4 = *reinterpret_cast<const float4*>(e_key + f);
      lo += (k4.x < lo_t) + (k4.y < lo_t) + (k4.z < lo_t) + (k4.w < lo_t);
      hi += (k4.x > hi_t) + (k4.y > hi_t) + (k4.z > hi_t) + (k4.w > hi_t);
    }
    int je, ce;
    if (!entry_code(sorted_l, sorted_m, e_idx[e], wcode_of(e_w[e]), mi, je, ce)) bad_shift = true;
    int rank = lo;
    if (ge4 - gs - lo - hi > 1) {  // FP32 cannot order some pairs: compare their exact keys
      const double re = exact_r2(g, xi, coord, je, ce);
      for (int f = gs; f < ge; ++f) {
        const float kf = e_key[f];
        if (f == e || kf < lo_t || kf > hi_t) continue;
        int jf, cf;
        entry_code(sorted_l, sorted_m, e_idx[f], wcode_of(e_w[f]), mi, jf, cf);
        const double rf = exact_r2(g, xi, coord, jf, cf);
        rank += rf != re ? rf < re : (jf != je ? jf < je : (unsigned)cf < (unsigned)ce);
      }
    }
    if (rank < g.sel[tj]) {
      const long slot = (long)i * g.nc + g.sel_off[tj] + rank;
      nl_j[slot] = je;
      nl_code[slot] = ce;
    }
  }
}

template <int CAP>
__global__ void __launch_bounds__(kNlWarps * 32)
    k_nlist(const NlGeom* __restrict__ G, const int* __restrict__ atom_frame, const int* __restrict__ cell_off,
            const int* __restrict__ n_sorted, int ncells_total, const double* __restrict__ coord,
            const int* __restrict__ cell_start, const float4* __restrict__ sorted_l, const int4* __restrict__ sorted_m,
            int* __restrict__ nl_j, int* __restrict__ nl_code, int* __restrict__ counts, DevStatus* __restrict__ st) {
  constexpr int CAPP = CAP + 4 * DP_MAX_TYPES;  // room for aligning each type's group to 4 entries
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* wb = smem + (size_t)warp * (CAPP * kNlEntryBytes + 32 * sizeof(NbCell));
  float* e_key = reinterpret_cast<float*>(wb);         // FP32 r^2 of each accepted entry
  int* e_idx = reinterpret_cast<int*>(wb + CAPP * 4);  // its sorted position
  int* e_w = reinterpret_cast<int*>(wb + CAPP * 8);    // wrap code of the cell it was seen through
  NbCell* cells = reinterpret_cast<NbCell*>(wb + CAPP * 12);

  const int w = blockIdx.x * kNlWarps + warp;
  if (w >= *n_sorted) return;  // warp-uniform; atoms of an invalid type were left out
  // warps take centre atoms in sorted (type, cell) order: neighbouring warps share candidates
  const float4 li = sorted_l[w];
  const int4 mi = sorted_m[w];
  const int i = __float_as_int(li.w);
  const int fr = atom_frame ? atom_frame[i] : 0;
  const NlGeom& g = G[fr];
  const int coff = cell_off ? cell_off[fr] : 0;
  const int c0 = (mi.w >> 20) & 1023, c1 = (mi.w >> 10) & 1023, c2 = mi.w & 1023;
  const int n0c = 2 * g.K[0] + 1, n1c = 2 * g.K[1] + 1, n2c = 2 * g.K[2] + 1;
  const int noff = n0c * n1c * n2c;
  const double* xi = coord + 3 * i;
  const float rc2_in = g.rc2_in, rc2_out = g.rc2_out, tw = g.tie_w;

  int cnt = 0;
  bool bad_shift = false;
  for (int tj = 0; tj < g.ntypes; ++tj) {
    cnt = (cnt + 3) & ~3;
    const int gs = cnt;  // this type's entries start here (a multiple of 4)
    const int kbase = tj * ncells_total + coff;
    for (int o0 = 0; o0 < noff; o0 += 32) {
      // ---- the chunk's surrounding cells: one per lane ----
      const int o = o0 + lane;
      int num = 0, beg = 0, W0 = 0, W1 = 0, W2 = 0;
      float f0 = 0.f, f1 = 0.f, f2 = 0.f;
      if (o < noff) {
        const int q0 = div_small(o, g.r_n12c);
        const int rem = o - q0 * (n1c * n2c);
        const int q1 = div_small(rem, g.r_n2c);
        const int d0 = q0 - g.K[0];
        const int d1 = q1 - g.K[1];
        const int d2 = rem - q1 * n2c - g.K[2];
        int v0 = c0 + d0, v1 = c1 + d1, v2 = c2 + d2;
        bool inside = true;
        if (g.periodic) {  // |W| <= ceil(K / ncell): a few steps at most
          while (v0 < 0) { v0 += g.ncell[0]; --W0; }
          while (v0 >= g.ncell[0]) { v0 -= g.ncell[0]; ++W0; }
          while (v1 < 0) { v1 += g.ncell[1]; --W1; }
          while (v1 >= g.ncell[1]) { v1 -= g.ncell[1]; ++W1; }
          while (v2 < 0) { v2 += g.ncell[2]; --W2; }
          while (v2 >= g.ncell[2]) { v2 -= g.ncell[2]; ++W2; }
        } else {
          inside = v0 >= 0 && v1 >= 0 && v2 >= 0 && v0 < g.ncell[0] && v1 < g.ncell[1] && v2 < g.ncell[2];
        }
        if (inside) {
          const int key = kbase + (v0 * g.ncell[1] + v1) * g.ncell[2] + v2;
          beg = cell_start[key];
          num = cell_start[key + 1] - beg;
        }
        const float e0 = small_int_to_float(d0), e1 = small_int_to_float(d1), e2 = small_int_to_float(d2);
        f0 = fmaf(e2, g.hc[6], fmaf(e1, g.hc[3], e0 * g.hc[0]));
        f1 = fmaf(e2, g.hc[7], fmaf(e1, g.hc[4], e0 * g.hc[1]));
        f2 = fmaf(e2, g.hc[8], fmaf(e1, g.hc[5], e0 * g.hc[2]));
      }
      int incl = num;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int x = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += x;
      }
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      const bool nonempty = num > 0;
      const unsigned nemask = __ballot_sync(0xffffffffu, nonempty);
      __syncwarp();
      if (nonempty) {
        NbCell c;
        c.o0 = f0;
        c.o1 = f1;
        c.o2 = f2;
        c.beg = beg;
        c.pex = incl - num;
        c.wcode = pack_shift(W0, W1, W2);
        c.wzero = (W0 | W1 | W2) == 0;
        c.pad = 0;
        cells[__popc(nemask & ((1u << lane) - 1u))] = c;
      }
      __syncwarp();
      // ---- the concatenated candidates of these cells, 32 at a time ----
      // position -> cell: nonempty cells ending at or before the batch start, plus the cell ends
      // inside the batch up to this lane
      auto locate = [&](int G0, int& r) {
        const int before = __popc(__ballot_sync(0xffffffffu, nonempty && incl <= G0));
        const int e = incl - G0;
        const unsigned ends = __reduce_or_sync(0xffffffffu, (nonempty && e > 0 && e < 32) ? (1u << e) : 0u);
        r = before + __popc(ends & ((2u << lane) - 1u));
      };
      int r_nx;
      locate(0, r_nx);
      float4 lj_nx = make_float4(0.f, 0.f, 0.f, 0.f);
      if (lane < total) {
        const NbCell& c = cells[r_nx];
        lj_nx = __ldg(sorted_l + c.beg + lane - c.pex);
      }
      for (int G0 = 0; G0 < total; G0 += 32) {
        const int gp = G0 + lane;
        const int r = r_nx;
        const float4 lj = lj_nx;
        if (G0 + 32 < total) {  // the next batch's positions are in flight while this one is tested
          locate(G0 + 32, r_nx);
          if (gp + 32 < total) {
            const NbCell& c = cells[r_nx];
            lj_nx = __ldg(sorted_l + c.beg + gp + 32 - c.pex);
          }
        }
        bool pass = false;
        int idx = 0, wcode = 0;
        float r2 = 0.f;
        if (gp < total) {
          const NbCell& c = cells[r];
          idx = c.beg + gp - c.pex;
          wcode = c.wcode;
          const float dx = (lj.x - li.x) + c.o0, dy = (lj.y - li.y) + c.o1, dz = (lj.z - li.z) + c.o2;
          r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          const bool self = idx == w && c.wzero;
          if (r2 < rc2_in) {
            pass = !self;
          } else if (r2 <= rc2_out && !self) {  // within the FP32 error of r_c: the exact FP64 test decides
            int j, code;
            if (entry_code(sorted_l, sorted_m, idx, wcode, mi, j, code))
              pass = exact_r2(g, xi, coord, j, code) < g.rc2;
            else
              bad_shift = true;
          }
        }
        const unsigned mask = __ballot_sync(0xffffffffu, pass);
        if (pass) {
          const int pos = cnt + __popc(mask & ((1u << lane) - 1u));
          if (pos < CAP) {
            e_key[pos] = r2;
            e_idx[pos] = idx;
            e_w[pos] = wcode;
          }
        }
        cnt += __popc(mask);
      }
      __syncwarp();  // cells[] is rewritten by the next chunk
    }
    // ---- rank this type's entries under the exact total order ----
    const int ng = cnt - gs;
    const int ge = min(cnt, CAP);
    const int ge4 = gs + ((max(ge - gs, 0) + 3) & ~3);
    if (ge + lane < ge4) e_key[ge + lane] = __int_as_float(0x7f800000);  // +inf: never smaller, always larger
    __syncwarp();
    rank_group(g, tj, i, xi, coord, sorted_l, sorted_m, mi, e_key, e_idx, e_w, gs, ge, ge4, tw,
               [](int wc) { return wc; }, lane, bad_shift, nl_j, nl_code);
    // padding, counts and overflow accounting of this type (entries beyond CAP, an error, are
    // not in the list)
    for (int q = max(ge - gs, 0) + lane; q < g.sel[tj]; q += 32) {
      const long slot = (long)i * g.nc + g.sel_off[tj] + q;
      nl_j[slot] = -1;
      nl_code[slot] = pack_shift(0, 0, 0);
    }
    if (lane == 0) {
      if (counts) counts[(long)i * g.ntypes + tj] = ng;
      if (ng > g.sel[tj]) atomicAdd(&st->sel_overflow, 1);
    }
    __syncwarp();
  }
  if (__any_sync(0xffffffffu, bad_shift) && lane == 0) atomicExch(&st->capacity, 2);
  if (cnt > CAP && lane == 0) atomicExch(&st->capacity, 1);
}


// =============================================================================================
// Cell-centred search: one CTA per cell.  The candidates of every (type, surrounding cell)
// range are staged once in shared memory, each type's stretch padded to a multiple of 64 with
// far-away sentinels: the FP32 position l_j + o (o the surrounding cell's corner offset), the
// atom index j, and W - m_j (the cell's periodic wrap minus j's image index) for the image
// code.  Each warp then owns one centre atom of the cell and walks a type's stretch 64
// candidates at a time with one shared load, three subtractions, three multiply-adds and one
// comparison against the outer FP32 bound per candidate; the accepted entries keep the FP32 r^2
// and the stream position.  Everything else happens on the few accepted entries of one type:
// the exact FP64 membership test of entries inside the FP32 error of r_c, the ranking under the
// exact total order (a bucket sort of the FP32 keys; exact keys only for entries with another key
// inside their tie window), and the image codes, all from shared memory.  Membership, ranking and
// outputs are those of k_nlist.
// =============================================================================================
constexpr int kCellWarps = 8;
constexpr int kMaxRanges = 256;  // (type, surrounding cell) ranges of one cell

// Dynamic shared memory: S staged candidates (24 bytes each) and per warp an entry buffer of
// cap + 4 entries (FP32 key, 16-bit stream position, 16-bit entry index in bucket order) and
// cap bucket counters (the FP32 keys of one type group are bucketed over [0, r_c^2 + eps], as
// many buckets as the buffer has entries).
__host__ __device__ constexpr size_t cell_smem_bytes(int cap, int S) {
  return (size_t)S * 24 + (size_t)kCellWarps * ((size_t)(cap + 4) * 8 + (size_t)cap * 4);
}

// Bucket of an FP32 key: monotone in x, so that every key of a lower bucket is smaller and every
// key of a higher bucket larger.
template <int NB>
__device__ __forceinline__ int key_bucket(float x, float inv_w) {
  return min(NB - 1, max(0, __float2int_rz(x * inv_w)));
}

// Cell of an orthogonal periodic box (zero off-diagonal entries): the diagonal and its negation.
struct OrthoCell {
  bool on;
  double h[3], nh[3];
};
__device__ __forceinline__ bool is_zero_bits(double x) { return (__double_as_longlong(x) << 1) == 0; }
__device__ __forceinline__ OrthoCell ortho_cell(const NlGeom& g) {
  OrthoCell o;
  o.on = g.periodic && is_zero_bits(g.h[1]) && is_zero_bits(g.h[2]) && is_zero_bits(g.h[3]) &&
         is_zero_bits(g.h[5]) && is_zero_bits(g.h[6]) && is_zero_bits(g.h[7]);
  for (int a = 0; a < 3; ++a) {
    o.h[a] = g.h[4 * a];
    o.nh[a] = __longlong_as_double(__double_as_longlong(o.h[a]) ^ (long long)0x8000000000000000ull);
  }
  return o;
}

// exact_r2 for the membership test and the ranking, which use only r^2.  In an orthogonal cell
// with every |n_a| <= 1 the translation component t_a = n_0 h_0a + n_1 h_1a + n_2 h_2a is n_a h_aa
// plus products with zero entries: -h_aa, a zero or h_aa exactly, taken without a multiplication.
// Zero terms leave the sums unchanged up to the sign of a zero, which r^2 does not see, so the
// result is the one of exact_r2 bit for bit.
__device__ __forceinline__ double exact_r2_rank(const NlGeom& g, const OrthoCell& oc, const double* xi,
                                                const double* __restrict__ coord, int j, int code) {
  int n0, n1, n2;
  unpack_shift(code, n0, n1, n2);
  if (code != pack_shift(0, 0, 0) && oc.on && abs(n0) <= 1 && abs(n1) <= 1 && abs(n2) <= 1) {
    const double* xj = coord + 3 * j;
    const double t0 = n0 == 0 ? 0.0 : (n0 > 0 ? oc.h[0] : oc.nh[0]);
    const double t1 = n1 == 0 ? 0.0 : (n1 > 0 ? oc.h[1] : oc.nh[1]);
    const double t2 = n2 == 0 ? 0.0 : (n2 > 0 ? oc.h[2] : oc.nh[2]);
    const double d0 = __dsub_rn(__dadd_rn(xj[0], t0), xi[0]);
    const double d1 = __dsub_rn(__dadd_rn(xj[1], t1), xi[1]);
    const double d2 = __dsub_rn(__dadd_rn(xj[2], t2), xi[2]);
    return norm2_exact(d0, d1, d2);
  }
  return exact_r2(g, xi, coord, j, code);
}

// W - m_j as three 21-bit two's-complement fields; bit 63 marks a value outside that range.
__device__ __forceinline__ unsigned long long pack_wm(int a, int b, int c) {
  const unsigned long long M = (1ull << 21) - 1;
  const bool ok = a >= -(1 << 20) && a < (1 << 20) && b >= -(1 << 20) && b < (1 << 20) && c >= -(1 << 20) &&
                  c < (1 << 20);
  return ok ? (((unsigned long long)(unsigned)a & M) | (((unsigned long long)(unsigned)b & M) << 21) |
               (((unsigned long long)(unsigned)c & M) << 42))
            : (1ull << 63);
}
// Image code n = (W - m_j) + m_i of a staged entry; false when n leaves the packable range.
__device__ __forceinline__ bool staged_code(unsigned long long wm, int mi0, int mi1, int mi2, int& code) {
  const int n0 = (int)((long long)(wm << 43) >> 43) + mi0;
  const int n1 = (int)((long long)(wm << 22) >> 43) + mi1;
  const int n2 = (int)((long long)(wm << 1) >> 43) + mi2;
  code = 0;
  if ((wm >> 63) || n0 <= -512 || n0 >= 512 || n1 <= -512 || n1 >= 512 || n2 <= -512 || n2 >= 512) return false;
  code = pack_shift(n0, n1, n2);
  return true;
}

template <int CAP>
__global__ void __launch_bounds__(kCellWarps * 32, 4)
    k_nlist_cell(const NlGeom* __restrict__ G, const int* __restrict__ cell_off, int nframes, int ncells_total,
                 int ntypes, const double* __restrict__ coord, const int* __restrict__ cell_start,
                 const float4* __restrict__ sorted_l, const int4* __restrict__ sorted_m, int S, int* __restrict__ nl_j,
                 int* __restrict__ nl_code, int* __restrict__ counts, float4* __restrict__ disp,
                 DevStatus* __restrict__ st) {
  constexpr int NT = kCellWarps * 32;
  constexpr int CAPP = CAP + 4;
  extern __shared__ __align__(16) unsigned char smem[];
  float4* stg = reinterpret_cast<float4*>(smem);                                        // l_j + o, j
  unsigned long long* stg_w = reinterpret_cast<unsigned long long*>(smem + (size_t)S * 16);  // W - m_j
  __shared__ int s_rbeg[kMaxRanges], s_rnum[kMaxRanges], s_rpex[kMaxRanges + 1];
  __shared__ float4 s_off[kMaxRanges];  // per surrounding cell: o, and its wrap code
  __shared__ int s_tpex[DP_MAX_TYPES + 1], s_tdel[DP_MAX_TYPES], s_cpre[DP_MAX_TYPES + 1], s_wsum[kCellWarps];
  __shared__ int s_sel[DP_MAX_TYPES], s_seloff[DP_MAX_TYPES];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
  constexpr int NB = CAP;  // key buckets
  float* e_key = reinterpret_cast<float*>(smem + (size_t)S * 24 + (size_t)warp * (CAPP * 8 + NB * 4));
  unsigned short* e_ref = reinterpret_cast<unsigned short*>(e_key + CAPP);  // stream position (S < 2^16)
  unsigned short* e_idx = e_ref + CAPP;                                     // entries in bucket order
  int* e_hist = reinterpret_cast<int*>(e_idx + CAPP);                       // bucket ends

  const int gc = blockIdx.x;  // cell, all frames
  int fr = 0;
  if (cell_off) {  // frame holding this cell
    int lo = 0, hi = nframes - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (cell_off[mid] <= gc) lo = mid; else hi = mid - 1;
    }
    fr = lo;
  }
  const NlGeom& g = G[fr];
  const int ci = gc - (cell_off ? cell_off[fr] : 0);
  const int kb0 = gc - ci;  // first cell of the frame
  const int c2 = ci % g.ncell[2];
  const int c1 = (ci / g.ncell[2]) % g.ncell[1];
  const int c0 = ci / (g.ncell[2] * g.ncell[1]);
  const int n0c = 2 * g.K[0] + 1, n1c = 2 * g.K[1] + 1, n2c = 2 * g.K[2] + 1;
  const int noff = n0c * n1c * n2c;
  const int oc = (g.K[0] * n1c + g.K[1]) * n2c + g.K[2];  // slot of the cell itself
  const int R = ntypes * noff;  // <= kMaxRanges (checked on the host)
  if (tid < ntypes) {
    s_sel[tid] = g.sel[tid];
    s_seloff[tid] = g.sel_off[tid];
  }

  // ---- the (type, surrounding cell) ranges and their positions in the candidate stream ----
  int num = 0;
  if (tid < R) {
    const int t = tid / noff, o = tid - t * noff;
    const int q0 = o / (n1c * n2c), rem = o - q0 * (n1c * n2c), q1 = rem / n2c;
    const int d0 = q0 - g.K[0], d1 = q1 - g.K[1], d2 = rem - q1 * n2c - g.K[2];
    int v0 = c0 + d0, v1 = c1 + d1, v2 = c2 + d2, W0 = 0, W1 = 0, W2 = 0;
    bool inside = true;
    if (g.periodic) {
      while (v0 < 0) { v0 += g.ncell[0]; --W0; }
      while (v0 >= g.ncell[0]) { v0 -= g.ncell[0]; ++W0; }
      while (v1 < 0) { v1 += g.ncell[1]; --W1; }
      while (v1 >= g.ncell[1]) { v1 -= g.ncell[1]; ++W1; }
      while (v2 < 0) { v2 += g.ncell[2]; --W2; }
      while (v2 >= g.ncell[2]) { v2 -= g.ncell[2]; ++W2; }
    } else {
      inside = v0 >= 0 && v1 >= 0 && v2 >= 0 && v0 < g.ncell[0] && v1 < g.ncell[1] && v2 < g.ncell[2];
    }
    int beg = 0;
    if (inside) {
      const int key = t * ncells_total + kb0 + (v0 * g.ncell[1] + v1) * g.ncell[2] + v2;
      beg = cell_start[key];
      num = cell_start[key + 1] - beg;
    }
    s_rbeg[tid] = beg;
    s_rnum[tid] = num;
    if (t == 0) {
      const float e0 = (float)d0, e1 = (float)d1, e2 = (float)d2;
      s_off[o] = make_float4(fmaf(e2, g.hc[6], fmaf(e1, g.hc[3], e0 * g.hc[0])),
                             fmaf(e2, g.hc[7], fmaf(e1, g.hc[4], e0 * g.hc[1])),
                             fmaf(e2, g.hc[8], fmaf(e1, g.hc[5], e0 * g.hc[2])), __int_as_float(pack_shift(W0, W1, W2)));
    }
  }
  int incl = num;  // block-wide inclusive scan of the range sizes (R <= NT)
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int x = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += x;
  }
  if (lane == 31) s_wsum[warp] = incl;
  __syncthreads();
  int wbase = 0;
  for (int k = 0; k < warp; ++k) wbase += s_wsum[k];
  if (tid < R) s_rpex[tid] = wbase + incl - num;
  if (tid == NT - 1) s_rpex[R] = wbase + incl;  // threads >= R hold no range: this is the total
  __syncthreads();
  if (tid == 0) {  // each type's stretch starts at a multiple of 64; centre atoms by type
    int p = 0, c = 0;
    for (int t = 0; t < ntypes; ++t) {
      const int a = s_rpex[t * noff], b = s_rpex[(t + 1) * noff];
      s_tpex[t] = p;
      s_tdel[t] = p - a;
      p += (b - a + 63) & ~63;
      s_cpre[t] = c;
      c += s_rnum[t * noff + oc];
    }
    s_tpex[ntypes] = p;
    s_cpre[ntypes] = c;
  }
  __syncthreads();
  if (tid < R) s_rpex[tid] += s_tdel[tid / noff];
  const int P = s_tpex[ntypes];
  const int nce = s_cpre[ntypes];
  if (nce == 0) return;  // CTA-uniform: no centre atom in this cell
  if (P > S) {  // CTA-uniform: the stream does not fit the staging buffer.  The call reports it
                // (and is retried on the per-atom kernel); meanwhile this cell's rows are left
                // empty, so that the kernels after the list stay in bounds.
    if (tid == 0) atomicExch(&st->capacity, 1);
    for (int q = warp; q < nce; q += kCellWarps) {
      int tc = 0;
      while (tc + 1 < ntypes && s_cpre[tc + 1] <= q) ++tc;
      const int w = s_rbeg[tc * noff + oc] + q - s_cpre[tc];
      const int i = __float_as_int(__ldg(&sorted_l[w].w));
      for (int k = lane; k < g.nc; k += 32) {
        nl_j[(long)i * g.nc + k] = -1;
        nl_code[(long)i * g.nc + k] = pack_shift(0, 0, 0);
        if (disp) disp[(long)w * g.nc + k] = make_float4(0.f, 0.f, 0.f, -1.f);
      }
      if (counts && lane < ntypes) counts[(long)i * ntypes + lane] = 0;
    }
    return;
  }
  __syncthreads();

  // ---- stage the stream ----
  for (int p = tid; p < P; p += NT) {
    int lo = 0, hi = R - 1;  // last range starting at or before p
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_rpex[mid] <= p) lo = mid; else hi = mid - 1;
    }
    const int k = p - s_rpex[lo];
    if (k < s_rnum[lo]) {
      const int src = s_rbeg[lo] + k;
      const float4 lj = __ldg(sorted_l + src);
      const int4 mj = __ldg(sorted_m + src);
      const float4 of = s_off[lo % noff];
      int W0, W1, W2;
      unpack_shift(__float_as_int(of.w), W0, W1, W2);
      stg[p] = make_float4(lj.x + of.x, lj.y + of.y, lj.z + of.z, lj.w);
      stg_w[p] = pack_wm(W0 - mj.x, W1 - mj.y, W2 - mj.z);
    } else {  // padding: never within r_c of anything
      stg[p] = make_float4(1e30f, 1e30f, 1e30f, __int_as_float(-1));
      stg_w[p] = 0;
    }
  }
  __syncthreads();

  const float rc2_in = g.rc2_in, rc2_out = g.rc2_out, tw = g.tie_w;
  const float inv_bw = (float)NB / rc2_out;
  const OrthoCell ocell = ortho_cell(g);
  const int nc = g.nc;
  const unsigned lt = (1u << lane) - 1u;
  const float kInf = __int_as_float(0x7f800000);
  for (int q = warp; q < nce; q += kCellWarps) {
    int tc = 0;
    while (tc + 1 < ntypes && s_cpre[tc + 1] <= q) ++tc;
    const int pc = s_rpex[tc * noff + oc] + q - s_cpre[tc];  // the centre's own entry (W = 0)
    const int w = s_rbeg[tc * noff + oc] + q - s_cpre[tc];  // its sorted position
    const float4 li = stg[pc];
    const int i = __float_as_int(li.w);
    bool bad_shift, over = false;
    int mi0, mi1, mi2;
    {
      const unsigned long long wm = stg_w[pc];  // -m_i
      mi0 = -(int)((long long)(wm << 43) >> 43);
      mi1 = -(int)((long long)(wm << 22) >> 43);
      mi2 = -(int)((long long)(wm << 1) >> 43);
      bad_shift = (wm >> 63) != 0;
    }
    const double* xi = coord + 3 * i;
    for (int tj = 0; tj < ntypes; ++tj) {
      // ---- walk: FP32 screening against the outer bound ----
      const int ts = s_tpex[tj], te = s_tpex[tj + 1];
      int cnt = 0;
      for (int p = ts + lane; p < te; p += 64) {
        const float4 sa = stg[p], sb = stg[p + 32];
        const float ax = sa.x - li.x, ay = sa.y - li.y, az = sa.z - li.z;
        const float bx = sb.x - li.x, by = sb.y - li.y, bz = sb.z - li.z;
        const float ra = fmaf(ax, ax, fmaf(ay, ay, az * az));
        const float rb = fmaf(bx, bx, fmaf(by, by, bz * bz));
        const bool pa = ra <= rc2_out && p != pc, pb = rb <= rc2_out && p + 32 != pc;
        const unsigned ma = __ballot_sync(0xffffffffu, pa), mb = __ballot_sync(0xffffffffu, pb);
        const int na = __popc(ma);
        if (pa) {
          const int pos = cnt + __popc(ma & lt);
          if (pos < CAP) {
            e_key[pos] = ra;
            e_ref[pos] = (unsigned short)p;
          }
        }
        if (pb) {
          const int pos = cnt + na + __popc(mb & lt);
          if (pos < CAP) {
            e_key[pos] = rb;
            e_ref[pos] = (unsigned short)(p + 32);
          }
        }
        cnt += na + __popc(mb);
      }
      over |= cnt > CAP;
      const int ge = min(cnt, CAP);
      __syncwarp();
      // ---- bucket order of the surviving FP32 keys ----
      // Counting sort into NB buckets of the keys' range: counts, exclusive scan, scatter of the
      // entry indices; afterwards e_hist[b] is the end of bucket b in e_idx.  The counting pass
      // first settles the entries within the FP32 error of r_c by the exact FP64 test (dropped
      // entries get the key +inf and no bucket).
      for (int b = lane; b < NB; b += 32) e_hist[b] = 0;
      __syncwarp();
      int removed = 0;
      for (int e0 = 0; e0 < ge; e0 += 32) {
        const int e = e0 + lane;
        float k = e < ge ? e_key[e] : kInf;
        const bool need = k != kInf && k >= rc2_in;
        if (__ballot_sync(0xffffffffu, need)) {
          bool drop = false;
          if (need) {
            const int p = e_ref[e];
            int code;
            if (staged_code(stg_w[p], mi0, mi1, mi2, code))
              drop = !(exact_r2_rank(g, ocell, xi, coord, __float_as_int(stg[p].w), code) < g.rc2);
            else
              drop = bad_shift = true;
            if (drop) {
              e_key[e] = kInf;
              k = kInf;
            }
          }
          removed += __popc(__ballot_sync(0xffffffffu, drop));
        }
        if (k != kInf) atomicAdd(&e_hist[key_bucket<NB>(k, inv_bw)], 1);
      }
      __syncwarp();
      {
        constexpr int PER = NB / 32;  // buckets per lane, contiguous
        int c[PER];
        int sum = 0;
#pragma unroll
        for (int v = 0; v < PER / 4; ++v) {
          const int4 x = reinterpret_cast<const int4*>(e_hist)[lane * (PER / 4) + v];
          c[4 * v] = x.x;
          c[4 * v + 1] = x.y;
          c[4 * v + 2] = x.z;
          c[4 * v + 3] = x.w;
          sum += x.x + x.y + x.z + x.w;
        }
        int incl = sum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const int x = __shfl_up_sync(0xffffffffu, incl, off);
          if (lane >= off) incl += x;
        }
        int run = incl - sum;
#pragma unroll
        for (int v = 0; v < PER / 4; ++v) {
          int4 x;
          x.x = run;
          run += c[4 * v];
          x.y = run;
          run += c[4 * v + 1];
          x.z = run;
          run += c[4 * v + 2];
          x.w = run;
          run += c[4 * v + 3];
          reinterpret_cast<int4*>(e_hist)[lane * (PER / 4) + v] = x;
        }
      }
      __syncwarp();
      for (int e = lane; e < ge; e += 32) {
        const float k = e_key[e];
        if (k != kInf) e_idx[atomicAdd(&e_hist[key_bucket<NB>(k, inv_bw)], 1)] = (unsigned short)e;
      }
      __syncwarp();
      // ---- rank under the exact total order (r^2, j, image code) ----
      // Entries more than the tie window below an entry's key are certainly smaller: all of the
      // buckets below the window's lower edge and the smaller keys of the edge bucket.  Entries
      // inside the window (in bucket order between the two edge buckets) take exact keys.
      const int sel = s_sel[tj];
      const long row = (long)i * nc + s_seloff[tj];
      for (int e0 = 0; e0 < ge; e0 += 32) {
        const int e = e0 + lane;
        const float ke = e < ge ? e_key[e] : kInf;
        const bool valid = ke != kInf;
        const float lo_t = ke - tw, hi_t = ke + tw;
        int lo = 0, nle = 0;  // keys certainly smaller; keys not certainly larger
        int wa = 0, wb = 0;   // bucket-order positions spanning the window
        if (valid) {
          const int bl = key_bucket<NB>(lo_t, inv_bw), bh = key_bucket<NB>(hi_t, inv_bw);
          wa = bl ? e_hist[bl - 1] : 0;
          wb = e_hist[bh];
          lo = wa;
          if (bl == bh) {  // the usual case: the window inside one bucket
            nle = wa;
            for (int q = wa; q < wb; ++q) {
              const float kq = e_key[e_idx[q]];
              lo += kq < lo_t;
              nle += kq <= hi_t;
            }
          } else {
            for (int q = wa, qe = e_hist[bl]; q < qe; ++q) lo += e_key[e_idx[q]] < lo_t;
            const int sh = e_hist[bh - 1];
            nle = sh;
            for (int q = sh; q < wb; ++q) nle += e_key[e_idx[q]] <= hi_t;
          }
        }
        int je = 0, ce = 0;
        if (valid) {
          const int p = e_ref[e];
          je = __float_as_int(stg[p].w);
          if (!staged_code(stg_w[p], mi0, mi1, mi2, ce)) bad_shift = true;
        }
        int rank = lo;
        const bool amb = valid && nle - lo > 1;  // the window holds another entry
        unsigned am = __ballot_sync(0xffffffffu, amb);
        if (am) {  // FP32 cannot order some pairs: their exact keys decide
          const double re = amb ? exact_r2_rank(g, ocell, xi, coord, je, ce) : 0.0;
          const unsigned am0 = am;
          while (am) {
            const int s = __ffs(am) - 1;
            am &= am - 1;
            const float lo_s = __shfl_sync(0xffffffffu, lo_t, s), hi_s = __shfl_sync(0xffffffffu, hi_t, s);
            const int je_s = __shfl_sync(0xffffffffu, je, s), ce_s = __shfl_sync(0xffffffffu, ce, s);
            const double re_s = __shfl_sync(0xffffffffu, re, s);
            const int wa_s = __shfl_sync(0xffffffffu, wa, s), wb_s = __shfl_sync(0xffffffffu, wb, s);
            int add = 0;
            for (int q0 = wa_s; q0 < wb_s; q0 += 32) {
              const int q = q0 + lane;
              const int f = q < wb_s ? e_idx[q] : -1;
              const float kf = f >= 0 ? e_key[f] : kInf;
              const bool in = f >= 0 && f != e0 + s && kf >= lo_s && kf <= hi_s;
              // a partner that is an ambiguous entry of this pass has its exact key in its lane
              const int src = (f - e0) & 31;
              const double r_src = __shfl_sync(0xffffffffu, re, src);
              const int j_src = __shfl_sync(0xffffffffu, je, src), c_src = __shfl_sync(0xffffffffu, ce, src);
              const bool known = f >= e0 && f < e0 + 32 && ((am0 >> src) & 1u);
              if (__ballot_sync(0xffffffffu, in)) {
                bool less = false;
                if (in) {
                  int jf, cf;
                  double rf;
                  if (known) {
                    jf = j_src;
                    cf = c_src;
                    rf = r_src;
                  } else {
                    const int p = e_ref[f];
                    jf = __float_as_int(stg[p].w);
                    staged_code(stg_w[p], mi0, mi1, mi2, cf);
                    rf = exact_r2_rank(g, ocell, xi, coord, jf, cf);
                  }
                  less = rf != re_s ? rf < re_s : (jf != je_s ? jf < je_s : (unsigned)cf < (unsigned)ce_s);
                }
                add += __popc(__ballot_sync(0xffffffffu, less));
              }
            }
            if (lane == s) rank += add;
          }
        }
        if (valid && rank < sel) {
          nl_j[row + rank] = je;
          nl_code[row + rank] = ce;
          if (disp) {
            const float4 sj = stg[e_ref[e]];
            disp[(long)w * nc + s_seloff[tj] + rank] =
                make_float4(sj.x - li.x, sj.y - li.y, sj.z - li.z, ke < rc2_in ? 1.f : 0.f);
          }
        }
      }
      // ---- padding, counts and overflow accounting of this type ----
      // The displacements' reader walks a type block in 32-slot batches and stops after the first
      // batch that holds padding, so padding displacements are written only up to the end of the
      // batch after the last real neighbour.
      const int ng = cnt - removed;  // entries beyond CAP (an error) are not in the list
      const int nreal = ge - removed;
      const int dlim = min(sel, ((nreal >> 5) + 1) << 5);
      for (int k = nreal + lane; k < sel; k += 32) {
        nl_j[row + k] = -1;
        nl_code[row + k] = pack_shift(0, 0, 0);
        if (disp && k < dlim) disp[(long)w * nc + s_seloff[tj] + k] = make_float4(0.f, 0.f, 0.f, -1.f);
      }
      if (lane == 0) {
        if (counts) counts[(long)i * ntypes + tj] = ng;
        if (ng > sel) atomicAdd(&st->sel_overflow, 1);
      }
      __syncwarp();  // the entry buffer is rewritten by the next type
    }
    if (__any_sync(0xffffffffu, bad_shift) && lane == 0) atomicExch(&st->capacity, 2);
    if (over && lane == 0) atomicExch(&st->capacity, 1);
  }
}

// Stable partition of atoms by type (one block, one pass): each thread takes a contiguous
// chunk of atoms, counts per type, and a block-wide exclusive scan of the counts gives every
// thread its output offset per type.  perm[p] = atom index, type_start[t].
__global__ void __launch_bounds__(1024)
    k_type_perm(const int* __restrict__ type, int n, int ntypes, int* __restrict__ perm, int* __restrict__ type_start,
                DevStatus* __restrict__ status, const TypeStartCheck chk) {
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
  if (bad) atomicExch(&status->bad_type, 1);
  if (chk.on && tid <= ntypes && tstart[tid] != chk.v[tid]) atomicExch(&status->type_change, 1);
  if (tid <= ntypes) type_start[tid] = tstart[tid];
}

}  // namespace

namespace {

float round_down(double v) {
  float f = (float)v;
  if ((double)f > v) f = std::nextafter(f, -INFINITY);
  return f;
}
float round_up(double v) {
  float f = (float)v;
  if ((double)f < v) f = std::nextafter(f, INFINITY);
  return f;
}

// Cell edge vectors and the FP32 screening thresholds.  The walks form the displacement as
// (l_j - l_i) + o or (l_j + o) - l_i with l the FP32 cell-local positions (|l_d| <= A) and o the
// FP32 offset of a surrounding cell (|o_d| <= B, three FP32 operations from the rounded edge
// vectors).  With u = 2^-24 each component is within u (6A + 6B) of the exact FP64
// displacement, plus a slack for FP64 rounding of coordinates up to 1e6 A.  For |d| <= R = r_c + 1 the FP32 r^2 (three
// rounded operations) is then within 2 sqrt(3) R dc + 3 dc^2 + 3 u R^2 of the FP64 r^2; eps
// doubles that.  Keys further apart than 2 eps (plus the rounding of the comparison itself)
// keep their FP64 order.
int screening_bounds(NlGeom& g, double rc) {
  const int n2c = 2 * g.K[2] + 1, n12c = (2 * g.K[1] + 1) * n2c;
  if ((long)(2 * g.K[0] + 1) * n12c >= (1L << 21)) {
    set_error("too many periodic images of the cell grid (box far narrower than r_c)");
    return DP_E_ARG;
  }
  g.r_n2c = (float)(1.0 / n2c);
  g.r_n12c = (float)(1.0 / n12c);
  for (int d = 0; d < 3; ++d) {
    g.rn[d] = 1.0 / g.ncell[d];
    g.rext[d] = g.periodic ? 0.0 : 1.0 / g.ext[d];
  }
  double hc[9];
  for (int e = 0; e < 3; ++e)
    for (int d = 0; d < 3; ++d)
      hc[e * 3 + d] = g.periodic ? g.h[e * 3 + d] / g.ncell[e] : (e == d ? g.ext[d] / g.ncell[d] : 0.0);
  double A = 0.0, B = 0.0;
  for (int d = 0; d < 3; ++d) {
    double a = 0.0, b = 0.0;
    for (int e = 0; e < 3; ++e) {
      a += std::fabs(hc[e * 3 + d]);
      b += g.K[e] * std::fabs(hc[e * 3 + d]);
    }
    A = std::max(A, a);
    B = std::max(B, b);
  }
  for (int k = 0; k < 9; ++k) g.hc[k] = (float)hc[k];
  A = 1.01 * A + 1e-6;
  B = 1.01 * B + 1e-6;
  const double u = std::ldexp(1.0, -24);
  const double dc = u * (6.0 * A + 6.0 * B) + 1e-9;
  if (dc > 1e-2) {
    set_error("cells too large for the FP32 distance screening of the neighbour search");
    return DP_E_ARG;
  }
  const double R = rc + 1.0;
  const double eps = 2.0 * (2.0 * std::sqrt(3.0) * R * dc + 3.0 * dc * dc + 3.0 * u * R * R);
  g.rc2_in = round_down(g.rc2 - eps);
  g.rc2_out = round_up(g.rc2 + eps);
  // Each FP32 key is within eps / 2 of its pair's FP64 r^2, and forming a window edge key -+ tie_w
  // in FP32 moves it by at most u (r_c^2 + eps): keys further apart than eps + 2u (r_c^2 + eps + 1)
  // keep their order in FP64.  The window is a quarter wider than that on the eps term and four
  // times on the rounding term.
  g.tie_w = round_up(1.25 * eps + 8.0 * u * (g.rc2_out + 1.0));
  return DP_OK;
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
  const double cellmin = rc * (1.0 + 1e-9) + 1e-9;
  if (box) {
    g.periodic = 1;
    const double* h = box;
    for (int k = 0; k < 9; ++k) g.h[k] = h[k];
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
  }
  return screening_bounds(g, rc);
}

int nlist_launches(const NlLaunch& L, int ntypes) { return (long)L.ncells_total * ntypes <= 8192 ? 3 : 4; }

cudaError_t launch_bbox(const double* coord, int natoms, double* out_lohi, cudaStream_t st) {
  k_bbox<<<1, 1024, 0, st>>>(coord, natoms, out_lohi);
  return cudaGetLastError();
}

cudaError_t launch_nlist_build(const NlLaunch& L, int ntypes, const double* coord, const int* type,
                               const NlScratch& sc, int* nl_j, int* nl_code, int* counts, DevStatus* status,
                               cudaStream_t st, NlExtras* ex) {
  if (ex) ex->disp_written = false;
  int* cell_count = sc.cell_count;
  int* cell_start = sc.cell_start;
  const float4* sorted_l = sc.sorted_l;
  const int4* sorted_m = sc.sorted_m;
  const int nkeys = L.ncells_total * ntypes;
  cudaError_t e = cudaMemsetAsync(cell_count, 0, sizeof(int) * nkeys, st);
  if (e != cudaSuccess) return e;
  const int nb = (L.natoms + 255) / 256;
  TypeStartCheck nochk;
  std::memset(&nochk, 0, sizeof(nochk));
  k_bin<<<nb, 256, 0, st>>>(L.geoms, L.atom_frame, L.cell_off, L.natoms, L.ncells_total, ntypes, coord, type,
                            cell_count, sc.atom_key, sc.atom_l, sc.atom_m, status, ex ? ex->boxes : nullptr,
                            ex ? ex->nframes : 0, ex ? ex->tshift : nullptr);
  if (nkeys <= 8192) {  // few keys: each fill block scans the counts itself (one launch fewer; nlist_launches)
    k_fill_scan<<<nb, 256, (size_t)(nkeys + 1) * sizeof(int), st>>>(
        L.natoms, cell_count, nkeys, cell_start, sc.atom_key, sc.atom_l, sc.atom_m, sc.sorted_l, sc.sorted_m,
        ex ? ex->perm : nullptr, ex ? ex->type_start : nullptr, L.ncells_total, ntypes, status, ex ? ex->chk : nochk);
  } else {
    k_scan_excl<<<1, 1024, 0, st>>>(cell_count, nkeys, cell_start, nullptr);
    k_fill<<<nb, 256, 0, st>>>(L.natoms, sc.atom_key, sc.atom_l, sc.atom_m, sc.sorted_l, sc.sorted_m,
                               ex ? ex->perm : nullptr, ex ? ex->type_start : nullptr, cell_start, L.ncells_total,
                               ntypes, status, ex ? ex->chk : nochk);
  }
  const int cap = L.cap <= 128 ? 128 : (L.cap <= 256 ? 256 : (L.cap <= 512 ? 512 : 1024));
  // cell-centred search, one CTA per cell, when a cell's candidate stream fits shared memory:
  // room for 1.25 times the mean stream of a cell plus each type's padding (a cell with more
  // reports a capacity error, and the call is retried on the per-atom kernel below)
  const double mean_stream = L.max_stream > 0 ? (double)L.max_stream
                                              : (double)L.natoms / std::max(1, L.ncells_total) * std::max(1, L.max_noff);
  const int S = std::max(1024, ((int)(1.25 * mean_stream) + 64 * ntypes + 64 + 127) & ~127);
  const size_t csm = cell_smem_bytes(cap, S);
  if (L.max_noff > 0 && (long)L.max_noff * ntypes <= kMaxRanges && cap <= 512 && csm <= 160 * 1024 && S < 65536) {
#define DPGB_NLC_LAUNCH(C)                                                                                       \
  do {                                                                                                           \
    e = allow_max_smem(k_nlist_cell<C>);                                                                         \
    if (e != cudaSuccess) return e;                                                                              \
    k_nlist_cell<C><<<L.ncells_total, kCellWarps * 32, csm, st>>>(L.geoms, L.cell_off, L.nframes,               \
                                                                  L.ncells_total, ntypes, coord, cell_start,     \
                                                                  sorted_l, sorted_m, S, nl_j, nl_code, counts,  \
                                                                  ex ? ex->disp : nullptr, status);              \
  } while (0)
    if (cap == 128)
      DPGB_NLC_LAUNCH(128);
    else if (cap == 256)
      DPGB_NLC_LAUNCH(256);
    else
      DPGB_NLC_LAUNCH(512);
#undef DPGB_NLC_LAUNCH
    if (ex) ex->disp_written = ex->disp != nullptr;
    return cudaGetLastError();
  }
  const size_t smem = (size_t)kNlWarps * ((size_t)(cap + 4 * DP_MAX_TYPES) * kNlEntryBytes + 32 * sizeof(NbCell));
  const unsigned blocks = (L.natoms + kNlWarps - 1) / kNlWarps;
#define DPGB_NL_LAUNCH(C)                                                                                       \
  do {                                                                                                          \
    e = allow_max_smem(k_nlist<C>);               \
    if (e != cudaSuccess) return e;                                                                             \
    k_nlist<C><<<blocks, kNlWarps * 32, smem, st>>>(L.geoms, L.atom_frame, L.cell_off, cell_start + nkeys,      \
                                                   L.ncells_total, coord, cell_start, sorted_l, sorted_m, nl_j, \
                                                   nl_code, counts, status);                                    \
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

cudaError_t launch_type_perm(const int* type, int natoms, int ntypes, int* perm, int* type_start, DevStatus* status,
                             const TypeStartCheck& chk,
                             cudaStream_t st) {
  k_type_perm<<<1, 1024, 0, st>>>(type, natoms, ntypes, perm, type_start, status, chk);
  return cudaGetLastError();
}

}  // namespace dpgb
