// The energy / force / virial path on CUDA cores (FP64 or FP32 networks), for the se_e2_a,
// se_e2_r, se_e3 and hybrid descriptors.
//
// Steps (sorted-atom index p, neighbour slot k, row = p * Nc + k):
//   env      R_k = (s, s u) with u = r_ij / r, s = s(r)            Eqs. (rij), (switch)
//   emb      G_k = N^{a_i, a_j}(s) layer by layer                  Eqs. (G2), (NN)
//   contract T = G^T R / Nc,  D = T T_<^T                          se_e2_a descriptor
//            D_r = G_r^T s / Nc                                    se_e2_r descriptor
//            D_3 = (R R^T) : G_3 / Nc^2                            se_e3 descriptor
//            (hybrid: D = [D_1, D_2], each part with its own cutoffs, sel and nets)  Sec. II.A.1
//   fit      E_i = F^{a_i}(D)                                      Eq. (fitting_energy)
//   backward dE/dD -> dE/dT -> (dE/dG, dE/dR) -> dE/ds -> dE/dr_ij
//   force    F_i += dE/dr_ij, F_j -= dE/dr_ij (FP64 atomics)        Sec. II.A.2
//   virial   Xi_ab = -sum (dE/dr_ij)_a (r_ij)_b (FP64, deterministic two-stage reduction)
//
// The pair displacement is always rebuilt from the neighbour list with the exact FP64
// formula.  In FP32 mode the switch and its derivative are evaluated in FP32 in a form without
// cancellation near r_c (env.cuh); energy, force and virial accumulate in FP64.
#include <type_traits>

#include "dp_internal.cuh"
#include "path.cuh"
#include "env.cuh"
#include "tabeval.cuh"

namespace dpgb {

namespace {

// ---- env ------------------------------------------------------------------------------------
template <class R>
__global__ void k_env(PathConst pc, const double* __restrict__ coord, const int* __restrict__ perm,
                      const int* __restrict__ nl_j, const int* __restrict__ nl_code, R* __restrict__ Renv) {
  const long row = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= (long)pc.natoms * pc.nc) return;
  const int p = (int)(row / pc.nc), k = (int)(row % pc.nc);
  const int i = perm[p];
  const long ls = (long)i * pc.lnc + list_slot(pc, k);
  const int j = nl_j[ls];
  R o[4] = {R(0), R(0), R(0), R(0)};
  double d0 = 0.0, d1 = 0.0, d2 = 0.0, r2 = 0.0;
  if (j >= 0) {
    listed_disp(coord + 3 * i, coord + 3 * j, nl_code[ls], pc, frame_of(pc, i), d0, d1, d2);
    r2 = norm2_exact(d0, d1, d2);
  }
  if (j >= 0 && r2 < pc.rc2) {
    R r, s, ds, u[3];
    pair_env<R>(d0, d1, d2, r2, pc.rs, pc.rc, pc.near2, r, s, ds, u);
    o[0] = s;
    o[1] = s * u[0];
    o[2] = s * u[1];
    o[3] = s * u[2];
  }
  reinterpret_cast<typename Vec4<R>::T*>(Renv)[row] = Vec4<R>::make(o[0], o[1], o[2], o[3]);
}

// ---- first embedding layer (1 -> w1), all nets in one launch --------------------------------
template <class R>
__global__ void k_emb_first(PathConst pc, NetPtrs<R> nets, const int* __restrict__ atom_type_sorted,
                            const R* __restrict__ Renv, int w1, int skip, R* __restrict__ Y, R* __restrict__ T) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long nrow = (long)pc.natoms * pc.nc;
  if (e >= nrow * w1) return;
  const long row = e / w1;
  const int o = (int)(e % w1);
  const int p = (int)(row / pc.nc), k = (int)(row % pc.nc);
  const int net = net_of(pc, atom_type_sorted[p], slot_block(pc, k));
  const R s = Renv[row * 4];
  // a zero row (padding; or, in FP32, s rounded to zero within ~1e-15 of r_c) is read by nobody:
  // the layers above skip it, and so do the contraction, its reverse and the force kernel
  if (s == R(0)) return;
  const R t = tanh_r(s * nets.w0[net][o] + nets.b0[net][o]);
  R y = t;
  if (skip) y += s;  // n_in = 1: both +x and +{x,x} add the scalar input
  Y[e] = y;
  T[e] = t;
}

template <class R>
__global__ void k_emb_first_bwd(PathConst pc, NetPtrs<R> nets, const int* __restrict__ atom_type_sorted,
                                const R* __restrict__ Renv, const R* __restrict__ GY, const R* __restrict__ T,
                                int w1, int skip, R* __restrict__ gs) {
  const long row = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= (long)pc.natoms * pc.nc) return;
  if (Renv[row * 4] == R(0)) return;  // a zero row: no layer outputs, not read by the force kernel
  const int p = (int)(row / pc.nc), k = (int)(row % pc.nc);
  const int net = net_of(pc, atom_type_sorted[p], slot_block(pc, k));
  const R* w = nets.w0[net];
  R acc = R(0);
  for (int o = 0; o < w1; ++o) {
    const R g = GY[row * w1 + o];
    const R t = T[row * w1 + o];
    acc += g * (R(1) - t * t) * w[o];
    if (skip) acc += g;
  }
  gs[row] = acc;
}

// End of each type block's leading nonzero environment rows of atom row rb (one warp): a block's
// listed pairs come nearest first and s falls with r, so its zero rows (padding, pairs beyond this
// part's cutoff, s rounded to zero just inside it) close the block.
template <class R>
__device__ __forceinline__ void block_ends(const PathConst& pc, const R* __restrict__ Renv, long rb, int* ends) {
  const int lane = threadIdx.x & 31;
  for (int t = 0; t < pc.ntypes; ++t) {
    int end = pc.sel_off[t + 1];
    for (int k0 = pc.sel_off[t]; k0 < pc.sel_off[t + 1]; k0 += 32) {
      const int k = k0 + lane;
      const unsigned zm = __ballot_sync(0xffffffffu, k < pc.sel_off[t + 1] && Renv[(rb + k) * 4] == R(0));
      if (zm) {
        end = k0 + __ffs(zm) - 1;
        break;
      }
    }
    if (lane == 0) ends[t] = end;
  }
}

// ---- T = G^T R / Nc and D = T T_<^T, one block per atom -------------------------------------
template <class R>
__global__ void k_contract(PathConst pc, const R* __restrict__ G, const R* __restrict__ Renv, R* __restrict__ Tm,
                           R* __restrict__ D) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  R* Ts = reinterpret_cast<R*>(sm_raw);  // [M][4]
  __shared__ int s_end[DP_MAX_TYPES];
  const int p = blockIdx.x;
  const int M = pc.M, A = pc.A, nc = pc.nc;
  const R inv_nc = R(1) / R(nc);
  const long rb = (long)p * nc;
  if (threadIdx.x < 32) block_ends<R>(pc, Renv, rb, s_end);  // zero rows add exact zeros; their G is not computed
  __syncthreads();
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    R a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    for (int t = 0; t < pc.ntypes; ++t)
    for (int k = pc.sel_off[t]; k < s_end[t]; ++k) {
      const R g = G[(rb + k) * M + m];
      const typename Vec4<R>::T r4 = reinterpret_cast<const typename Vec4<R>::T*>(Renv)[rb + k];
      a0 += g * r4.x;
      a1 += g * r4.y;
      a2 += g * r4.z;
      a3 += g * r4.w;
    }
    a0 *= inv_nc;
    a1 *= inv_nc;
    a2 *= inv_nc;
    a3 *= inv_nc;
    Ts[m * 4 + 0] = a0;
    Ts[m * 4 + 1] = a1;
    Ts[m * 4 + 2] = a2;
    Ts[m * 4 + 3] = a3;
    reinterpret_cast<typename Vec4<R>::T*>(Tm)[(long)p * M + m] = Vec4<R>::make(a0, a1, a2, a3);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < M * A; idx += blockDim.x) {
    const int m = idx / A, l = idx % A;
    D[(long)p * pc.Dw + pc.doff + idx] =
        Ts[m * 4] * Ts[l * 4] + Ts[m * 4 + 1] * Ts[l * 4 + 1] + Ts[m * 4 + 2] * Ts[l * 4 + 2] + Ts[m * 4 + 3] * Ts[l * 4 + 3];
  }
}

// ---- dE/dT from dE/dD, then dE/dG (rows) and dE/dR (rows), one block per atom ----------------
template <class R>
__global__ void k_descr_bwd(PathConst pc, const R* __restrict__ Tm, const R* __restrict__ gD,
                            const R* __restrict__ G, const R* __restrict__ Renv, R* __restrict__ gG,
                            R* __restrict__ gR) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int M = pc.M, A = pc.A, nc = pc.nc;
  R* Ts = reinterpret_cast<R*>(sm_raw);  // [M][4]
  R* gTs = Ts + M * 4;                   // [M][4]
  R* gDs = gTs + M * 4;                  // [M][A]
  const int p = blockIdx.x;
  for (int e = threadIdx.x; e < M * 4; e += blockDim.x) Ts[e] = Tm[(long)p * M * 4 + e];
  for (int e = threadIdx.x; e < M * A; e += blockDim.x) gDs[e] = gD[(long)p * pc.Dw + pc.doff + e];
  __syncthreads();
  for (int e = threadIdx.x; e < M * 4; e += blockDim.x) {
    const int m = e / 4, c = e % 4;
    R acc = 0;
    for (int l = 0; l < A; ++l) acc += gDs[m * A + l] * Ts[l * 4 + c];
    if (m < A)
      for (int q = 0; q < M; ++q) acc += gDs[q * A + m] * Ts[q * 4 + c];
    gTs[e] = acc;
  }
  __syncthreads();
  const R inv_nc = R(1) / R(nc);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int k = warp; k < nc; k += nw) {
    const long row = (long)p * nc + k;
    const typename Vec4<R>::T r4 = reinterpret_cast<const typename Vec4<R>::T*>(Renv)[row];
    if (r4.x == R(0)) continue;  // warp-uniform: a zero row is read by nobody downstream
    R a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    for (int m = lane; m < M; m += 32) {
      const R g = G[row * M + m];
      a0 += gTs[m * 4] * g;
      a1 += gTs[m * 4 + 1] * g;
      a2 += gTs[m * 4 + 2] * g;
      a3 += gTs[m * 4 + 3] * g;
      gG[row * M + m] =
          (gTs[m * 4] * r4.x + gTs[m * 4 + 1] * r4.y + gTs[m * 4 + 2] * r4.z + gTs[m * 4 + 3] * r4.w) * inv_nc;
    }
    for (int off = 16; off > 0; off >>= 1) {
      a0 += __shfl_xor_sync(0xffffffffu, a0, off);
      a1 += __shfl_xor_sync(0xffffffffu, a1, off);
      a2 += __shfl_xor_sync(0xffffffffu, a2, off);
      a3 += __shfl_xor_sync(0xffffffffu, a3, off);
    }
    if (lane == 0)
      reinterpret_cast<typename Vec4<R>::T*>(gR)[row] = Vec4<R>::make(a0 * inv_nc, a1 * inv_nc, a2 * inv_nc, a3 * inv_nc);
  }
}

// ---- se_e2_r block: D_r[m] = (1/Nc) sum_k G_r[k][m] s_k, one block per atom -------------------
// G rows hold M values; D_r goes to the part's block of D (row stride Dw).
template <class R>
__global__ void k_contract_r(PathConst pc, const R* __restrict__ G, const R* __restrict__ Renv, R* __restrict__ D) {
  __shared__ int s_end[DP_MAX_TYPES];
  const int p = blockIdx.x;
  const int M = pc.M, nc = pc.nc;
  const long rb = (long)p * nc;
  if (threadIdx.x < 32) block_ends<R>(pc, Renv, rb, s_end);  // zero rows add exact zeros; their G is not computed
  __syncthreads();
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    R acc = 0;
    for (int t = 0; t < pc.ntypes; ++t)
      for (int k = pc.sel_off[t]; k < s_end[t]; ++k) acc += G[(rb + k) * M + m] * Renv[(rb + k) * 4];
    D[(long)p * pc.Dw + pc.doff + m] = acc / R(nc);
  }
}

// Reverse of k_contract_r: dE/dG_r[k][m] = gD_r[m] s_k / Nc into gG, and the direct term
// dE/ds_k = sum_m gD_r[m] G_r[k][m] / Nc as the radial component of gR (the other three zero).
// One block per atom, a warp per row.
template <class R>
__global__ void k_descr_bwd_r(PathConst pc, const R* __restrict__ gD, const R* __restrict__ G,
                              const R* __restrict__ Renv, R* __restrict__ gG, R* __restrict__ gR) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  R* gDs = reinterpret_cast<R*>(sm_raw);  // [M]
  const int p = blockIdx.x;
  const int M = pc.M, nc = pc.nc;
  for (int e = threadIdx.x; e < M; e += blockDim.x) gDs[e] = gD[(long)p * pc.Dw + pc.doff + e];
  __syncthreads();
  const R inv_nc = R(1) / R(nc);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int k = warp; k < nc; k += nw) {
    const long row = (long)p * nc + k;
    const R s = Renv[row * 4];
    if (s == R(0)) continue;  // warp-uniform: a zero row is read by nobody downstream
    R acc = 0;
    for (int m = lane; m < M; m += 32) {
      acc += gDs[m] * G[row * M + m];
      gG[row * M + m] = gDs[m] * s * inv_nc;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) reinterpret_cast<typename Vec4<R>::T*>(gR)[row] = Vec4<R>::make(acc * inv_nc, R(0), R(0), R(0));
  }
}

// ---- compressed se_e2_r part (Eq. (compress)): G_k from the pieces in s, folded into D_r on the
// fly (operator merging: G never reaches memory); one block per atom, a thread per output m.
template <class R>
__global__ void k_rtab_fwd(PathConst pc, const R* __restrict__ tab, TabConst tc, const int* __restrict__ tsorted,
                           const R* __restrict__ Renv, R* __restrict__ D, int* __restrict__ range_flag) {
  const int p = blockIdx.x;
  const int M = pc.M, nc = pc.nc, ti = tsorted[p];
  const long rb = (long)p * nc;
  bool oor = false;
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    R acc = 0;
    for (int k = 0; k < nc; ++k) {
      const R s = Renv[(rb + k) * 4];
      if (s == R(0)) continue;  // padding (or beyond this part's cutoff)
      R tt;
      const int l = tab_interval<R>(tc, s, tt, oor);
      const int net = net_of(pc, ti, slot_block(pc, k));
      const Quint<R> q = load_quint(tab + ((((long)net * tc.lc + l) * M) + m) * kCoefStride);
      acc += quint_value(q, tt) * s;
    }
    D[(long)p * pc.Dw + pc.doff + m] = acc / R(nc);
  }
  if (oor && range_flag) atomicOr(range_flag, 1);
}

// Its reverse: dE/ds_k = (1/Nc) sum_m gD_m (G_m'(s_k) s_k + G_m(s_k)) into the radial component of
// gR (the other three zero); one block per atom, a warp per row, lanes over m.
template <class R>
__global__ void k_rtab_bwd(PathConst pc, const R* __restrict__ tab, TabConst tc, const int* __restrict__ tsorted,
                           const R* __restrict__ Renv, const R* __restrict__ gD, R* __restrict__ gR) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  R* gDs = reinterpret_cast<R*>(sm_raw);  // [M]
  const int p = blockIdx.x;
  const int M = pc.M, nc = pc.nc, ti = tsorted[p];
  for (int e = threadIdx.x; e < M; e += blockDim.x) gDs[e] = gD[(long)p * pc.Dw + pc.doff + e];
  __syncthreads();
  const R inv_nc = R(1) / R(nc);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  bool oor = false;
  for (int k = warp; k < nc; k += nw) {
    const long row = (long)p * nc + k;
    const R s = Renv[row * 4];
    R acc = 0;
    if (s != R(0)) {
      R tt;
      const int l = tab_interval<R>(tc, s, tt, oor);
      const int net = net_of(pc, ti, slot_block(pc, k));
      const R* base = tab + (((long)net * tc.lc + l) * M) * kCoefStride;
      for (int m = lane; m < M; m += 32) {
        const Quint<R> q = load_quint(base + (long)m * kCoefStride);
        acc += gDs[m] * (quint_slope(q, tt) * s + quint_value(q, tt));
      }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) reinterpret_cast<typename Vec4<R>::T*>(gR)[row] = Vec4<R>::make(acc * inv_nc, R(0), R(0), R(0));
  }
}

// ---- se_e3 part: fused pair kernel, one block per atom -------------------------------------------
// Over the pairs (j, k) of the atom's real neighbours (rows with s > 0), theta = R_j . R_k and
// G = N^{a_j,a_k}(theta), with dG/dtheta carried forward alongside (the nets have a scalar input):
//   forward   D_m = (1/Nc^2) sum_jk theta G_m
//   backward  dE/dtheta_jk = (1/Nc^2) sum_m gD_m (G_m + theta G'_m),
//             dE/dR_j += dE/dtheta_jk R_k,  dE/dR_k += dE/dtheta_jk R_j
// Nothing of G is stored: the backward pass evaluates the nets again.  All of the part's nets sit
// in shared memory; a warp takes rows j, its lanes the partners k (below).
struct E3Net {
  int nl;
  int in[DP_MAX_LAYERS], out[DP_MAX_LAYERS], skip[DP_MAX_LAYERS];
  int loff[DP_MAX_LAYERS];  // offset of layer l's W inside one net (b follows W)
  int per_net;              // parameters per net
};

// Any net of widths <= W: the parameters in shared memory in their own layout, every layer a
// W x W loop with the shapes as run-time bounds.
template <class R, int W>
struct E3Any {
  static constexpr int kM = W;
  static constexpr bool kItemBwd = true;  // backward over the warp's item stream (evaluation-bound)
  E3Net nt;
  __device__ int per_net() const { return nt.per_net; }
  __device__ void fill(R* wsm, const R* __restrict__ params, int n_nets, int tid, int nth) const {
    for (long e = tid; e < (long)n_nets * nt.per_net; e += nth) wsm[e] = params[e];
  }
  template <bool DERIV>
  __device__ __forceinline__ void eval(const R* __restrict__ wsm, int net, R th, R* g, R* dg, bool&) const {
    const R* w = wsm + (long)net * nt.per_net;
    R x[W], dx[W];
#pragma unroll
    for (int o = 0; o < W; ++o) {
      x[o] = R(0);
      dx[o] = R(0);
    }
    x[0] = th;
    dx[0] = R(1);
    for (int l = 0; l < nt.nl; ++l) {
      const int ni = nt.in[l], no = nt.out[l], sk = nt.skip[l];
      const R* Wl = w + nt.loff[l];
      const R* bl = Wl + ni * no;
      R y[W], dy[W];
#pragma unroll
      for (int o = 0; o < W; ++o) {
        if (o < no) {
          R z = bl[o], dz = R(0);
#pragma unroll
          for (int i = 0; i < W; ++i)
            if (i < ni) {
              const R wv = Wl[i * no + o];
              z += x[i] * wv;
              if (DERIV) dz += dx[i] * wv;
            }
          const R t = tanh_r(z);
          R yo = t, dyo = DERIV ? (R(1) - t * t) * dz : R(0);
          if (sk == 1) {
            yo += x[o];
            if (DERIV) dyo += dx[o];
          } else if (sk == 2) {
            const int q = o < ni ? o : o - ni;  // {x, x}: n_out = 2 n_in
            R xq = R(0), dxq = R(0);
#pragma unroll
            for (int i = 0; i < W; ++i)  // a select chain keeps x in registers
              if (i == q) {
                xq = x[i];
                dxq = dx[i];
              }
            yo += xq;
            if (DERIV) dyo += dxq;
          }
          y[o] = yo;
          dy[o] = dyo;
        } else {
          y[o] = R(0);
          dy[o] = R(0);
        }
      }
#pragma unroll
      for (int o = 0; o < W; ++o) {
        x[o] = y[o];
        dx[o] = dy[o];
      }
    }
#pragma unroll
    for (int o = 0; o < W; ++o) {
      g[o] = x[o];
      dg[o] = dx[o];
    }
  }
};

// Three layers of widths A, B, C known at compile time (the paper's se_e3 nets are 2/4/8): every
// loop unrolled without bounds, skip kinds fixed, and each net's rows padded to multiples of four
// values in shared memory so that a row loads as 16-byte vectors.
template <class R, int A, int B, int C>
struct E3Fixed {
  static constexpr int kM = C;
  static constexpr bool kItemBwd = true;
  static constexpr int PA = (A + 3) / 4 * 4, PB = (B + 3) / 4 * 4, PC = (C + 3) / 4 * 4;
  // padded layout of one net: w0 [PA], b0 [PA], W1 [A][PB], b1 [PB], W2 [B][PC], b2 [PC]
  static constexpr int OW0 = 0, OB0 = PA, OW1 = 2 * PA, OB1 = OW1 + A * PB, OW2 = OB1 + PB, OB2 = OW2 + B * PC;
  static constexpr int PN = OB2 + PC;
  static constexpr int SK0 = (A == 1) ? 1 : (A == 2 ? 2 : 0);
  static constexpr int SK1 = (B == A) ? 1 : (B == 2 * A ? 2 : 0);
  static constexpr int SK2 = (C == B) ? 1 : (C == 2 * B ? 2 : 0);
  int per_net_global;  // parameters of one net in the global layout
  __device__ int per_net() const { return PN; }
  __device__ void fill(R* wsm, const R* __restrict__ params, int n_nets, int tid, int nth) const {
    for (int e = tid; e < n_nets * PN; e += nth) {
      const int n = e / PN, q = e % PN;
      const R* src = params + (long)n * per_net_global;  // global: W0 [1][A] b0 [A] W1 [A][B] b1 [B] W2 [B][C] b2 [C]
      R v = R(0);
      if (q < OB0) {
        if (q < A) v = src[q];
      } else if (q < OW1) {
        if (q - OB0 < A) v = src[A + (q - OB0)];
      } else if (q < OB1) {
        const int i = (q - OW1) / PB, o = (q - OW1) % PB;
        if (o < B) v = src[2 * A + i * B + o];
      } else if (q < OW2) {
        if (q - OB1 < B) v = src[2 * A + A * B + (q - OB1)];
      } else if (q < OB2) {
        const int i = (q - OW2) / PC, o = (q - OW2) % PC;
        if (o < C) v = src[2 * A + A * B + B + i * C + o];
      } else {
        if (q - OB2 < C) v = src[2 * A + A * B + B + B * C + (q - OB2)];
      }
      wsm[e] = v;
    }
  }
  template <int P>
  static __device__ __forceinline__ void ldrow(const R* __restrict__ p, R* v) {
    if constexpr (sizeof(R) == 4) {
#pragma unroll
      for (int c = 0; c < P / 4; ++c) {
        const float4 f = reinterpret_cast<const float4*>(p)[c];
        v[4 * c] = f.x;
        v[4 * c + 1] = f.y;
        v[4 * c + 2] = f.z;
        v[4 * c + 3] = f.w;
      }
    } else {
#pragma unroll
      for (int c = 0; c < P / 2; ++c) {
        const double2 f = reinterpret_cast<const double2*>(p)[c];
        v[2 * c] = f.x;
        v[2 * c + 1] = f.y;
      }
    }
  }
  template <bool DERIV>
  __device__ __forceinline__ void eval(const R* __restrict__ wsm, int net, R th, R* g, R* dg, bool&) const {
    const R* w = wsm + net * PN;
    R x0[A], d0[A], x1[B], d1[B];
    {
      R wv[PA], bv[PA];
      ldrow<PA>(w + OW0, wv);
      ldrow<PA>(w + OB0, bv);
#pragma unroll
      for (int o = 0; o < A; ++o) {
        const R t = tanh_r(th * wv[o] + bv[o]);
        x0[o] = t + (SK0 ? th : R(0));
        if (DERIV) d0[o] = (R(1) - t * t) * wv[o] + (SK0 ? R(1) : R(0));
      }
    }
    {
      R z[PB], dz[PB];
      ldrow<PB>(w + OB1, z);
#pragma unroll
      for (int o = 0; o < B; ++o) dz[o] = R(0);
#pragma unroll
      for (int i = 0; i < A; ++i) {
        R wr[PB];
        ldrow<PB>(w + OW1 + i * PB, wr);
#pragma unroll
        for (int o = 0; o < B; ++o) {
          z[o] += x0[i] * wr[o];
          if (DERIV) dz[o] += d0[i] * wr[o];
        }
      }
#pragma unroll
      for (int o = 0; o < B; ++o) {
        const R t = tanh_r(z[o]);
        const int q = SK1 == 2 ? o % A : o;
        x1[o] = t + (SK1 ? x0[q] : R(0));
        if (DERIV) d1[o] = (R(1) - t * t) * dz[o] + (SK1 ? d0[q] : R(0));
      }
    }
    {
      R z[PC], dz[PC];
      ldrow<PC>(w + OB2, z);
#pragma unroll
      for (int o = 0; o < C; ++o) dz[o] = R(0);
#pragma unroll
      for (int i = 0; i < B; ++i) {
        R wr[PC];
        ldrow<PC>(w + OW2 + i * PC, wr);
#pragma unroll
        for (int o = 0; o < C; ++o) {
          z[o] += x1[i] * wr[o];
          if (DERIV) dz[o] += d1[i] * wr[o];
        }
      }
#pragma unroll
      for (int o = 0; o < C; ++o) {
        const R t = tanh_r(z[o]);
        const int q = SK2 == 2 ? o % B : o;
        g[o] = t + (SK2 ? x1[q] : R(0));
        if (DERIV) dg[o] = (R(1) - t * t) * dz[o] + (SK2 ? d1[q] : R(0));
      }
    }
  }
};

// Compressed nets (Eq. (compress)): G and dG/dtheta from the quintic pieces in theta of each net;
// the M <= MW outputs' coefficients are read through the L1 cache (the tables stay in L2).
template <class R, int MW>
struct E3Tab {
  static constexpr int kM = MW;
  // backward a warp per row: the table pieces are L1 loads, whose latencies the lanes overlap best
  // without a warp-wide step per item
  static constexpr bool kItemBwd = false;
  const R* tab;  // [net][interval][M][kCoefStride]
  TabConst tc;
  int M;
  __device__ int per_net() const { return 0; }
  __device__ void fill(R*, const R* __restrict__, int, int, int) const {}
  template <bool DERIV>
  __device__ __forceinline__ void eval(const R* __restrict__, int net, R th, R* g, R* dg, bool& oor) const {
    R tt;
    const int l = tab_interval<R>(tc, th, tt, oor);
    const R* row = tab + (((long)net * tc.lc + l) * M) * kCoefStride;
#pragma unroll
    for (int m = 0; m < MW; ++m) {
      if (m < M) {
        const Quint<R> q = load_quint(row + (long)m * kCoefStride);
        g[m] = quint_value(q, tt);
        dg[m] = DERIV ? quint_slope(q, tt) : R(0);
      } else {
        g[m] = R(0);
        dg[m] = R(0);
      }
    }
  }
};

constexpr int kE3Warps = 4;  // warps per CTA of the se_e3 pair kernel

// BWD = 0: D block; BWD = 1: dE/dR rows (gR, [rows][4], every row of the atom written).
template <class R, class Ev, int BWD>
__global__ void __launch_bounds__(kE3Warps * 32)
    k_e3(PathConst pc, Ev ev, const R* __restrict__ params, int n_nets, const R* __restrict__ Renv,
         const R* __restrict__ gD, R* __restrict__ D, R* __restrict__ gR, int* __restrict__ range_flag) {
  constexpr int W = Ev::kM;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  typedef typename Vec4<R>::T V4;
  const int nc = pc.nc, M = pc.M, nt_types = pc.ntypes;
  const int pn = ev.per_net();
  V4* Rv = reinterpret_cast<V4*>(sm_raw);     // [nc] rows of the real neighbours, compacted
  V4* gRv = Rv + nc;                          // [nc] dE/dR of those rows (backward)
  R* wsm = reinterpret_cast<R*>(gRv + nc);    // [n_nets * per_net]
  R* red = wsm + (long)n_nets * pn;           // [W] D sums / gD
  int* tv = reinterpret_cast<int*>(red + W);  // [nc] neighbour type of each compacted row
  int* kv = tv + nc;                          // [nc] slot of each compacted row
  __shared__ int nv_s;
  __shared__ int tstart_s[DP_MAX_TYPES + 1];  // first compacted row of each neighbour type
  const int p = blockIdx.x;
  const long rb = (long)p * nc;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  ev.fill(wsm, params, n_nets, tid, blockDim.x);
  if (tid < W) red[tid] = (BWD && tid < M) ? gD[(long)p * pc.Dw + pc.doff + tid] : R(0);
  if (warp == 0) {  // compaction of the rows with s > 0, in slot order
    int nv = 0;
    for (int base = 0; base < nc; base += 32) {
      const int k = base + lane;
      const bool v = k < nc && Renv[(rb + k) * 4] != R(0);
      const unsigned mask = __ballot_sync(0xffffffffu, v);
      if (v) {
        const int at = nv + __popc(mask & ((1u << lane) - 1u));
        Rv[at] = reinterpret_cast<const V4*>(Renv)[rb + k];
        tv[at] = slot_block(pc, k);
        kv[at] = k;
      }
      nv += __popc(mask);
    }
    if (lane == 0) nv_s = nv;
    __syncwarp();
    if (lane <= nt_types) {  // the compacted rows keep the slot order, so their types never decrease
      int lo = 0, hi = nv;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (tv[mid] < lane) lo = mid + 1; else hi = mid;
      }
      tstart_s[lane] = lo;
    }
  }
  __syncthreads();
  const int nv = nv_s;
  if (BWD)
    for (int e = tid; e < nv; e += blockDim.x) gRv[e] = Vec4<R>::make(R(0), R(0), R(0), R(0));
  __syncthreads();
  const R inv = R(1) / (R(nc) * R(nc));
  bool oor = false;
  R acc[W];
#pragma unroll
  for (int m = 0; m < W; ++m) acc[m] = R(0);
  // theta_jk = theta_kj, and a pair of neighbours of one type takes one net both ways: such a pair
  // is evaluated once, from its lower row, with weight 2 (the diagonal j = k once, weight 1).  Row j
  // pairs with every row k outside its type block and with the rows of its own type from j on:
  // nv - (j - b0) partners, partner q at k = q below the block start b0, else q + (j - b0).
  if (!BWD) {
    // forward: warp w's rows w, w + nw, ... as one stream of (row, partner) items, so that a lane
    // moves on to the next row without waiting for the others (the sums go to D, not to the rows)
    int jr = warp, rbeg = 0, rlen = 0, b0 = 0, tj = 0;
    V4 rj = Vec4<R>::make(R(0), R(0), R(0), R(0));
    auto open_row = [&]() {
      if (jr < nv) {
        rj = Rv[jr];
        tj = tv[jr];
        b0 = tstart_s[tj];
        rlen = nv - (jr - b0);
      }
    };
    open_row();
    for (int t = lane;; t += 32) {
      while (jr < nv && t >= rbeg + rlen) {
        rbeg += rlen;
        jr += nw;
        open_row();
      }
      if (jr >= nv) break;
      const int q = t - rbeg;
      const int k = q < b0 ? q : q + (jr - b0);
      const V4 rk = Rv[k];
      const int tk = tv[k];
      const R th = ((rj.x * rk.x + rj.y * rk.y) + rj.z * rk.z) + rj.w * rk.w;
      R g[W], dg[W];
      ev.template eval<false>(wsm, tj * nt_types + tk, th, g, dg, oor);
      const R wth = ((tk == tj && k != jr) ? R(2) : R(1)) * th;
#pragma unroll
      for (int m = 0; m < W; ++m) acc[m] += wth * g[m];
    }
  } else if (!Ev::kItemBwd) {
    // backward, a warp per row: its own term summed over the lanes
    for (int j = warp; j < nv; j += nw) {
      const V4 rj = Rv[j];
      const int tj = tv[j];
      const int b0 = tstart_s[tj], skip = j - b0;
      R gj0 = 0, gj1 = 0, gj2 = 0, gj3 = 0;
      for (int q = lane; q < nv - skip; q += 32) {
        const int k = q < b0 ? q : q + skip;
        const V4 rk = Rv[k];
        const int tk = tv[k];
        const R th = ((rj.x * rk.x + rj.y * rk.y) + rj.z * rk.z) + rj.w * rk.w;
        R g[W], dg[W];
        ev.template eval<true>(wsm, tj * nt_types + tk, th, g, dg, oor);
        R gth = 0;
#pragma unroll
        for (int m = 0; m < W; ++m) gth += red[m] * (g[m] + th * dg[m]);
        gth *= inv * ((tk == tj && k != j) ? R(2) : R(1));
        gj0 += gth * rk.x;
        gj1 += gth * rk.y;
        gj2 += gth * rk.z;
        gj3 += gth * rk.w;
        atomicAdd(&gRv[k].x, gth * rj.x);
        atomicAdd(&gRv[k].y, gth * rj.y);
        atomicAdd(&gRv[k].z, gth * rj.z);
        atomicAdd(&gRv[k].w, gth * rj.w);
      }
      for (int o = 16; o > 0; o >>= 1) {
        gj0 += __shfl_xor_sync(0xffffffffu, gj0, o);
        gj1 += __shfl_xor_sync(0xffffffffu, gj1, o);
        gj2 += __shfl_xor_sync(0xffffffffu, gj2, o);
        gj3 += __shfl_xor_sync(0xffffffffu, gj3, o);
      }
      if (lane == 0) {
        atomicAdd(&gRv[j].x, gj0);
        atomicAdd(&gRv[j].y, gj1);
        atomicAdd(&gRv[j].z, gj2);
        atomicAdd(&gRv[j].w, gj3);
      }
    }
  } else {
    // backward: the same item streams.  Row j's own term (sum over partners of dE/dtheta R_k) is
    // summed per lane while the lane is in the row; a lane leaving a row of 32 or more items (every
    // lane has items there) parks its sum in a slot of part[] chosen by the parity of the long rows
    // passed, and once lane 0 -- the last lane out of any row -- has left it, the warp adds the 32
    // sums; a lane leaving a shorter row adds its sum itself.  A lane cannot leave the next long row
    // but one before lane 0 has left this one, so two slots suffice.
    __shared__ V4 part[2][kE3Warps][32];
    int jr = warp, rbeg = 0, rlen = 0, b0 = 0, tj = 0;
    V4 rj = Vec4<R>::make(R(0), R(0), R(0), R(0));
    auto open_row = [&]() {
      if (jr < nv) {
        rj = Rv[jr];
        tj = tv[jr];
        b0 = tstart_s[tj];
        rlen = nv - (jr - b0);
      }
    };
    open_row();
    R gj0 = 0, gj1 = 0, gj2 = 0, gj3 = 0;
    int nlong = 0, done = 0;  // long rows this lane has left; long rows the warp has added
    int lrow0 = 0, lrow1 = 0;  // row index of the long rows in slots 0 and 1
    for (int t = lane;; t += 32) {
      while (jr < nv && t >= rbeg + rlen) {  // leaving row jr
        if (rlen >= 32) {
          part[nlong & 1][warp][lane] = Vec4<R>::make(gj0, gj1, gj2, gj3);
          if (nlong & 1) lrow1 = jr; else lrow0 = jr;
          ++nlong;
        } else if (gj0 != R(0) || gj1 != R(0) || gj2 != R(0) || gj3 != R(0)) {
          atomicAdd(&gRv[jr].x, gj0);
          atomicAdd(&gRv[jr].y, gj1);
          atomicAdd(&gRv[jr].z, gj2);
          atomicAdd(&gRv[jr].w, gj3);
        }
        gj0 = gj1 = gj2 = gj3 = R(0);
        rbeg += rlen;
        jr += nw;
        open_row();
      }
      __syncwarp();
      if (__shfl_sync(0xffffffffu, nlong, 0) > done) {  // lane 0 left long row number done
        const V4 v = part[done & 1][warp][lane];
        R x = v.x, y = v.y, z = v.z, w = v.w;
        for (int o = 16; o > 0; o >>= 1) {
          x += __shfl_xor_sync(0xffffffffu, x, o);
          y += __shfl_xor_sync(0xffffffffu, y, o);
          z += __shfl_xor_sync(0xffffffffu, z, o);
          w += __shfl_xor_sync(0xffffffffu, w, o);
        }
        if (lane == 0) {
          const int jd = (done & 1) ? lrow1 : lrow0;
          atomicAdd(&gRv[jd].x, x);
          atomicAdd(&gRv[jd].y, y);
          atomicAdd(&gRv[jd].z, z);
          atomicAdd(&gRv[jd].w, w);
        }
        ++done;
        __syncwarp();
      }
      if (__all_sync(0xffffffffu, jr >= nv)) break;
      if (jr < nv) {
        const int q = t - rbeg;
        const int k = q < b0 ? q : q + (jr - b0);
        const V4 rk = Rv[k];
        const int tk = tv[k];
        const R th = ((rj.x * rk.x + rj.y * rk.y) + rj.z * rk.z) + rj.w * rk.w;
        R g[W], dg[W];
        ev.template eval<true>(wsm, tj * nt_types + tk, th, g, dg, oor);
        R gth = 0;
#pragma unroll
        for (int m = 0; m < W; ++m) gth += red[m] * (g[m] + th * dg[m]);
        gth *= inv * ((tk == tj && k != jr) ? R(2) : R(1));
        gj0 += gth * rk.x;
        gj1 += gth * rk.y;
        gj2 += gth * rk.z;
        gj3 += gth * rk.w;
        atomicAdd(&gRv[k].x, gth * rj.x);
        atomicAdd(&gRv[k].y, gth * rj.y);
        atomicAdd(&gRv[k].z, gth * rj.z);
        atomicAdd(&gRv[k].w, gth * rj.w);
      }
    }
  }
  __syncwarp();
  if (oor && range_flag) atomicOr(range_flag, 1);
  if (!BWD) {
#pragma unroll
    for (int m = 0; m < W; ++m) {
      R v = acc[m];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0 && m < M) atomicAdd(&red[m], v);
    }
    __syncthreads();
    if (tid < M) D[(long)p * pc.Dw + pc.doff + tid] = red[tid] * inv;
  } else {
    __syncthreads();
    V4* out = reinterpret_cast<V4*>(gR) + rb;
    for (int k = tid; k < nc; k += blockDim.x) out[k] = Vec4<R>::make(R(0), R(0), R(0), R(0));
    __syncthreads();
    for (int e = tid; e < nv; e += blockDim.x) out[kv[e]] = gRv[e];
  }
}

// ---- dE/dr_ij, force scatter and per-block virial partials -----------------------------------
template <class R>
__global__ void __launch_bounds__(256)
    k_force(PathConst pc, const double* __restrict__ coord, const int* __restrict__ perm,
            const int* __restrict__ nl_j, const int* __restrict__ nl_code, const R* __restrict__ gs_emb,
            const R* __restrict__ gR, double* __restrict__ force, double* __restrict__ avir) {
  const long row = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (row < (long)pc.natoms * pc.nc) {
    const int p = (int)(row / pc.nc), k = (int)(row % pc.nc);
    const int i = perm[p];
    const long ls = (long)i * pc.lnc + list_slot(pc, k);
    const int j = nl_j[ls];
    double d[3] = {0.0, 0.0, 0.0}, r2 = 0.0;
    if (j >= 0) {
      listed_disp(coord + 3 * i, coord + 3 * j, nl_code[ls], pc, frame_of(pc, i), d[0], d[1], d[2]);
      r2 = norm2_exact(d[0], d[1], d[2]);
    }
    if (j >= 0 && r2 < pc.rc2) {
      R r, s, ds, u[3];
      pair_env<R>(d[0], d[1], d[2], r2, pc.rs, pc.rc, pc.near2, r, s, ds, u);
      // s rounded to zero (FP32, within ~1e-15 of r_c): its rows were not written, and its force
      // terms (s = 0, |ds/dr| below 1e-29) are zero
      if (s == R(0)) return;
      const typename Vec4<R>::T g4 = reinterpret_cast<const typename Vec4<R>::T*>(gR)[row];
      const R gvu = g4.y * u[0] + g4.z * u[1] + g4.w * u[2];
      const R gsum = (gs_emb ? gs_emb[row] : R(0)) + g4.x + gvu;
      const R a = ds * gsum, b = s / r;
      const R gv[3] = {g4.y, g4.z, g4.w};
      double gd[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) gd[c] = (double)(a * u[c] + b * (gv[c] - gvu * u[c]));
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        atomicAdd(force + 3 * i + c, gd[c]);
        atomicAdd(force + 3 * j + c, -gd[c]);
      }
#pragma unroll
      for (int aa = 0; aa < 3; ++aa)
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) atomicAdd(avir + 9L * i + aa * 3 + bb, -gd[aa] * d[bb]);
    }
  }
}

// Sum of `n` vectors of width `w` in order (one block) -> out[w]  (virial partials).
// Column sums of an [n][w] FP64 array, one block per column, fixed summation order (the
// FP64 pipe of one SM is narrow on GB300: spread the columns over SMs).
__global__ void k_sum_rows(const double* __restrict__ in, long n, int w, double* __restrict__ out) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  double acc = 0.0;
  for (long r = threadIdx.x; r < n; r += blockDim.x) acc += in[r * w + c];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if (threadIdx.x == 0) out[c] = t;
  }
}

// Per-atom energies as nparts column-block partial sums [nparts][n] (sorted order), added in
// a fixed order and scattered to input order in FP64.
__global__ void k_energy_parts(const float* __restrict__ parts, int nparts, const int* __restrict__ perm, int n,
                               double* __restrict__ atom_e) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  float e = parts[p];
  for (int k = 1; k < nparts; ++k) e += parts[(long)k * n + p];
  atom_e[perm[p]] = (double)e;
}

// Per-atom energies from the sorted order to input order, widened to FP64.
template <class R>
__global__ void k_energy(const R* __restrict__ Esorted, const int* __restrict__ perm, int n,
                         double* __restrict__ atom_e) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) atom_e[perm[p]] = widen(Esorted[p]);
}

// Translation vectors t(n) = n0 h0 + n1 h1 + n2 h2 for n in {-1,0,1}^3, formed exactly as the
// neighbour builder forms them.
__global__ void k_shift_table(PathConst pc, double* __restrict__ out) {
  const int q = threadIdx.x;
  if (q >= 27) return;
  const int n0 = q / 9 - 1, n1 = (q / 3) % 3 - 1, n2 = q % 3 - 1;
  for (int a = 0; a < 3; ++a)
    out[q * 3 + a] = __dadd_rn(__dadd_rn(__dmul_rn((double)n0, pc.h[a]), __dmul_rn((double)n1, pc.h[3 + a])),
                               __dmul_rn((double)n2, pc.h[6 + a]));
}

__global__ void k_sorted_types(const int* __restrict__ type, const int* __restrict__ perm, int n,
                               int* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) out[p] = type[perm[p]];
}

template <class R>
__global__ void k_fill(R* __restrict__ x, long n, R v) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) x[e] = v;
}

inline unsigned nblk(long n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

// =============================================================================================
// Orchestration of one frame on CUDA cores
// =============================================================================================
template <class R>
int run_fitting(const DeviceModel& m, const PathConst& pc, const R* params, const R* D, const PathIO& io, Arena& ar,
                cudaStream_t st, const R** gD_out) {
  const long N = pc.natoms;
  const int nfl = m.n_fit_layers;
  int maxw = pc.Dw;
  for (int l = 0; l < nfl; ++l) maxw = std::max(maxw, m.fit[l].n_out);
  std::vector<R*> Yf(nfl), Tf(nfl);
  for (int l = 0; l < nfl; ++l) {
    Yf[l] = ar.get<R>(N * m.fit[l].n_out);
    Tf[l] = ar.get<R>(N * m.fit[l].n_out);
  }
  R* gA = ar.get<R>(N * maxw);
  R* gB = ar.get<R>(N * maxw);
  if (ar.measure) return DP_OK;
  if (!ar.ok()) {
    set_error("scratch allocation failed");
    return DP_E_OOM;
  }
  for (int t = 0; t < pc.ntypes; ++t) {
    RowMap rm{0, io.type_start[t], 0, 0, 0, 0, io.type_start[t + 1] - io.type_start[t]};
    const R* X = D;
    for (int l = 0; l < nfl; ++l) {
      const LayerDesc& L = m.fit[(size_t)t * nfl + l];
      const R* W = params + L.w_off;
      {
        ProfScope _ps(io.prof, "fit_fwd", st);
        DP_CUDA_TRY(launch_dense_fwd<R>(rm, X, L.n_in, W, W + (long)L.n_in * L.n_out, L.n_out, L.skip, L.tanh_act,
                                        Yf[l], Tf[l], st));
      }
      X = Yf[l];
    }
  }
  {
    ProfScope _ps(io.prof, "energy_sum", st);
    k_energy<R><<<nblk(N, 256), 256, 0, st>>>(Yf[nfl - 1], io.perm, (int)N, io.atom_energy);
  }
  // backward through the fitting net, seeded with dE_i/dE_i = 1
  {
    ProfScope _ps(io.prof, "fill", st);
    k_fill<R><<<nblk(N, 256), 256, 0, st>>>(gA, N, R(1));
  }
  // layer by layer over all types, so both ping-pong buffers always hold one layer's stride
  R* gy = gA;
  R* gx = gB;
  for (int l = nfl - 1; l >= 0; --l) {
    for (int t = 0; t < pc.ntypes; ++t) {
      RowMap rm{0, io.type_start[t], 0, 0, 0, 0, io.type_start[t + 1] - io.type_start[t]};
      const LayerDesc& L = m.fit[(size_t)t * nfl + l];
      ProfScope _ps(io.prof, "fit_bwd", st);
      DP_CUDA_TRY(launch_dense_bwd<R>(rm, gy, L.tanh_act ? Tf[l] : nullptr, L.n_in, params + L.w_off, L.n_out, L.skip,
                                      gx, st));
    }
    std::swap(gy, gx);
  }
  *gD_out = gy;
  return DP_OK;
}

// Per-part scratch of the CUDA-core path.
template <class R>
struct PartBufs {
  PathConst pc;
  R* Renv = nullptr;       // [rows][4]
  std::vector<R*> Y, T;    // two-body parts: per layer outputs and tanh values
  R* Tm = nullptr;         // se_e2_a: [N][M][4]
  R* gR = nullptr;         // [rows][4]
  R* gs = nullptr;         // two-body parts: dE/ds through the nets [rows]
  NetPtrs<R> nets;         // first layers of the part's nets
};

bool e3_supported(const PartDesc& P, int precision) {
  int w = 1;
  for (int l = 0; l < P.nl; ++l) w = std::max(w, P.emb[l].n_out);
  const size_t bytes = (size_t)P.n_nets * P.per_net * (precision == DP_PREC_FP64 ? 8 : 4);
  return w <= 32 && bytes <= 96 * 1024 && P.nc <= 4096;
}

template <class R, class Ev>
cudaError_t launch_e3_ev(const PathConst& pc, const Ev& ev, int per_net_smem, const R* w, int n_nets, const R* Renv,
                         const R* gD, R* D, R* gR, bool bwd, cudaStream_t st, int* range_flag = nullptr) {
  const size_t smem = sizeof(typename Vec4<R>::T) * 2 * pc.nc +
                      sizeof(R) * ((size_t)n_nets * per_net_smem + Ev::kM) + sizeof(int) * 2 * pc.nc;
  auto kf = k_e3<R, Ev, 0>;
  auto kb = k_e3<R, Ev, 1>;
  if (smem > 48 * 1024) {
    cudaError_t e = allow_max_smem(bwd ? kb : kf);
    if (e != cudaSuccess) return e;
  }
  if (bwd)
    kb<<<(unsigned)pc.natoms, kE3Warps * 32, smem, st>>>(pc, ev, w, n_nets, Renv, gD, D, gR, range_flag);
  else
    kf<<<(unsigned)pc.natoms, kE3Warps * 32, smem, st>>>(pc, ev, w, n_nets, Renv, gD, D, gR, range_flag);
  return cudaGetLastError();
}

// se_e3 part with compressed nets: the quintic pieces in theta (tab: the model's FP64 or FP32 copy).
template <class R>
cudaError_t launch_e3_tab(const DeviceModel& m, const PartDesc& P, const PathConst& pc, const R* tab, const R* Renv,
                          const R* gD, R* D, R* gR, bool bwd, int* range_flag, cudaStream_t st) {
  const TabConst tc = tab_const(m);
  if (P.M <= 8)
    return launch_e3_ev<R>(pc, E3Tab<R, 8>{tab, tc, P.M}, 0, nullptr, P.n_nets, Renv, gD, D, gR, bwd, st, range_flag);
  if (P.M <= 16)
    return launch_e3_ev<R>(pc, E3Tab<R, 16>{tab, tc, P.M}, 0, nullptr, P.n_nets, Renv, gD, D, gR, bwd, st, range_flag);
  return launch_e3_ev<R>(pc, E3Tab<R, 32>{tab, tc, P.M}, 0, nullptr, P.n_nets, Renv, gD, D, gR, bwd, st, range_flag);
}

template <class R>
cudaError_t launch_e3(const PartDesc& P, const PathConst& pc, const R* params, const R* Renv, const R* gD, R* D,
                      R* gR, bool bwd, cudaStream_t st) {
  const R* wp = params + P.w_off;
  int w = 1;
  for (int l = 0; l < P.nl; ++l) w = std::max(w, P.emb[l].n_out);
  if (P.nl == 3) {  // the paper's shapes, unrolled
    const int a = P.emb[0].n_out, b = P.emb[1].n_out, c = P.emb[2].n_out;
#define DP_E3_FIXED(A_, B_, C_)                                                                           \
    if (a == A_ && b == B_ && c == C_) {                                                                   \
      E3Fixed<R, A_, B_, C_> ev;                                                                           \
      ev.per_net_global = (int)P.per_net;                                                                  \
      return launch_e3_ev<R>(pc, ev, E3Fixed<R, A_, B_, C_>::PN, wp, P.n_nets, Renv, gD, D, gR, bwd, st); \
    }
    DP_E3_FIXED(2, 4, 8)
    DP_E3_FIXED(4, 8, 16)
    DP_E3_FIXED(8, 16, 32)
#undef DP_E3_FIXED
  }
  E3Net nt;
  std::memset(&nt, 0, sizeof(nt));
  nt.nl = P.nl;
  for (int l = 0; l < P.nl; ++l) {
    const LayerDesc& L = P.emb[l];
    nt.in[l] = L.n_in;
    nt.out[l] = L.n_out;
    nt.skip[l] = L.skip;
    nt.loff[l] = (int)(L.w_off - P.w_off);
  }
  nt.per_net = (int)P.per_net;
  if (w <= 8) return launch_e3_ev<R>(pc, E3Any<R, 8>{nt}, nt.per_net, wp, P.n_nets, Renv, gD, D, gR, bwd, st);
  if (w <= 16) return launch_e3_ev<R>(pc, E3Any<R, 16>{nt}, nt.per_net, wp, P.n_nets, Renv, gD, D, gR, bwd, st);
  return launch_e3_ev<R>(pc, E3Any<R, 32>{nt}, nt.per_net, wp, P.n_nets, Renv, gD, D, gR, bwd, st);
}

// ---- se_e2_r part: fused per-neighbour kernel -------------------------------------------------
// D_m = (1/Nc) sum_k G_m(s_k) s_k over the atom's real neighbours (rows with s > 0) and, in
// reverse, dE/ds_k = (1/Nc) sum_m gD_m (G_m(s_k) + s_k G_m'(s_k)) into the radial component of gR
// (the other three zero).  The nets have a scalar input, as the se_e3 nets do, and run on the same
// evaluators (dG/ds carried forward alongside), all of the part's nets in shared memory: nothing of
// G is stored.  Persistent blocks of four warps, a warp per atom, its lanes over the atom's real
// neighbours, compacted first.
constexpr int kRWarps = 4;  // four warps: the evaluator's registers leave room for three blocks per SM

template <class R, class Ev, int BWD>
__global__ void __launch_bounds__(kRWarps * 32)
    k_rnet(PathConst pc, Ev ev, const R* __restrict__ params, int n_nets, const int* __restrict__ tsorted,
           const R* __restrict__ Renv, const R* __restrict__ gD, R* __restrict__ D, R* __restrict__ gR) {
  constexpr int W = Ev::kM;
  typedef typename Vec4<R>::T V4;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int nc = pc.nc, M = pc.M;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  R* wsm = reinterpret_cast<R*>(sm_raw);                   // [n_nets * per_net]
  R* gdw = wsm + (long)n_nets * ev.per_net() + warp * W;   // [kRWarps][W] the atom's dE/dD block
  int* kw = reinterpret_cast<int*>(wsm + (long)n_nets * ev.per_net() + kRWarps * W) + warp * nc;  // [kRWarps][nc]
  ev.fill(wsm, params, n_nets, threadIdx.x, blockDim.x);
  __syncthreads();
  const R inv_nc = R(1) / R(nc);
  bool oor = false;
  for (long p = (long)blockIdx.x * kRWarps + warp; p < pc.natoms; p += (long)gridDim.x * kRWarps) {  // warp-uniform
    const int ti = tsorted[p];
    const long rb = p * nc;
    int nv = 0;
    for (int base = 0; base < nc; base += 32) {
      const int k = base + lane;
      const bool v = k < nc && Renv[(rb + k) * 4] != R(0);
      const unsigned mask = __ballot_sync(0xffffffffu, v);
      if (v) kw[nv + __popc(mask & ((1u << lane) - 1u))] = k;
      if (BWD && k < nc && !v) reinterpret_cast<V4*>(gR)[rb + k] = Vec4<R>::make(R(0), R(0), R(0), R(0));
      nv += __popc(mask);
    }
    if (BWD)
      for (int m = lane; m < W; m += 32) gdw[m] = m < M ? gD[p * pc.Dw + pc.doff + m] : R(0);
    __syncwarp();
    if (!BWD) {
      R acc[W];
#pragma unroll
      for (int m = 0; m < W; ++m) acc[m] = R(0);
      for (int e = lane; e < nv; e += 32) {
        const int k = kw[e];
        const R sk = Renv[(rb + k) * 4];
        R g[W], dg[W];
        ev.template eval<false>(wsm, net_of(pc, ti, slot_block(pc, k)), sk, g, dg, oor);
#pragma unroll
        for (int m = 0; m < W; ++m) acc[m] += g[m] * sk;
      }
#pragma unroll
      for (int m = 0; m < W; ++m) {
        R v = acc[m];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == (m & 31) && m < M) D[p * pc.Dw + pc.doff + m] = v * inv_nc;
      }
    } else {
      for (int e = lane; e < nv; e += 32) {
        const int k = kw[e];
        const R sk = Renv[(rb + k) * 4];
        R g[W], dg[W];
        ev.template eval<true>(wsm, net_of(pc, ti, slot_block(pc, k)), sk, g, dg, oor);
        R gs = R(0);
#pragma unroll
        for (int m = 0; m < W; ++m) gs += gdw[m] * (g[m] + sk * dg[m]);
        reinterpret_cast<V4*>(gR)[rb + k] = Vec4<R>::make(gs * inv_nc, R(0), R(0), R(0));
      }
    }
    __syncwarp();  // kw and gdw are rewritten for the warp's next atom
  }
}

template <class R, class Ev>
cudaError_t launch_rnet_ev(const PathConst& pc, const Ev& ev, int per_net_smem, const R* w, int n_nets,
                           const int* tsorted, const R* Renv, const R* gD, R* D, R* gR, bool bwd, cudaStream_t st) {
  const size_t smem = sizeof(R) * ((size_t)n_nets * per_net_smem + (size_t)kRWarps * Ev::kM) +
                      sizeof(int) * (size_t)kRWarps * pc.nc;
  auto kf = k_rnet<R, Ev, 0>;
  auto kb = k_rnet<R, Ev, 1>;
  cudaError_t e = allow_max_smem(bwd ? kb : kf);
  if (e != cudaSuccess) return e;
  int per_sm = 1;  // persistent: as many blocks as fit the SMs at once (each fills the nets once)
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bwd ? kb : kf, kRWarps * 32, smem) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  const long warps = pc.natoms;
  const unsigned blocks =
      (unsigned)std::max<long>(1, std::min<long>((warps + kRWarps - 1) / kRWarps, (long)per_sm * sm_count()));
  if (bwd)
    kb<<<blocks, kRWarps * 32, smem, st>>>(pc, ev, w, n_nets, tsorted, Renv, gD, D, gR);
  else
    kf<<<blocks, kRWarps * 32, smem, st>>>(pc, ev, w, n_nets, tsorted, Renv, gD, D, gR);
  return cudaGetLastError();
}

// The se_e2_r part's nets on the fused kernel: three-layer nets of the shapes below, or any nets of
// widths up to 32 whose parameters fit shared memory beside the compaction lists.
bool rnet_supported(const PartDesc& P, int precision) {
  if (P.kind != PART_R) return false;
  int w = 1;
  for (int l = 0; l < P.nl; ++l) w = std::max(w, P.emb[l].n_out);
  const bool fixed = P.nl == 3 && P.emb[0].n_out == 10 && P.emb[1].n_out == 20 && P.emb[2].n_out == 40;
  const size_t bytes = (size_t)P.n_nets * (P.per_net + 64) * (precision == DP_PREC_FP64 ? 8 : 4);
  return (fixed || w <= 32) && bytes <= 96 * 1024 && P.nc <= 2048;
}

template <class R>
cudaError_t launch_rnet(const PartDesc& P, const PathConst& pc, const R* params, const int* tsorted, const R* Renv,
                        const R* gD, R* D, R* gR, bool bwd, cudaStream_t st) {
  const R* wp = params + P.w_off;
  int w = 1;
  for (int l = 0; l < P.nl; ++l) w = std::max(w, P.emb[l].n_out);
  if (P.nl == 3) {
    const int a = P.emb[0].n_out, b = P.emb[1].n_out, c = P.emb[2].n_out;
#define DP_RNET_FIXED(A_, B_, C_)                                                                              \
    if (a == A_ && b == B_ && c == C_) {                                                                        \
      E3Fixed<R, A_, B_, C_> ev;                                                                                \
      ev.per_net_global = (int)P.per_net;                                                                       \
      return launch_rnet_ev<R>(pc, ev, E3Fixed<R, A_, B_, C_>::PN, wp, P.n_nets, tsorted, Renv, gD, D, gR, bwd, \
                               st);                                                                             \
    }
    DP_RNET_FIXED(10, 20, 40)
    DP_RNET_FIXED(2, 4, 8)
    DP_RNET_FIXED(4, 8, 16)
    DP_RNET_FIXED(8, 16, 32)
#undef DP_RNET_FIXED
  }
  E3Net nt;
  std::memset(&nt, 0, sizeof(nt));
  nt.nl = P.nl;
  for (int l = 0; l < P.nl; ++l) {
    const LayerDesc& L = P.emb[l];
    nt.in[l] = L.n_in;
    nt.out[l] = L.n_out;
    nt.skip[l] = L.skip;
    nt.loff[l] = (int)(L.w_off - P.w_off);
  }
  nt.per_net = (int)P.per_net;
  if (w <= 8)
    return launch_rnet_ev<R>(pc, E3Any<R, 8>{nt}, nt.per_net, wp, P.n_nets, tsorted, Renv, gD, D, gR, bwd, st);
  if (w <= 16)
    return launch_rnet_ev<R>(pc, E3Any<R, 16>{nt}, nt.per_net, wp, P.n_nets, tsorted, Renv, gD, D, gR, bwd, st);
  return launch_rnet_ev<R>(pc, E3Any<R, 32>{nt}, nt.per_net, wp, P.n_nets, tsorted, Renv, gD, D, gR, bwd, st);
}

// The whole path on CUDA cores for any descriptor: each part (Sec. II.A.1) builds its own
// environment rows from its slots of the one neighbour list, runs its embedding nets and writes
// its block of D; one fitting net reads D; each part then runs its reverse pass and scatters its
// pair forces and virials.
template <class R>
int run_generic(const DeviceModel& m, const PathConst& pc, const R* params, const PathIO& io, Arena& ar,
                cudaStream_t st) {
  const long N = pc.natoms;
  const int nparts = (int)m.parts.size();
  std::vector<PartBufs<R>> pb(nparts);
  // compressed models (se_e2_r, se_e3): the first part's nets are replaced by the quintic pieces
  const R* tab = reinterpret_cast<const R*>(std::is_same<R, double>::value ? (const void*)m.tab64
                                                                           : (const void*)m.tab32);
  auto tabulated = [&](int q) { return m.compressed && q == 0; };
  // se_e2_r parts on the fused per-neighbour kernel (uncompressed nets)
  auto rfused = [&](int q) { return !tabulated(q) && rnet_supported(m.parts[q], m.precision); };
  int* range_flag = &io.status->table_range;
  long maxe = 1;  // widest embedding-gradient buffer over the parts
  for (int q = 0; q < nparts; ++q) {
    const PartDesc& P = m.parts[q];
    PartBufs<R>& b = pb[q];
    b.pc = part_pc(pc, P);
    const long rows = N * P.nc;
    b.Renv = ar.get<R>(rows * 4);
    b.gR = ar.get<R>(rows * 4);
    if (P.kind == PART_E3 || tabulated(q) || rfused(q)) continue;
    for (int l = 0; l < P.nl; ++l) {
      const int w = P.emb[l].n_out;
      b.Y.push_back(ar.get<R>(rows * w));
      b.T.push_back(ar.get<R>(rows * w));
      maxe = std::max(maxe, rows * w);
    }
    if (P.kind == PART_A) b.Tm = ar.get<R>(N * P.M * 4);
    b.gs = ar.get<R>(rows);
  }
  R* D = ar.get<R>(N * pc.Dw);
  R* geA = ar.get<R>(maxe);
  R* geB = ar.get<R>(maxe);
  int* tsorted = ar.get<int>(N);
  const R* gD = nullptr;
  if (ar.measure) return run_fitting<R>(m, pc, params, D, io, ar, st, &gD);
  if (!ar.ok()) {
    set_error("scratch allocation failed");
    return DP_E_OOM;
  }
  {
    ProfScope _ps(io.prof, "sorted_types", st);
    k_sorted_types<<<nblk(N, 256), 256, 0, st>>>(io.type, io.perm, (int)N, tsorted);
  }
  // ---- forward, part by part ----
  for (int q = 0; q < nparts; ++q) {
    const PartDesc& P = m.parts[q];
    PartBufs<R>& b = pb[q];
    const PathConst& pq = b.pc;
    const long rows = N * P.nc;
    {
      ProfScope _ps(io.prof, "env", st);
      k_env<R><<<nblk(rows, 256), 256, 0, st>>>(pq, io.coord, io.perm, io.nl_j, io.nl_code, b.Renv);
    }
    if (P.kind == PART_E3) {
      ProfScope _ps(io.prof, "e3_fwd", st);
      if (tabulated(q))
        DP_CUDA_TRY(launch_e3_tab<R>(m, P, pq, tab, b.Renv, nullptr, D, nullptr, false, range_flag, st));
      else
        DP_CUDA_TRY(launch_e3<R>(P, pq, params, b.Renv, nullptr, D, nullptr, false, st));
      continue;
    }
    if (tabulated(q)) {  // se_e2_r
      ProfScope _ps(io.prof, "rtab_fwd", st);
      k_rtab_fwd<R><<<(unsigned)N, 64, 0, st>>>(pq, tab, tab_const(m), tsorted, b.Renv, D, range_flag);
      continue;
    }
    if (rfused(q)) {
      ProfScope _ps(io.prof, "rnet_fwd", st);
      DP_CUDA_TRY(launch_rnet<R>(P, pq, params, tsorted, b.Renv, nullptr, D, nullptr, false, st));
      continue;
    }
    for (int n = 0; n < P.n_nets; ++n) {
      const LayerDesc& L0 = P.emb[(size_t)n * P.nl];
      b.nets.w0[n] = params + L0.w_off;
      b.nets.b0[n] = params + L0.w_off + (long)L0.n_in * L0.n_out;
    }
    {
      const LayerDesc& L0 = P.emb[0];
      ProfScope _ps(io.prof, "emb_first", st);
      k_emb_first<R><<<nblk(rows * L0.n_out, 256), 256, 0, st>>>(pq, b.nets, tsorted, b.Renv, L0.n_out, L0.skip,
                                                                    b.Y[0], b.T[0]);
    }
    for (int ti = 0; ti < pc.ntypes; ++ti)
      for (int tj = 0; tj < pc.ntypes; ++tj) {
        const int net = pc.type_one_side ? tj : ti * pc.ntypes + tj;
        RowMap rm{1, 0, io.type_start[ti], pq.sel[tj], pq.sel_off[tj], P.nc,
                  (io.type_start[ti + 1] - io.type_start[ti]) * pq.sel[tj]};
        rm.zrow = b.Renv;  // padding rows: no layer outputs
        for (int l = 1; l < P.nl; ++l) {
          const LayerDesc& L = P.emb[(size_t)net * P.nl + l];
          const R* W = params + L.w_off;
          ProfScope _ps(io.prof, "emb_fwd", st);
          DP_CUDA_TRY(launch_dense_fwd<R>(rm, b.Y[l - 1], L.n_in, W, W + (long)L.n_in * L.n_out, L.n_out, L.skip, 1,
                                          b.Y[l], b.T[l], st));
        }
      }
    const R* G = b.Y[P.nl - 1];
    if (P.kind == PART_A) {
      ProfScope _ps(io.prof, "contract", st);
      k_contract<R><<<(unsigned)N, 128, sizeof(R) * P.M * 4, st>>>(pq, G, b.Renv, b.Tm, D);
    } else {
      ProfScope _ps(io.prof, "contract_r", st);
      k_contract_r<R><<<(unsigned)N, 64, 0, st>>>(pq, G, b.Renv, D);
    }
  }
  int rc = run_fitting<R>(m, pc, params, D, io, ar, st, &gD);
  if (rc != DP_OK) return rc;
  // ---- backward and forces, part by part ----
  for (int q = 0; q < nparts; ++q) {
    const PartDesc& P = m.parts[q];
    PartBufs<R>& b = pb[q];
    const PathConst& pq = b.pc;
    const long rows = N * P.nc;
    if (P.kind == PART_E3) {
      ProfScope _ps(io.prof, "e3_bwd", st);
      if (tabulated(q))
        DP_CUDA_TRY(launch_e3_tab<R>(m, P, pq, tab, b.Renv, gD, nullptr, b.gR, true, nullptr, st));
      else
        DP_CUDA_TRY(launch_e3<R>(P, pq, params, b.Renv, gD, nullptr, b.gR, true, st));
    } else if (tabulated(q)) {  // se_e2_r
      ProfScope _ps(io.prof, "rtab_bwd", st);
      k_rtab_bwd<R><<<(unsigned)N, 128, sizeof(R) * P.M, st>>>(pq, tab, tab_const(m), tsorted, b.Renv, gD, b.gR);
    } else if (rfused(q)) {
      ProfScope _ps(io.prof, "rnet_bwd", st);
      DP_CUDA_TRY(launch_rnet<R>(P, pq, params, tsorted, b.Renv, gD, nullptr, b.gR, true, st));
    } else {
      const R* G = b.Y[P.nl - 1];
      if (P.kind == PART_A) {
        ProfScope _ps(io.prof, "descr_bwd", st);
        k_descr_bwd<R><<<(unsigned)N, 128, sizeof(R) * (P.M * 8 + P.M * P.A), st>>>(pq, b.Tm, gD, G, b.Renv, geA,
                                                                                    b.gR);
      } else {
        ProfScope _ps(io.prof, "descr_bwd_r", st);
        k_descr_bwd_r<R><<<(unsigned)N, 128, sizeof(R) * P.M, st>>>(pq, gD, G, b.Renv, geA, b.gR);
      }
      R* gy = geA;
      R* gx = geB;
      for (int l = P.nl - 1; l >= 1; --l) {
        for (int ti = 0; ti < pc.ntypes; ++ti)
          for (int tj = 0; tj < pc.ntypes; ++tj) {
            const int net = pc.type_one_side ? tj : ti * pc.ntypes + tj;
            RowMap rm{1, 0, io.type_start[ti], pq.sel[tj], pq.sel_off[tj], P.nc,
                      (io.type_start[ti + 1] - io.type_start[ti]) * pq.sel[tj]};
            rm.zrow = b.Renv;
            const LayerDesc& L = P.emb[(size_t)net * P.nl + l];
            ProfScope _ps(io.prof, "emb_bwd", st);
            DP_CUDA_TRY(launch_dense_bwd<R>(rm, gy, b.T[l], L.n_in, params + L.w_off, L.n_out, L.skip, gx, st));
          }
        std::swap(gy, gx);
      }
      const LayerDesc& L0 = P.emb[0];
      ProfScope _ps(io.prof, "emb_first_bwd", st);
      k_emb_first_bwd<R><<<nblk(rows, 256), 256, 0, st>>>(pq, b.nets, tsorted, b.Renv, gy, b.T[0], L0.n_out, L0.skip,
                                                         b.gs);
    }
    ProfScope _ps(io.prof, "force", st);
    k_force<R><<<nblk(rows, 256), 256, 0, st>>>(pq, io.coord, io.perm, io.nl_j, io.nl_code, b.gs, b.gR, io.force,
                                                io.atom_virial);
  }
  DP_CUDA_TRY(cudaGetLastError());
  return DP_OK;
}

cudaError_t launch_energy_f32(const float* Eparts, int nparts, const int* perm, int n, double* atom_e,
                              cudaStream_t st) {
  k_energy_parts<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Eparts, nparts, perm, n, atom_e);
  return cudaGetLastError();
}

cudaError_t launch_shift_table(const PathConst& pc, double* out, cudaStream_t st) {
  k_shift_table<<<1, 32, 0, st>>>(pc, out);
  return cudaGetLastError();
}

cudaError_t launch_sum_rows(const double* in, long n, int w, double* out, cudaStream_t st) {
  k_sum_rows<<<w, 256, 0, st>>>(in, n, w, out);
  return cudaGetLastError();
}

template int run_generic<double>(const DeviceModel&, const PathConst&, const double*, const PathIO&, Arena&,
                                 cudaStream_t);
template int run_generic<float>(const DeviceModel&, const PathConst&, const float*, const PathIO&, Arena&,
                                cudaStream_t);
template int run_fitting<double>(const DeviceModel&, const PathConst&, const double*, const double*, const PathIO&,
                                 Arena&, cudaStream_t, const double**);
template int run_fitting<float>(const DeviceModel&, const PathConst&, const float*, const float*, const PathIO&,
                                Arena&, cudaStream_t, const float**);

}  // namespace dpgb
