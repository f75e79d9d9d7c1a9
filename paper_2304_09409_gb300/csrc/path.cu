// The energy / force / virial path on CUDA cores (FP64 or FP32 networks), for the se_e2_a,
// se_e2_r and hybrid descriptors.
//
// Steps (sorted-atom index p, neighbour slot k, row = p * Nc + k):
//   env      R_k = (s, s u) with u = r_ij / r, s = s(r)            Eqs. (rij), (switch)
//   emb      G_k = N^{a_i, a_j}(s) layer by layer                  Eqs. (G2), (NN)
//   contract T = G^T R / Nc,  D = T T_<^T                          se_e2_a descriptor
//            D_r = G_r^T s / Nc                                    se_e2_r descriptor
//            (hybrid: D = [D_a, D_r], each part with its own nets) Sec. II.A.1
//   fit      E_i = F^{a_i}(D)                                      Eq. (fitting_energy)
//   backward dE/dD -> dE/dT -> (dE/dG, dE/dR) -> dE/ds -> dE/dr_ij
//   force    F_i += dE/dr_ij, F_j -= dE/dr_ij (FP64 atomics)        Sec. II.A.2
//   virial   Xi_ab = -sum (dE/dr_ij)_a (r_ij)_b (FP64, deterministic two-stage reduction)
//
// The pair displacement is always rebuilt from the neighbour list with the exact FP64
// formula.  In FP32 mode the switch and its derivative are evaluated in FP32 in a form without
// cancellation near r_c (env.cuh); energy, force and virial accumulate in FP64.
#include "dp_internal.cuh"
#include "path.cuh"
#include "env.cuh"

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
  const int j = nl_j[(long)i * pc.nc + k];
  R o[4] = {R(0), R(0), R(0), R(0)};
  if (j >= 0) {
    double d0, d1, d2;
    listed_disp(coord + 3 * i, coord + 3 * j, nl_code[(long)i * pc.nc + k], pc, frame_of(pc, i), d0, d1, d2);
    const double r2 = norm2_exact(d0, d1, d2);
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
  const R t = tanh_r(s * nets.w0[net][o] + nets.b0[net][o]);
  R y = t;
  if (skip) y += s;  // n_in = 1: both +x and +{x,x} add the scalar input
  Y[e] = y;
  T[e] = t;
}

// dE/ds through the first layer; `accum` adds to gs (a second embedding family of a hybrid).
template <class R>
__global__ void k_emb_first_bwd(PathConst pc, NetPtrs<R> nets, const int* __restrict__ atom_type_sorted,
                                const R* __restrict__ GY, const R* __restrict__ T, int w1, int skip,
                                R* __restrict__ gs, int accum) {
  const long row = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= (long)pc.natoms * pc.nc) return;
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
  gs[row] = accum ? gs[row] + acc : acc;
}

// ---- T = G^T R / Nc and D = T T_<^T, one block per atom -------------------------------------
template <class R>
__global__ void k_contract(PathConst pc, const R* __restrict__ G, const R* __restrict__ Renv, R* __restrict__ Tm,
                           R* __restrict__ D) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  R* Ts = reinterpret_cast<R*>(sm_raw);  // [M][4]
  const int p = blockIdx.x;
  const int M = pc.M, A = pc.A, nc = pc.nc;
  const R inv_nc = R(1) / R(nc);
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    R a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    const long rb = (long)p * nc;
    for (int k = 0; k < nc; ++k) {
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
    D[(long)p * pc.Dw + idx] =
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
  for (int e = threadIdx.x; e < M * A; e += blockDim.x) gDs[e] = gD[(long)p * pc.Dw + e];
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
// G rows hold Mr values; D_r is written at column `off` of D (row stride Dw).
template <class R>
__global__ void k_contract_r(PathConst pc, const R* __restrict__ G, const R* __restrict__ Renv, int off,
                             R* __restrict__ D) {
  const int p = blockIdx.x;
  const int Mr = pc.Mr, nc = pc.nc;
  const long rb = (long)p * nc;
  for (int m = threadIdx.x; m < Mr; m += blockDim.x) {
    R acc = 0;
    for (int k = 0; k < nc; ++k) acc += G[(rb + k) * Mr + m] * Renv[(rb + k) * 4];
    D[(long)p * pc.Dw + off + m] = acc / R(nc);
  }
}

// Reverse of k_contract_r: dE/dG_r[k][m] = gD_r[m] s_k / Nc into gG, and the direct term
// dE/ds_k = sum_m gD_r[m] G_r[k][m] / Nc into the radial component of gR (added to what the
// se_e2_a block wrote when `accum`, else gR = (term, 0, 0, 0)).  One block per atom, a warp per row.
template <class R>
__global__ void k_descr_bwd_r(PathConst pc, const R* __restrict__ gD, int off, const R* __restrict__ G,
                              const R* __restrict__ Renv, R* __restrict__ gG, R* __restrict__ gR, int accum) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  R* gDs = reinterpret_cast<R*>(sm_raw);  // [Mr]
  const int p = blockIdx.x;
  const int Mr = pc.Mr, nc = pc.nc;
  for (int e = threadIdx.x; e < Mr; e += blockDim.x) gDs[e] = gD[(long)p * pc.Dw + off + e];
  __syncthreads();
  const R inv_nc = R(1) / R(nc);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int k = warp; k < nc; k += nw) {
    const long row = (long)p * nc + k;
    const R s = Renv[row * 4];
    R acc = 0;
    for (int m = lane; m < Mr; m += 32) {
      acc += gDs[m] * G[row * Mr + m];
      gG[row * Mr + m] = gDs[m] * s * inv_nc;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      typename Vec4<R>::T* g4 = reinterpret_cast<typename Vec4<R>::T*>(gR) + row;
      if (accum) {
        typename Vec4<R>::T v = *g4;
        v.x += acc * inv_nc;
        *g4 = v;
      } else {
        *g4 = Vec4<R>::make(acc * inv_nc, R(0), R(0), R(0));
      }
    }
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
    const int j = nl_j[(long)i * pc.nc + k];
    if (j >= 0) {
      double d[3];
      listed_disp(coord + 3 * i, coord + 3 * j, nl_code[(long)i * pc.nc + k], pc, frame_of(pc, i), d[0], d[1], d[2]);
      const double r2 = norm2_exact(d[0], d[1], d[2]);
      R r, s, ds, u[3];
      pair_env<R>(d[0], d[1], d[2], r2, pc.rs, pc.rc, pc.near2, r, s, ds, u);
      const typename Vec4<R>::T g4 = reinterpret_cast<const typename Vec4<R>::T*>(gR)[row];
      const R gvu = g4.y * u[0] + g4.z * u[1] + g4.w * u[2];
      const R gsum = gs_emb[row] + g4.x + gvu;
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

// One family of embedding nets (the se_e2_a nets, or the se_e2_r nets of a hybrid): layer
// descriptors, layer count and per-layer outputs / tanh values over all rows.
template <class R>
struct EmbFamily {
  const std::vector<LayerDesc>* layers;
  int nl;
  std::vector<R*> Y, T;
};

template <class R>
int run_generic(const DeviceModel& m, const PathConst& pc, const R* params, const PathIO& io, Arena& ar,
                cudaStream_t st) {
  const long N = pc.natoms, nc = pc.nc, rows = N * nc;
  const int M = pc.M, A = pc.A, desc = m.cfg.descriptor;
  const bool ang = desc != DP_DESC_SE_E2_R, rad = desc != DP_DESC_SE_E2_A;
  // family 0: nets of embed[] (se_e2_a, or se_e2_r alone); family 1: the hybrid's se_e2_r nets
  const int nfam = desc == DP_DESC_HYBRID ? 2 : 1;
  EmbFamily<R> fam[2];
  fam[0].layers = &m.emb;
  fam[0].nl = m.cfg.n_embed;
  fam[1].layers = &m.emb_r;
  fam[1].nl = m.cfg.n_embed_r;
  // ---- scratch ----
  R* Renv = ar.get<R>(rows * 4);
  int maxe = 1;
  for (int f = 0; f < nfam; ++f)
    for (int l = 0; l < fam[f].nl; ++l) {
      const int w = (*fam[f].layers)[l].n_out;
      fam[f].Y.push_back(ar.get<R>(rows * w));
      fam[f].T.push_back(ar.get<R>(rows * w));
      maxe = std::max(maxe, w);
    }
  R* Tm = ang ? ar.get<R>(N * M * 4) : nullptr;
  R* D = ar.get<R>(N * pc.Dw);
  R* geA = ar.get<R>(rows * maxe);
  R* geB = ar.get<R>(rows * maxe);
  R* gR = ar.get<R>(rows * 4);
  R* gs = ar.get<R>(rows);
  int* tsorted = ar.get<int>(N);
  const unsigned fblocks = nblk(rows, 256);
  const R* gD = nullptr;
  if (ar.measure) return run_fitting<R>(m, pc, params, D, io, ar, st, &gD);
  if (!ar.ok()) {
    set_error("scratch allocation failed");
    return DP_E_OOM;
  }
  // ---- forward ----
  {
    ProfScope _ps(io.prof, "sorted_types", st);
    k_sorted_types<<<nblk(N, 256), 256, 0, st>>>(io.type, io.perm, (int)N, tsorted);
  }
  {
    ProfScope _ps(io.prof, "env", st);
    k_env<R><<<nblk(rows, 256), 256, 0, st>>>(pc, io.coord, io.perm, io.nl_j, io.nl_code, Renv);
  }
  NetPtrs<R> nets[2];
  for (int f = 0; f < nfam; ++f) {
    const std::vector<LayerDesc>& Ls = *fam[f].layers;
    const int ne = fam[f].nl;
    for (int n = 0; n < m.n_embed_nets; ++n) {
      const LayerDesc& L0 = Ls[(size_t)n * ne];
      nets[f].w0[n] = params + L0.w_off;
      nets[f].b0[n] = params + L0.w_off + (long)L0.n_in * L0.n_out;
    }
    const LayerDesc& L0 = Ls[0];
    {
      ProfScope _ps(io.prof, "emb_first", st);
      k_emb_first<R><<<nblk(rows * L0.n_out, 256), 256, 0, st>>>(pc, nets[f], tsorted, Renv, L0.n_out, L0.skip,
                                                                    fam[f].Y[0], fam[f].T[0]);
    }
    for (int ti = 0; ti < pc.ntypes; ++ti)
      for (int tj = 0; tj < pc.ntypes; ++tj) {
        const int net = pc.type_one_side ? tj : ti * pc.ntypes + tj;
        RowMap rm{1, 0, io.type_start[ti], pc.sel[tj], pc.sel_off[tj], (int)nc,
                  (io.type_start[ti + 1] - io.type_start[ti]) * pc.sel[tj]};
        for (int l = 1; l < ne; ++l) {
          const LayerDesc& L = Ls[(size_t)net * ne + l];
          const R* W = params + L.w_off;
          ProfScope _ps(io.prof, "emb_fwd", st);
          DP_CUDA_TRY(launch_dense_fwd<R>(rm, fam[f].Y[l - 1], L.n_in, W, W + (long)L.n_in * L.n_out, L.n_out, L.skip,
                                          1, fam[f].Y[l], fam[f].T[l], st));
        }
      }
  }
  const R* Ga = fam[0].Y[fam[0].nl - 1];
  const R* Gr = fam[nfam - 1].Y[fam[nfam - 1].nl - 1];
  const int da = ang ? M * A : 0;
  if (ang) {
    ProfScope _ps(io.prof, "contract", st);
    k_contract<R><<<(unsigned)N, 128, sizeof(R) * M * 4, st>>>(pc, Ga, Renv, Tm, D);
  }
  if (rad) {
    ProfScope _ps(io.prof, "contract_r", st);
    k_contract_r<R><<<(unsigned)N, 64, 0, st>>>(pc, Gr, Renv, da, D);
  }
  int rc = run_fitting<R>(m, pc, params, D, io, ar, st, &gD);
  if (rc != DP_OK) return rc;
  // ---- backward: per family, descriptor block -> dE/dG -> embedding layers -> dE/ds ----
  for (int f = 0; f < nfam; ++f) {
    const bool fam_ang = ang && f == 0;  // the se_e2_a block reads family 0 when present
    const std::vector<LayerDesc>& Ls = *fam[f].layers;
    const int ne = fam[f].nl;
    if (fam_ang) {
      ProfScope _ps(io.prof, "descr_bwd", st);
      k_descr_bwd<R><<<(unsigned)N, 128, sizeof(R) * (M * 8 + M * A), st>>>(pc, Tm, gD, Ga, Renv, geA, gR);
    } else {
      ProfScope _ps(io.prof, "descr_bwd_r", st);
      k_descr_bwd_r<R><<<(unsigned)N, 128, sizeof(R) * pc.Mr, st>>>(pc, gD, da, Gr, Renv, geA, gR, ang ? 1 : 0);
    }
    R* gy = geA;
    R* gx = geB;
    for (int l = ne - 1; l >= 1; --l) {
      for (int ti = 0; ti < pc.ntypes; ++ti)
        for (int tj = 0; tj < pc.ntypes; ++tj) {
          const int net = pc.type_one_side ? tj : ti * pc.ntypes + tj;
          RowMap rm{1, 0, io.type_start[ti], pc.sel[tj], pc.sel_off[tj], (int)nc,
                    (io.type_start[ti + 1] - io.type_start[ti]) * pc.sel[tj]};
          const LayerDesc& L = Ls[(size_t)net * ne + l];
          ProfScope _ps(io.prof, "emb_bwd", st);
          DP_CUDA_TRY(launch_dense_bwd<R>(rm, gy, fam[f].T[l], L.n_in, params + L.w_off, L.n_out, L.skip, gx, st));
        }
      std::swap(gy, gx);
    }
    const LayerDesc& L0 = Ls[0];
    {
      ProfScope _ps(io.prof, "emb_first_bwd", st);
      k_emb_first_bwd<R><<<nblk(rows, 256), 256, 0, st>>>(pc, nets[f], tsorted, gy, fam[f].T[0], L0.n_out, L0.skip, gs,
                                                          f > 0 ? 1 : 0);
    }
  }
  // ---- forces and virial ----
  {
    ProfScope _ps(io.prof, "force", st);
    k_force<R><<<fblocks, 256, 0, st>>>(pc, io.coord, io.perm, io.nl_j, io.nl_code, gs, gR, io.force,
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
