// Compressed embedding (Sec. II.A.6 "Compression of neural networks"):
//   tabulated inference  G_m(s) = quintic piece of interval l at t = s - x_l   Eq. (compress)
//   operator merging     each row G_k is formed in registers and immediately folded into
//                        T = G^T R / Nc; G never reaches memory
//   precise indexing     only the real neighbours of each type block are visited
//
// GB300 design.  One warp owns one centre atom.  Forward: the lanes of the warp split the
// M outputs (lane m, m+32, ...), so the coefficient loads of one interval are coalesced
// 128-byte rows and T accumulates in registers with no reduction; the environment of 32
// neighbours at a time is computed lane-parallel (exact FP64 displacement) and broadcast by
// shuffles.  D = T T_<^T is formed from registers.  Backward: four groups of eight lanes
// each take one neighbour, recompute G and G' from the table, reduce dE/dR and dE/ds over
// the eight lanes, and scatter the pair force with FP64 atomics; F_i is accumulated in
// registers and written once per atom.
#include <cuda_bf16.h>

#include <type_traits>
#include <vector>

#include "env.cuh"
#include "fit_tc.cuh"
#include "mom.cuh"
#include "table.cuh"
#include "tabeval.cuh"

namespace dpgb {

namespace {

// Values, first and second derivatives of every output of net `net` at node l (jets).
__global__ void k_table_nodes(const double* __restrict__ p64, const LayerDesc* __restrict__ layers, int n_embed,
                              TabConst tc, int M, int maxw, double* __restrict__ y, double* __restrict__ y1,
                              double* __restrict__ y2) {
  extern __shared__ double jet[];  // 2 buffers x 3 x maxw
  const int l = blockIdx.x, net = blockIdx.y;
  double* xv = jet;
  double* xd = jet + maxw;
  double* xdd = jet + 2 * maxw;
  double* yv = jet + 3 * maxw;
  double* yd = jet + 4 * maxw;
  double* ydd = jet + 5 * maxw;
  if (threadIdx.x == 0) {
    xv[0] = node_at(tc, l);
    xd[0] = 1.0;
    xdd[0] = 0.0;
  }
  __syncthreads();
  for (int q = 0; q < n_embed; ++q) {
    const LayerDesc L = layers[(size_t)net * n_embed + q];
    const double* W = p64 + L.w_off;
    const double* b = W + (long)L.n_in * L.n_out;
    for (int o = threadIdx.x; o < L.n_out; o += blockDim.x) {
      double z = b[o], z1 = 0.0, z2 = 0.0;
      for (int i = 0; i < L.n_in; ++i) {
        const double w = W[(long)i * L.n_out + o];
        z += xv[i] * w;
        z1 += xd[i] * w;
        z2 += xdd[i] * w;
      }
      const double t = tanh(z), g = 1.0 - t * t;
      double a = t, a1 = g * z1, a2 = g * z2 - 2.0 * t * g * z1 * z1;
      if (L.skip) {
        const int src = (L.skip == 1) ? o : o % L.n_in;
        a += xv[src];
        a1 += xd[src];
        a2 += xdd[src];
      }
      yv[o] = a;
      yd[o] = a1;
      ydd[o] = a2;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < L.n_out; o += blockDim.x) {
      xv[o] = yv[o];
      xd[o] = yd[o];
      xdd[o] = ydd[o];
    }
    __syncthreads();
  }
  const size_t base = ((size_t)net * (tc.lc + 1) + l) * M;
  for (int o = threadIdx.x; o < M; o += blockDim.x) {
    y[base + o] = xv[o];
    y1[base + o] = xd[o];
    y2[base + o] = xdd[o];
  }
}

// Eq. (compress): coefficients a..f of interval l from the two node jets.
__global__ void k_table_coef(TabConst tc, int M, int nets, const double* __restrict__ y,
                             const double* __restrict__ y1, const double* __restrict__ y2, double* __restrict__ tab64,
                             float* __restrict__ tab32) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long total = (long)nets * tc.lc * M;
  if (e >= total) return;
  const int m = (int)(e % M);
  const int l = (int)((e / M) % tc.lc);
  const int net = (int)(e / ((long)M * tc.lc));
  const size_t a = ((size_t)net * (tc.lc + 1) + l) * M + m, b = a + M;
  const double dx = node_at(tc, l + 1) - node_at(tc, l);
  const double h = y[b] - y[a];
  const double d0 = y1[a], d1 = y1[b], dd0 = y2[a], dd1 = y2[b];
  const double dx2 = dx * dx, dx3 = dx2 * dx;
  double c[6];
  c[0] = (12.0 * h - 6.0 * (d1 + d0) * dx + (dd1 - dd0) * dx2) / (2.0 * dx3 * dx2);
  c[1] = (-30.0 * h + (14.0 * d1 + 16.0 * d0) * dx + (-2.0 * dd1 + 3.0 * dd0) * dx2) / (2.0 * dx2 * dx2);
  c[2] = (20.0 * h - (8.0 * d1 + 12.0 * d0) * dx + (dd1 - 3.0 * dd0) * dx2) / (2.0 * dx3);
  c[3] = 0.5 * dd0;
  c[4] = d0;
  c[5] = y[a];
  const size_t o = (((size_t)net * tc.lc + l) * M + m) * kCoefStride;
#pragma unroll
  for (int q = 0; q < kCoefStride; ++q) {
    tab64[o + q] = q < 6 ? c[q] : 0.0;
    tab32[o + q] = q < 6 ? (float)c[q] : 0.f;
  }
}

// ---- per-slot environment of the listed pairs: (s, u) and (ds/dr, r), once per step --------
template <class R>
__global__ void __launch_bounds__(256)
    k_env_tab(PathConst pc, const double* __restrict__ coord, const int* __restrict__ perm,
              const int* __restrict__ nl_j, const int* __restrict__ nl_code, typename Vec4<R>::T* __restrict__ env) {
  const long row = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= (long)pc.natoms * pc.nc) return;
  const int p = (int)(row / pc.nc), k = (int)(row % pc.nc);
  const int i = perm[p];
  const long slot = (long)i * pc.nc + k;
  const int j = nl_j[slot];
  if (j < 0) return;  // padding is never read
  double d0, d1, d2;
  listed_disp(coord + 3 * i, coord + 3 * j, nl_code[slot], pc, frame_of(pc, i), d0, d1, d2);
  R r, s, ds, u[3];
  pair_env<R>(d0, d1, d2, norm2_exact(d0, d1, d2), pc.rs, pc.rc, pc.near2, r, s, ds, u);
  env[row * 2] = Vec4<R>::make(s, u[0], u[1], u[2]);
  env[row * 2 + 1] = Vec4<R>::make(ds, r, R(0), R(0));
}

// ---- forward: T = G^T R / Nc with G from the table, then D = T T_<^T --------------------------
template <class DT, class R>
__device__ __forceinline__ DT to_dt(R v) {
  return (DT)v;
}
template <>
__device__ __forceinline__ __nv_bfloat16 to_dt<__nv_bfloat16, float>(float v) {
  return __float2bfloat16_rn(v);
}

template <class R, int MPL, class DT>
__global__ void __launch_bounds__(128)
    k_tab_fwd(PathConst pc, TabConst tc, const R* __restrict__ tab, const double* __restrict__ coord,
              const int* __restrict__ perm, const int* __restrict__ type, const int* __restrict__ nl_j,
              const typename Vec4<R>::T* __restrict__ env, R* __restrict__ Tm, DT* __restrict__ D,
              DevStatus* __restrict__ st) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = blockIdx.x * 4 + warp;
  if (p >= pc.natoms) return;
  const int i = perm[p], ti = type[i];
  const int M = pc.M, nc = pc.nc, A = pc.A;
  R acc[MPL][4];
#pragma unroll
  for (int u = 0; u < MPL; ++u) acc[u][0] = acc[u][1] = acc[u][2] = acc[u][3] = R(0);
  bool oor = false;
  const double* xi = coord + 3 * i;
  Quint<R> cq[MPL];  // coefficients of the current interval for this lane's outputs
  for (int t = 0; t < pc.ntypes; ++t) {
    const R* tabn = tab + (size_t)net_of(pc, ti, t) * tc.lc * M * kCoefStride;
    const int kend = pc.sel_off[t + 1];
    int cur = -1;  // interval whose coefficients sit in cq (warp-uniform)
    for (int base = pc.sel_off[t]; base < kend; base += 32) {
      const int k = base + lane;
      const int j = (k < kend) ? nl_j[(long)i * nc + k] : -1;
      R e0 = 0, e1 = 0, e2 = 0, e3 = 0, tt = 0;
      int l = 0;
      if (j >= 0) {
        const typename Vec4<R>::T a4 = env[((long)p * nc + k) * 2];  // (s, u)
        const R s = a4.x;
        e0 = s;
        e1 = s * a4.y;
        e2 = s * a4.z;
        e3 = s * a4.w;
        l = tab_interval<R>(tc, s, tt, oor);
      }
      const unsigned valid = __ballot_sync(0xffffffffu, j >= 0);
      unsigned mask = valid;
      while (mask) {
        const int q = __ffs(mask) - 1;
        mask &= mask - 1;
        const R tq = __shfl_sync(0xffffffffu, tt, q);
        const int lq = __shfl_sync(0xffffffffu, l, q);
        const R r0 = __shfl_sync(0xffffffffu, e0, q), r1 = __shfl_sync(0xffffffffu, e1, q);
        const R r2 = __shfl_sync(0xffffffffu, e2, q), r3 = __shfl_sync(0xffffffffu, e3, q);
        if (lq != cur) {  // neighbours are sorted by distance: runs share an interval
          cur = lq;
          const R* c = tabn + (size_t)lq * M * kCoefStride;
#pragma unroll
          for (int u = 0; u < MPL; ++u) {
            const int m = lane + 32 * u;
            if (m < M) cq[u] = load_quint(c + (size_t)m * kCoefStride);
          }
        }
#pragma unroll
        for (int u = 0; u < MPL; ++u) {
          const int m = lane + 32 * u;
          if (m < M) {
            const R g = quint_value<R>(cq[u], tq);
            acc[u][0] += g * r0;
            acc[u][1] += g * r1;
            acc[u][2] += g * r2;
            acc[u][3] += g * r3;
          }
        }
      }
      if (valid != 0xffffffffu) break;  // real neighbours fill the front of each type block
    }
  }
  if (__any_sync(0xffffffffu, oor) && lane == 0) atomicOr(&st->table_range, 1);
  const R inv_nc = R(1) / R(nc);
#pragma unroll
  for (int u = 0; u < MPL; ++u) {
    acc[u][0] *= inv_nc;
    acc[u][1] *= inv_nc;
    acc[u][2] *= inv_nc;
    acc[u][3] *= inv_nc;
    const int m = lane + 32 * u;
    if (m < M) reinterpret_cast<typename Vec4<R>::T*>(Tm)[(long)p * M + m] =
        Vec4<R>::make(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
  }
  DT* Dp = D + (long)p * M * A;
  for (int lq = 0; lq < A; ++lq) {
    const R t0 = __shfl_sync(0xffffffffu, acc[0][0], lq), t1 = __shfl_sync(0xffffffffu, acc[0][1], lq);
    const R t2 = __shfl_sync(0xffffffffu, acc[0][2], lq), t3 = __shfl_sync(0xffffffffu, acc[0][3], lq);
#pragma unroll
    for (int u = 0; u < MPL; ++u) {
      const int m = lane + 32 * u;
      if (m < M) Dp[m * A + lq] = to_dt<DT, R>(acc[u][0] * t0 + acc[u][1] * t1 + acc[u][2] * t2 + acc[u][3] * t3);
    }
  }
}

// ---- backward: dE/dT, then per neighbour dE/dR, dE/ds -> pair force, force scatter, virial ----
template <class R>
__global__ void __launch_bounds__(128)
    k_tab_bwd(PathConst pc, TabConst tc, const R* __restrict__ tab, const double* __restrict__ coord,
              const int* __restrict__ perm, const int* __restrict__ type, const int* __restrict__ nl_j,
              const typename Vec4<R>::T* __restrict__ env, const R* __restrict__ Tm,
              const R* __restrict__ gD, double* __restrict__ force, double* __restrict__ avir) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int M = pc.M, nc = pc.nc, A = pc.A;
  R* Ts = reinterpret_cast<R*>(sm_raw) + (size_t)warp * (M * 8);
  R* gTs = Ts + M * 4;
  const int p = blockIdx.x * 4 + warp;
  // per-atom partial sums over the atom's neighbours stay in the path's precision; every
  // accumulation across atoms (the force scatter, the virial sum) is FP64
  R v[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) v[q] = R(0);
  if (p < pc.natoms) {
    const int i = perm[p], ti = type[i];
    for (int e = lane; e < M * 4; e += 32) Ts[e] = Tm[(long)p * M * 4 + e];
    __syncwarp();
    // dE/dT[m][c] = sum_l dE/dD[m][l] T[l][c] + [m < M_<] sum_q dE/dD[q][m] T[q][c]
    const R* gDp = gD + (long)p * M * A;
    for (int e = lane; e < M * 4; e += 32) {
      const int m = e >> 2, c = e & 3;
      R acc = 0;
      for (int lq = 0; lq < A; ++lq) acc += gDp[m * A + lq] * Ts[lq * 4 + c];
      if (m < A)
        for (int q = 0; q < M; ++q) acc += gDp[q * A + m] * Ts[q * 4 + c];
      gTs[e] = acc;
    }
    __syncwarp();
    const int grp = lane >> 3, sub = lane & 7;
    const R inv_nc = R(1) / R(nc);
    R fi0 = 0, fi1 = 0, fi2 = 0;
    for (int t = 0; t < pc.ntypes; ++t) {
      const R* tabn = tab + (size_t)net_of(pc, ti, t) * tc.lc * M * kCoefStride;
      const int kend = pc.sel_off[t + 1];
      for (int base = pc.sel_off[t]; base < kend; base += 32) {
        const int k = base + lane;
        const int j = (k < kend) ? nl_j[(long)i * nc + k] : -1;
        R s = 0, ds = 0, r = 1, u0 = 0, u1 = 0, u2 = 0, tt = 0;
        int l = 0;
        if (j >= 0) {
          const long row = (long)p * nc + k;
          const typename Vec4<R>::T a4 = env[row * 2], b4 = env[row * 2 + 1];  // (s, u), (ds, r)
          s = a4.x;
          u0 = a4.y;
          u1 = a4.z;
          u2 = a4.w;
          ds = b4.x;
          r = b4.y;
          bool oor = false;
          l = tab_interval<R>(tc, s, tt, oor);
        }
        const unsigned valid = __ballot_sync(0xffffffffu, j >= 0);
        const int nvalid = __popc(valid);
        for (int idx = 0; idx < nvalid; idx += 4) {
          const int my = idx + grp;
          const bool have = my < nvalid;
          int q = 0;
          if (have) {
            unsigned rest = valid;
            for (int c = 0; c < my; ++c) rest &= rest - 1;
            q = __ffs(rest) - 1;
          }
          const R sq = __shfl_sync(0xffffffffu, s, q), dsq = __shfl_sync(0xffffffffu, ds, q);
          const R rq = __shfl_sync(0xffffffffu, r, q), tq = __shfl_sync(0xffffffffu, tt, q);
          const R uq0 = __shfl_sync(0xffffffffu, u0, q), uq1 = __shfl_sync(0xffffffffu, u1, q);
          const R uq2 = __shfl_sync(0xffffffffu, u2, q);
          const int lq = __shfl_sync(0xffffffffu, l, q), jq = __shfl_sync(0xffffffffu, j, q);

          R g0 = 0, g1 = 0, g2 = 0, g3 = 0, gse = 0;
          if (have) {
            const R* c = tabn + (size_t)lq * M * kCoefStride;
            const R e1 = sq * uq0, e2 = sq * uq1, e3 = sq * uq2;
            for (int m = sub; m < M; m += 8) {
              const Quint<R> cq = load_quint(c + (size_t)m * kCoefStride);
              const R G = quint_value<R>(cq, tq), Gp = quint_slope<R>(cq, tq);
              const typename Vec4<R>::T g4 = reinterpret_cast<const typename Vec4<R>::T*>(gTs)[m];
              const R a0 = g4.x, a1 = g4.y, a2 = g4.z, a3 = g4.w;
              g0 += a0 * G;
              g1 += a1 * G;
              g2 += a2 * G;
              g3 += a3 * G;
              gse += (a0 * sq + a1 * e1 + a2 * e2 + a3 * e3) * Gp;
            }
          }
#pragma unroll
          for (int off = 4; off > 0; off >>= 1) {
            g0 += __shfl_xor_sync(0xffffffffu, g0, off);
            g1 += __shfl_xor_sync(0xffffffffu, g1, off);
            g2 += __shfl_xor_sync(0xffffffffu, g2, off);
            g3 += __shfl_xor_sync(0xffffffffu, g3, off);
            gse += __shfl_xor_sync(0xffffffffu, gse, off);
          }
          if (have && sub == 0) {
            g0 *= inv_nc;
            g1 *= inv_nc;
            g2 *= inv_nc;
            g3 *= inv_nc;
            gse *= inv_nc;
            const R gvu = g1 * uq0 + g2 * uq1 + g3 * uq2;
            const R a = dsq * (gse + g0 + gvu), b = sq / rq;
            const R gd0 = a * uq0 + b * (g1 - gvu * uq0);
            const R gd1 = a * uq1 + b * (g2 - gvu * uq1);
            const R gd2 = a * uq2 + b * (g3 - gvu * uq2);
            fi0 += gd0;
            fi1 += gd1;
            fi2 += gd2;
            atomicAdd(force + 3 * jq, widen(-gd0));
            atomicAdd(force + 3 * jq + 1, widen(-gd1));
            atomicAdd(force + 3 * jq + 2, widen(-gd2));
            const R gdv[3] = {gd0, gd1, gd2};
            const R dv[3] = {rq * uq0, rq * uq1, rq * uq2};
#pragma unroll
            for (int aa = 0; aa < 3; ++aa)
#pragma unroll
              for (int bb = 0; bb < 3; ++bb) v[aa * 3 + bb] -= gdv[aa] * dv[bb];
          }
        }
        if (valid != 0xffffffffu) break;
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      fi0 += __shfl_xor_sync(0xffffffffu, fi0, off);
      fi1 += __shfl_xor_sync(0xffffffffu, fi1, off);
      fi2 += __shfl_xor_sync(0xffffffffu, fi2, off);
    }
    if (lane == 0) {
      atomicAdd(force + 3 * i, widen(fi0));
      atomicAdd(force + 3 * i + 1, widen(fi1));
      atomicAdd(force + 3 * i + 2, widen(fi2));
    }
  }
  // per-atom virial (input order): one warp owns one atom
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    R x = v[q];
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    if (lane == 0 && p < pc.natoms) avir[9L * perm[p] + q] = widen(x);
  }
}

template <class R, class DT>
int run_tab(const DeviceModel& m, const PathConst& pc, const PathIO& io, Arena& ar, cudaStream_t st,
            const R* params, const R* tab) {
  constexpr bool kTensor = std::is_same<DT, __nv_bfloat16>::value;
  const long N = pc.natoms;
  const int M = pc.M, A = pc.A;
  R* Tm = ar.get<R>(N * M * 4);
  DT* D = ar.get<DT>(N * M * A);
  typedef typename Vec4<R>::T V4;
  V4* env = ar.get<V4>(N * pc.nc * 2);
  const unsigned blocks = (unsigned)((N + 3) / 4);
  const R* gD = nullptr;
  if (ar.measure) {
    if constexpr (kTensor) {
      const float* g = nullptr;
      return run_fitting_tc(m, pc, D, io, ar, st, &g);
    } else {
      return run_fitting<R>(m, pc, params, D, io, ar, st, &gD);
    }
  }
  if (!ar.ok()) {
    set_error("scratch allocation failed");
    return DP_E_OOM;
  }
  const TabConst tc = tab_const(m);
  const int mpl = (M + 31) / 32;
  {
    ProfScope _ps(io.prof, "env", st);
    const long rows = N * pc.nc;
    k_env_tab<R><<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(pc, io.coord, io.perm, io.nl_j, io.nl_code, env);
  }
  {
    ProfScope _ps(io.prof, "tab_fwd", st);
    if (mpl <= 1)
      k_tab_fwd<R, 1, DT><<<blocks, 128, 0, st>>>(pc, tc, tab, io.coord, io.perm, io.type, io.nl_j, env, Tm,
                                                  D, io.status);
    else if (mpl <= 2)
      k_tab_fwd<R, 2, DT><<<blocks, 128, 0, st>>>(pc, tc, tab, io.coord, io.perm, io.type, io.nl_j, env, Tm,
                                                  D, io.status);
    else if (mpl <= 4)
      k_tab_fwd<R, 4, DT><<<blocks, 128, 0, st>>>(pc, tc, tab, io.coord, io.perm, io.type, io.nl_j, env, Tm,
                                                  D, io.status);
    else
      k_tab_fwd<R, 8, DT><<<blocks, 128, 0, st>>>(pc, tc, tab, io.coord, io.perm, io.type, io.nl_j, env, Tm,
                                                  D, io.status);
  }
  DP_CUDA_TRY(cudaGetLastError());
  int rc;
  if constexpr (kTensor) {
    const float* g = nullptr;
    rc = run_fitting_tc(m, pc, D, io, ar, st, &g);
    gD = g;
  } else {
    rc = run_fitting<R>(m, pc, params, D, io, ar, st, &gD);
  }
  if (rc != DP_OK) return rc;
  const size_t smem = sizeof(R) * 4 * (size_t)(M * 8);
  DP_CUDA_TRY(allow_max_smem(k_tab_bwd<R>));
  {
    ProfScope _ps(io.prof, "tab_bwd", st);
    k_tab_bwd<R><<<blocks, 128, smem, st>>>(pc, tc, tab, io.coord, io.perm, io.type, io.nl_j, env, Tm,
                                            gD, io.force, io.atom_virial);
  }
  DP_CUDA_TRY(cudaGetLastError());
  return DP_OK;
}

}  // namespace

int build_tables(DeviceModel& m) {
  const dp_model_config& c = m.cfg;
  if (m.M > 256 || m.A > 32 || m.M < m.A) {
    set_error("compressed path supports M <= 256 and M_< <= 32");
    return DP_E_UNSUPPORTED;
  }
  // s in [0, 1/r_s]: stride 0.01 on the first 90 % of the range, 0.1 on the rest; se_e3 pieces are
  // in theta = R_j . R_k in [0, 2/r_s^2] (|R_j|^2 = 2 s_j^2, 1 + cos >= 0): the same grid scaled by 2/r_s
  const double smax = 1.0 / c.rcut_smth;
  const double scale = c.descriptor == DP_DESC_SE_E3 ? 2.0 / c.rcut_smth : 1.0;
  m.tab.s0 = 0.0;
  m.tab.stride1 = 0.01 * scale;
  m.tab.n1 = (int)std::floor(0.9 * smax / 0.01 + 0.5);
  m.tab.stride2 = 0.1 * scale;
  const double rest = smax - m.tab.n1 * 0.01;
  m.tab.n2 = rest > 0 ? (int)std::ceil(rest / 0.1 - 1e-9) : 1;
  if (m.tab.n2 < 1) m.tab.n2 = 1;
  const TabConst tc = tab_const(m);
  int maxw = 1;
  for (int l = 0; l < c.n_embed; ++l) maxw = std::max(maxw, c.embed[l]);
  const int nets = m.n_embed_nets;
  const size_t nodes = (size_t)nets * (tc.lc + 1) * m.M;
  const size_t ncoef = (size_t)nets * tc.lc * kCoefStride * m.M;
  double *y = nullptr, *y1 = nullptr, *y2 = nullptr;
  LayerDesc* dl = nullptr;
  DP_CUDA_TRY(cudaMalloc(&y, sizeof(double) * nodes * 3));
  y1 = y + nodes;
  y2 = y1 + nodes;
  DP_CUDA_TRY(cudaMalloc(&dl, sizeof(LayerDesc) * m.emb.size()));
  DP_CUDA_TRY(cudaMemcpy(dl, m.emb.data(), sizeof(LayerDesc) * m.emb.size(), cudaMemcpyHostToDevice));
  DP_CUDA_TRY(cudaMalloc(&m.tab64, sizeof(double) * ncoef));
  DP_CUDA_TRY(cudaMalloc(&m.tab32, sizeof(float) * ncoef));
  dim3 grid(tc.lc + 1, nets);
  k_table_nodes<<<grid, 128, sizeof(double) * 6 * maxw>>>(m.p64, dl, c.n_embed, tc, m.M, maxw, y, y1, y2);
  DP_CUDA_TRY(cudaGetLastError());
  const long total = (long)nets * tc.lc * m.M;
  k_table_coef<<<(unsigned)((total + 255) / 256), 256>>>(tc, m.M, nets, y, y1, y2, m.tab64, m.tab32);
  DP_CUDA_TRY(cudaGetLastError());
  DP_CUDA_TRY(cudaDeviceSynchronize());
  cudaFree(y);
  cudaFree(dl);
  if (c.descriptor != DP_DESC_SE_E2_A) return DP_OK;  // the moment path is se_e2_a's
  return build_mom_tables(m);
}

int export_tables(const DeviceModel& m, double* out) {
  if (!m.tab64) {
    set_error("model is not compressed");
    return DP_E_ARG;
  }
  const int lc = m.tab.n1 + m.tab.n2, M = m.M;
  const size_t nrow = (size_t)m.n_embed_nets * lc * M;
  std::vector<double> h(nrow * kCoefStride);
  DP_CUDA_TRY(cudaMemcpy(h.data(), m.tab64, sizeof(double) * h.size(), cudaMemcpyDeviceToHost));
  for (size_t r = 0; r < nrow; ++r)
    for (int q = 0; q < 6; ++q) out[r * 6 + q] = h[r * kCoefStride + q];
  return DP_OK;
}

int run_compressed(const DeviceModel& m, const PathConst& pc, const PathIO& io, Arena& ar, cudaStream_t st) {
  if (m.mom_npass) return run_mom(m, pc, io, ar, st);
  if (m.precision == DP_PREC_FP64) return run_tab<double, double>(m, pc, io, ar, st, m.p64, m.tab64);
  if (m.precision == DP_PREC_BF16) return run_tab<float, __nv_bfloat16>(m, pc, io, ar, st, m.p32, m.tab32);
  return run_tab<float, float>(m, pc, io, ar, st, m.p32, m.tab32);
}

}  // namespace dpgb
