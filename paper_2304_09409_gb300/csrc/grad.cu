// Parameter gradient of an energy + force objective (Sec. II.B, loss function):
//
//   Phi(theta) = sum_f a_f E_f + sum_i w_i . F_i = sum_f a_f E_f - D_w E,
//
// where D_w E is the derivative of E along the coordinate direction w.  For the loss
//   L = (1/B) sum_f [ pE dE_f^2 / N_f + pF sum_i |dF_i|^2 / (3 N_f) ]
// the caller passes a_f = 2 pE dE_f / (N_f B) and w_i = 2 pF dF_i / (3 N_f B), and dPhi/dtheta
// is dL/dtheta.  This is the "double backward" of the force: a tangent pass along w through
// every step (pair geometry, embedding, descriptor, fitting) gives D_w E; a reverse pass over
// both the primal and the tangent computation then gives the gradient with respect to every
// weight and bias.  Everything runs on CUDA cores in the model's precision (FP32 or FP64) with
// accumulation in the same precision; there is no framework autograd underneath.
//
// Dense layer (Eq. (NN)) with tangent:  z = x W + b, t = tanh z, y = t + skip(x)
//                                       zd = xd W,  yd = (1 - t^2) zd + skip(xd)
// reverse, given gy = dPhi/dy and gyd = dPhi/dyd:
//   gzd = gyd (1 - t^2);  gz = (gy - 2 t zd gyd) (1 - t^2)
//   gx = gz W^T + skip^T(gy);  gxd = gzd W^T + skip^T(gyd);  gW += x^T gz + xd^T gzd;  gb += sum gz
#include <cstring>

#include "capi_internal.cuh"
#include "env.cuh"
#include "grad.cuh"

namespace dpgb {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

__device__ __forceinline__ long rowi(const RowMap& m, int r) {
  if (m.kind == 0) return m.r0 + r;
  return (long)(m.p0 + r / m.nk) * m.nc + m.k0 + r % m.nk;
}

inline unsigned nb(long n, int b) { return (unsigned)((n + b - 1) / b); }
inline int net_index(const PathConst& pc, int ti, int tj) { return pc.type_one_side ? tj : ti * pc.ntypes + tj; }

// ---- pair geometry and its tangent along w -----------------------------------------------------
template <class R>
__global__ void k_env_tan(PathConst pc, const double* __restrict__ coord, const double* __restrict__ w,
                          const double* __restrict__ gv, const int* __restrict__ perm, const int* __restrict__ nl_j,
                          const int* __restrict__ nl_code, R* __restrict__ Renv, R* __restrict__ Rdot) {
  const long row = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= (long)pc.natoms * pc.nc) return;
  const int p = (int)(row / pc.nc), k = (int)(row % pc.nc);
  const int i = perm[p];
  const int j = nl_j[(long)i * pc.nc + k];
  R o[4] = {0, 0, 0, 0}, od[4] = {0, 0, 0, 0};
  if (j >= 0) {
    double d0, d1, d2;
    listed_disp(coord + 3 * i, coord + 3 * j, nl_code[(long)i * pc.nc + k], pc, frame_of(pc, i), d0, d1, d2);
    R r, s, ds, u[3];
    pair_env<R>(d0, d1, d2, norm2_exact(d0, d1, d2), pc.rs, pc.rc, pc.near2, r, s, ds, u);
    // dd = (w_j - w_i) + g_f r_ij (the virial seed of the frame: sum_ab g_ab Xi_ab is minus the
    // derivative of E along the homogeneous deformation r_ij -> r_ij + g r_ij); dr = u . dd;
    // du = (dd - dr u) / r; ds/de = s' dr
    double e0 = w[3 * j] - w[3 * i], e1 = w[3 * j + 1] - w[3 * i + 1], e2 = w[3 * j + 2] - w[3 * i + 2];
    if (gv) {
      const double* g = gv + 9L * frame_of(pc, i);
      e0 += g[0] * d0 + g[1] * d1 + g[2] * d2;
      e1 += g[3] * d0 + g[4] * d1 + g[5] * d2;
      e2 += g[6] * d0 + g[7] * d1 + g[8] * d2;
    }
    const R dd[3] = {R(e0), R(e1), R(e2)};
    const R dr = u[0] * dd[0] + u[1] * dd[1] + u[2] * dd[2];
    const R sd = ds * dr;
    o[0] = s;
    od[0] = sd;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const R ud = (dd[a] - dr * u[a]) / r;
      o[1 + a] = s * u[a];
      od[1 + a] = sd * u[a] + s * ud;
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    Renv[row * 4 + a] = o[a];
    Rdot[row * 4 + a] = od[a];
  }
}

// ---- first embedding layer (scalar input), primal and tangent ----------------------------------
template <class R>
__global__ void k_emb0_tan(PathConst pc, NetPtrs<R> nets, const int* __restrict__ tsorted, const R* __restrict__ Renv,
                           const R* __restrict__ Rdot, int w1, int skip, R* __restrict__ Y, R* __restrict__ T,
                           R* __restrict__ Yd, R* __restrict__ Zd) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long nrow = (long)pc.natoms * pc.nc;
  if (e >= nrow * w1) return;
  const long row = e / w1;
  const int o = (int)(e % w1);
  const int p = (int)(row / pc.nc), k = (int)(row % pc.nc);
  const int net = net_of(pc, tsorted[p], slot_block(pc, k));
  const R s = Renv[row * 4], sd = Rdot[row * 4];
  const R wv = nets.w0[net][o];
  const R t = tanh_r(s * wv + nets.b0[net][o]);
  const R zd = sd * wv;
  Y[e] = t + (skip ? s : R(0));
  T[e] = t;
  Zd[e] = zd;
  Yd[e] = (R(1) - t * t) * zd + (skip ? sd : R(0));
}

// ---- dense layer tangent: zd = xd W; yd = (1 - t^2) zd + skip(xd) --------------------------------
template <class R>
__global__ void __launch_bounds__(256)
    k_dense_tan(RowMap rm, const R* __restrict__ Xd, int n_in, const R* __restrict__ W, int n_out, int skip,
                int tanh_act, const R* __restrict__ T, R* __restrict__ Yd, R* __restrict__ Zd) {
  // FP32: the transposed A tile's rows padded to 68 values, so that a thread's four rows (and
  // its four B columns) load as one 16-byte vector each
  __shared__ __align__(16) R As[BK][BM + (sizeof(R) == 4 ? 4 : 1)];
  __shared__ __align__(16) R Bs[BK][BN];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int r0 = blockIdx.x * BM, c0 = blockIdx.y * BN;
  R acc[4][4] = {};
  for (int k0 = 0; k0 < n_in; k0 += BK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + q * 256;
      const int r = e / BK, kk = e % BK;
      As[kk][r] = (r0 + r < rm.nrows && k0 + kk < n_in) ? Xd[rowi(rm, r0 + r) * n_in + k0 + kk] : R(0);
      const int kb = e / BN, cb = e % BN;
      Bs[kb][cb] = (k0 + kb < n_in && c0 + cb < n_out) ? W[(long)(k0 + kb) * n_out + c0 + cb] : R(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      R av[4], bv[4];
      if constexpr (sizeof(R) == 4) {
        const float4 a4 = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
        const float4 b4 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
        av[0] = a4.x; av[1] = a4.y; av[2] = a4.z; av[3] = a4.w;
        bv[0] = b4.x; bv[1] = b4.y; bv[2] = b4.z; bv[3] = b4.w;
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          av[q] = As[kk][ty * 4 + q];
          bv[q] = Bs[kk][tx * 4 + q];
        }
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int r = r0 + ty * 4 + a;
    if (r >= rm.nrows) continue;
    const long row = rowi(rm, r);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = c0 + tx * 4 + b;
      if (c >= n_out) continue;
      const R zd = acc[a][b];
      R yd = zd;
      if (tanh_act) {
        const R t = T[row * n_out + c];
        yd = (R(1) - t * t) * zd;
      }
      if (skip == 1) yd += Xd[row * n_in + c];
      if (skip == 2) yd += Xd[row * n_in + c % n_in];
      Yd[row * n_out + c] = yd;
      if (Zd) Zd[row * n_out + c] = zd;
    }
  }
}

// ---- reverse through tanh: gz, gzd from gy, gyd, t, zd (elementwise) -----------------------------
template <class R>
__global__ void k_rev_tanh(RowMap rm, int n, const R* __restrict__ GY, const R* __restrict__ GYd,
                           const R* __restrict__ T, const R* __restrict__ Zd, R* __restrict__ GZ, R* __restrict__ GZd) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)rm.nrows * n) return;
  const long idx = rowi(rm, (int)(e / n)) * n + e % n;
  const R t = T[idx], g = R(1) - t * t;
  const R gyd = GYd[idx];
  GZd[idx] = gyd * g;
  GZ[idx] = (GY[idx] - R(2) * t * Zd[idx] * gyd) * g;
}

// ---- gx = gz W^T + skip^T(gy) (and the same for the tangent pair) --------------------------------
template <class R>
__global__ void __launch_bounds__(256)
    k_dense_bx(RowMap rm, const R* __restrict__ GZ, const R* __restrict__ GY, int n_in, const R* __restrict__ W,
               int n_out, int skip, R* __restrict__ GX) {
  // FP32: the transposed A tile's rows padded to 68 values, so that a thread's four rows (and
  // its four B columns) load as one 16-byte vector each
  __shared__ __align__(16) R As[BK][BM + (sizeof(R) == 4 ? 4 : 1)];
  __shared__ __align__(16) R Bs[BK][BN];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int r0 = blockIdx.x * BM, c0 = blockIdx.y * BN;
  R acc[4][4] = {};
  for (int k0 = 0; k0 < n_out; k0 += BK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + q * 256;
      const int r = e / BK, kk = e % BK;
      As[kk][r] = (r0 + r < rm.nrows && k0 + kk < n_out) ? GZ[rowi(rm, r0 + r) * n_out + k0 + kk] : R(0);
      const int kb = e / BN, cb = e % BN;
      Bs[kb][cb] = (k0 + kb < n_out && c0 + cb < n_in) ? W[(long)(c0 + cb) * n_out + k0 + kb] : R(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      R av[4], bv[4];
      if constexpr (sizeof(R) == 4) {
        const float4 a4 = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
        const float4 b4 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
        av[0] = a4.x; av[1] = a4.y; av[2] = a4.z; av[3] = a4.w;
        bv[0] = b4.x; bv[1] = b4.y; bv[2] = b4.z; bv[3] = b4.w;
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          av[q] = As[kk][ty * 4 + q];
          bv[q] = Bs[kk][tx * 4 + q];
        }
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int r = r0 + ty * 4 + a;
    if (r >= rm.nrows) continue;
    const long row = rowi(rm, r);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = c0 + tx * 4 + b;
      if (c >= n_in) continue;
      R g = acc[a][b];
      if (skip == 1) g += GY[row * n_out + c];
      if (skip == 2) g += GY[row * n_out + c] + GY[row * n_out + c + n_in];
      GX[row * n_in + c] = g;
    }
  }
}

// ---- weight and bias gradients: gW += X^T GZ + Xd^T GZd, gb += sum_rows GZ ----------------------
// One block owns a TI x TI tile of gW and a slab of rows; partial sums go to gW with atomics.  Each
// thread keeps PT x PT outputs; FP32 takes 4 x 4 with 16-byte shared loads (two loads per eight
// FMAs), FP64 2 x 2 (its pipe, not the loads, is the limit there).
template <class R>
struct WGrad;
template <>
struct WGrad<float> {
  static constexpr int TI = 64, PT = 4, RR = 32, LD = TI + 4;  // rows 16-byte aligned
};
template <>
struct WGrad<double> {
  static constexpr int TI = 32, PT = 2, RR = 32, LD = TI + 1;
};

template <class R>
__global__ void __launch_bounds__(256)
    k_wgrad(RowMap rm, const R* __restrict__ X, const R* __restrict__ Xd, int n_in, const R* __restrict__ GZ,
            const R* __restrict__ GZd, int n_out, int rows_per_block, R* __restrict__ gW, R* __restrict__ gb) {
  constexpr int TI = WGrad<R>::TI, PT = WGrad<R>::PT, RR = WGrad<R>::RR, LD = WGrad<R>::LD;
  __shared__ __align__(16) R xs[RR][LD], xds[RR][LD], gs[RR][LD], gds[RR][LD];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.x * TI, o0 = blockIdx.y * TI;
  const int rbeg = blockIdx.z * rows_per_block;
  const int rend = min(rm.nrows, rbeg + rows_per_block);
  R acc[PT][PT] = {}, bacc[PT] = {};
  for (int r0 = rbeg; r0 < rend; r0 += RR) {
    for (int e = tid; e < RR * TI; e += 256) {
      const int r = e / TI, c = e % TI;
      const bool rv = r0 + r < rend;
      const long row = rv ? rowi(rm, r0 + r) : 0;
      xs[r][c] = (rv && i0 + c < n_in) ? X[row * n_in + i0 + c] : R(0);
      xds[r][c] = (rv && Xd && i0 + c < n_in) ? Xd[row * n_in + i0 + c] : R(0);
      gs[r][c] = (rv && o0 + c < n_out) ? GZ[row * n_out + o0 + c] : R(0);
      gds[r][c] = (rv && GZd && o0 + c < n_out) ? GZd[row * n_out + o0 + c] : R(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < RR; ++r) {
      R xa[PT], xda[PT], ga[PT], gda[PT];
      if constexpr (PT == 4) {
        const float4 x4 = *reinterpret_cast<const float4*>(&xs[r][ty * 4]);
        const float4 xd4 = *reinterpret_cast<const float4*>(&xds[r][ty * 4]);
        const float4 g4 = *reinterpret_cast<const float4*>(&gs[r][tx * 4]);
        const float4 gd4 = *reinterpret_cast<const float4*>(&gds[r][tx * 4]);
        xa[0] = x4.x; xa[1] = x4.y; xa[2] = x4.z; xa[3] = x4.w;
        xda[0] = xd4.x; xda[1] = xd4.y; xda[2] = xd4.z; xda[3] = xd4.w;
        ga[0] = g4.x; ga[1] = g4.y; ga[2] = g4.z; ga[3] = g4.w;
        gda[0] = gd4.x; gda[1] = gd4.y; gda[2] = gd4.z; gda[3] = gd4.w;
      } else {
#pragma unroll
        for (int a = 0; a < PT; ++a) {
          xa[a] = xs[r][ty * PT + a];
          xda[a] = xds[r][ty * PT + a];
          ga[a] = gs[r][tx * PT + a];
          gda[a] = gds[r][tx * PT + a];
        }
      }
#pragma unroll
      for (int a = 0; a < PT; ++a)
#pragma unroll
        for (int b = 0; b < PT; ++b) acc[a][b] += xa[a] * ga[b] + xda[a] * gda[b];
      if (blockIdx.x == 0 && ty == 0)
#pragma unroll
        for (int b = 0; b < PT; ++b) bacc[b] += ga[b];
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < PT; ++a)
#pragma unroll
    for (int b = 0; b < PT; ++b) {
      const int i = i0 + ty * PT + a, o = o0 + tx * PT + b;
      if (i < n_in && o < n_out) atomicAdd(gW + (long)i * n_out + o, acc[a][b]);
    }
  if (blockIdx.x == 0 && ty == 0 && gb)
#pragma unroll
    for (int b = 0; b < PT; ++b) {
      const int o = o0 + tx * PT + b;
      if (o < n_out) atomicAdd(gb + o, bacc[b]);
    }
}

// ---- first embedding layer reverse and its weight/bias gradients (all nets) ----------------------
template <class R>
__global__ void __launch_bounds__(256)
    k_emb0_rev(PathConst pc, const int* __restrict__ tsorted, const R* __restrict__ Renv, const R* __restrict__ Rdot,
               int w1, const R* __restrict__ GY, const R* __restrict__ GYd, const R* __restrict__ T,
               const R* __restrict__ Zd, long rows_per_block, R* __restrict__ grad, NetOffsets off) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  R* acc = reinterpret_cast<R*>(sm_raw);  // [nets][w1][2] (gw, gb)
  const int nets = off.nets;
  for (int e = threadIdx.x; e < nets * w1 * 2; e += blockDim.x) acc[e] = R(0);
  __syncthreads();
  const long nrow = (long)pc.natoms * pc.nc;
  const long beg = blockIdx.x * rows_per_block, end = min(nrow, beg + rows_per_block);
  for (long e = beg * w1 + threadIdx.x; e < end * w1; e += blockDim.x) {
    const long row = e / w1;
    const int o = (int)(e % w1);
    const int p = (int)(row / pc.nc), k = (int)(row % pc.nc);
    const int net = net_of(pc, tsorted[p], slot_block(pc, k));
    const R t = T[e], g = R(1) - t * t;
    const R gyd = GYd[e];
    const R gzd = gyd * g;
    const R gz = (GY[e] - R(2) * t * Zd[e] * gyd) * g;
    const R s = Renv[row * 4], sd = Rdot[row * 4];
    atomicAdd(acc + (net * w1 + o) * 2, s * gz + sd * gzd);
    atomicAdd(acc + (net * w1 + o) * 2 + 1, gz);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nets * w1; e += blockDim.x) {
    const int net = e / w1, o = e % w1;
    atomicAdd(grad + off.w[net] + o, acc[e * 2]);
    atomicAdd(grad + off.w[net] + w1 + o, acc[e * 2 + 1]);
  }
}

// ---- T, Td, D, Dd per atom --------------------------------------------------------------------
template <class R>
__global__ void k_contract_tan(PathConst pc, const R* __restrict__ G, const R* __restrict__ Gd,
                               const R* __restrict__ Renv, const R* __restrict__ Rdot, R* __restrict__ Tm,
                               R* __restrict__ Tmd, R* __restrict__ D, R* __restrict__ Dd) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int M = pc.M, A = pc.A, nc = pc.nc;
  R* Ts = reinterpret_cast<R*>(sm_raw);
  R* Tds = Ts + M * 4;
  const int p = blockIdx.x;
  const R inv = R(1) / R(nc);
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    R a[4] = {0, 0, 0, 0}, ad[4] = {0, 0, 0, 0};
    for (int k = 0; k < nc; ++k) {
      const long row = (long)p * nc + k;
      const R g = G[row * M + m], gd = Gd[row * M + m];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const R rr = Renv[row * 4 + c], rd = Rdot[row * 4 + c];
        a[c] += g * rr;
        ad[c] += gd * rr + g * rd;
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      Ts[m * 4 + c] = a[c] * inv;
      Tds[m * 4 + c] = ad[c] * inv;
      Tm[((long)p * M + m) * 4 + c] = a[c] * inv;
      Tmd[((long)p * M + m) * 4 + c] = ad[c] * inv;
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < M * A; idx += blockDim.x) {
    const int m = idx / A, l = idx % A;
    R v = 0, vd = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      v += Ts[m * 4 + c] * Ts[l * 4 + c];
      vd += Tds[m * 4 + c] * Ts[l * 4 + c] + Ts[m * 4 + c] * Tds[l * 4 + c];
    }
    D[(long)p * M * A + idx] = v;
    Dd[(long)p * M * A + idx] = vd;
  }
}

// ---- dPhi/dT, dPhi/dTd from dPhi/dD, dPhi/dDd; then dPhi/dG, dPhi/dGd per slot -------------------
template <class R>
__global__ void k_descr_rev(PathConst pc, const R* __restrict__ Tm, const R* __restrict__ Tmd,
                            const R* __restrict__ gD, const R* __restrict__ gDd, const R* __restrict__ Renv,
                            const R* __restrict__ Rdot, R* __restrict__ gG, R* __restrict__ gGd) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int M = pc.M, A = pc.A, nc = pc.nc;
  R* Ts = reinterpret_cast<R*>(sm_raw);
  R* Tds = Ts + M * 4;
  R* gTs = Tds + M * 4;
  R* gTds = gTs + M * 4;
  const int p = blockIdx.x;
  for (int e = threadIdx.x; e < M * 4; e += blockDim.x) {
    Ts[e] = Tm[(long)p * M * 4 + e];
    Tds[e] = Tmd[(long)p * M * 4 + e];
  }
  __syncthreads();
  const R* gDp = gD + (long)p * M * A;
  const R* gDdp = gDd + (long)p * M * A;
  for (int e = threadIdx.x; e < M * 4; e += blockDim.x) {
    const int m = e >> 2, c = e & 3;
    R gt = 0, gtd = 0;
    for (int l = 0; l < A; ++l) {
      gt += gDp[m * A + l] * Ts[l * 4 + c] + gDdp[m * A + l] * Tds[l * 4 + c];
      gtd += gDdp[m * A + l] * Ts[l * 4 + c];
    }
    if (m < A)
      for (int q = 0; q < M; ++q) {
        gt += gDp[q * A + m] * Ts[q * 4 + c] + gDdp[q * A + m] * Tds[q * 4 + c];
        gtd += gDdp[q * A + m] * Ts[q * 4 + c];
      }
    gTs[e] = gt;
    gTds[e] = gtd;
  }
  __syncthreads();
  const R inv = R(1) / R(nc);
  for (int e = threadIdx.x; e < nc * M; e += blockDim.x) {
    const int k = e / M, m = e % M;
    const long row = (long)p * nc + k;
    R g = 0, gd = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const R rr = Renv[row * 4 + c], rd = Rdot[row * 4 + c];
      g += gTs[m * 4 + c] * rr + gTds[m * 4 + c] * rd;
      gd += gTds[m * 4 + c] * rr;
    }
    gG[row * M + m] = g * inv;
    gGd[row * M + m] = gd * inv;
  }
}

// ---- last (linear) fitting layer reverse: seeds a_f (energy) and -1 (tangent) ------------------
template <class R>
__global__ void k_fit_last_rev(int n, const int* __restrict__ perm, const int* __restrict__ atom_frame,
                               const double* __restrict__ a_frame, double b, const R* __restrict__ wl, int n_in,
                               R* __restrict__ gx, R* __restrict__ gxd, R* __restrict__ gz, R* __restrict__ gzd) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)n * n_in) return;
  const int p = (int)(e / n_in), c = (int)(e % n_in);
  const int i = perm[p];
  const R a = (R)a_frame[atom_frame ? atom_frame[i] : 0];
  gx[e] = a * wl[c];
  gxd[e] = (R)b * wl[c];
  if (c == 0) {
    gz[p] = a;
    gzd[p] = (R)b;
  }
}

template <class R>
__global__ void k_to_double(const R* __restrict__ x, long n, double* __restrict__ y) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) y[e] = (double)x[e];
}

__global__ void k_types_sorted(const int* __restrict__ type, const int* __restrict__ perm, int n,
                               int* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) out[p] = type[perm[p]];
}

template <class R>
__global__ void k_zero(R* __restrict__ x, long n) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) x[e] = R(0);
}

template <class R>
void launch_wgrad(const RowMap& rm, const R* X, const R* Xd, int n_in, const R* GZ, const R* GZd, int n_out, R* gW,
                  R* gb, cudaStream_t st) {
  if (rm.nrows <= 0) return;
  constexpr int TI = WGrad<R>::TI;
  const long tiles = (long)nb(n_in, TI) * nb(n_out, TI);
  // row slabs of 4096, fewer rows when that leaves under two blocks per SM (small layers)
  int rpb = 4096;
  while (rpb > 512 && tiles * nb(rm.nrows, rpb) < 2L * 152) rpb /= 2;
  dim3 grid(nb(n_in, TI), nb(n_out, TI), nb(rm.nrows, rpb));
  k_wgrad<R><<<grid, 256, 0, st>>>(rm, X, Xd, n_in, GZ, GZd, n_out, rpb, gW, gb);
}

}  // namespace

template <class R>
int run_grad(const DeviceModel& m, const PathConst& pc, const R* params, const PathIO& io, const double* w_dev,
             const double* a_dev, const double* gv_dev, double b, Arena& ar, cudaStream_t st, R** grad_out) {
  const long N = pc.natoms, nc = pc.nc, rows = N * nc;
  const int M = pc.M, A = pc.A, ne = m.cfg.n_embed, nfl = m.n_fit_layers, nt = pc.ntypes;
  // ---- scratch ----
  R* Renv = ar.get<R>(rows * 4);
  R* Rdot = ar.get<R>(rows * 4);
  std::vector<R*> Ye(ne), Te(ne), Yed(ne), Zed(ne);
  int maxe = 1;
  for (int l = 0; l < ne; ++l) {
    const long wl = m.cfg.embed[l];
    maxe = std::max(maxe, (int)wl);
    Ye[l] = ar.get<R>(rows * wl);
    Te[l] = ar.get<R>(rows * wl);
    Yed[l] = ar.get<R>(rows * wl);
    Zed[l] = ar.get<R>(rows * wl);
  }
  R* Tm = ar.get<R>(N * M * 4);
  R* Tmd = ar.get<R>(N * M * 4);
  R* D = ar.get<R>(N * M * A);
  R* Dd = ar.get<R>(N * M * A);
  std::vector<R*> Yf(nfl), Tf(nfl), Yfd(nfl), Zfd(nfl);
  int maxf = M * A;
  for (int l = 0; l < nfl; ++l) {
    const long wl = m.fit[l].n_out;
    maxf = std::max(maxf, (int)wl);
    Yf[l] = ar.get<R>(N * wl);
    Tf[l] = ar.get<R>(N * wl);
    Yfd[l] = ar.get<R>(N * wl);
    Zfd[l] = ar.get<R>(N * wl);
  }
  R* fa = ar.get<R>(N * maxf);
  R* fad = ar.get<R>(N * maxf);
  R* fb = ar.get<R>(N * maxf);
  R* fbd = ar.get<R>(N * maxf);
  R* fz = ar.get<R>(N * maxf);
  R* fzd = ar.get<R>(N * maxf);
  R* ea = ar.get<R>(rows * maxe);
  R* ead = ar.get<R>(rows * maxe);
  R* eb = ar.get<R>(rows * maxe);
  R* ebd = ar.get<R>(rows * maxe);
  R* ez = ar.get<R>(rows * maxe);
  R* ezd = ar.get<R>(rows * maxe);
  int* tsorted = ar.get<int>(N);
  R* grad = ar.get<R>(m.n_params);
  if (ar.measure) return DP_OK;
  if (!ar.ok()) {
    set_error("scratch allocation failed");
    return DP_E_OOM;
  }
  k_zero<R><<<nb(m.n_params, 256), 256, 0, st>>>(grad, m.n_params);
  k_types_sorted<<<nb(N, 256), 256, 0, st>>>(io.type, io.perm, (int)N, tsorted);
  // ---- forward: primal and tangent ----
  {
    ProfScope _ps(io.prof, "grad_env", st);
    k_env_tan<R><<<nb(rows, 256), 256, 0, st>>>(pc, io.coord, w_dev, gv_dev, io.perm, io.nl_j, io.nl_code, Renv,
                                                 Rdot);
  }
  NetPtrs<R> nets;
  NetOffsets off;
  off.nets = m.n_embed_nets;
  for (int n = 0; n < m.n_embed_nets; ++n) {
    const LayerDesc& L0 = m.emb[(size_t)n * ne];
    nets.w0[n] = params + L0.w_off;
    nets.b0[n] = params + L0.w_off + (long)L0.n_in * L0.n_out;
    off.w[n] = L0.w_off;
  }
  const int w1 = m.cfg.embed[0];
  k_emb0_tan<R><<<nb(rows * w1, 256), 256, 0, st>>>(pc, nets, tsorted, Renv, Rdot, w1, m.emb[0].skip, Ye[0], Te[0],
                                                     Yed[0], Zed[0]);
  auto emb_rows = [&](int ti, int tj) {
    return RowMap{1, 0, io.type_start[ti], pc.sel[tj], pc.sel_off[tj], (int)nc,
                  (io.type_start[ti + 1] - io.type_start[ti]) * pc.sel[tj]};
  };
  for (int ti = 0; ti < nt; ++ti)
    for (int tj = 0; tj < nt; ++tj) {
      const int net = net_index(pc, ti, tj);
      const RowMap rm = emb_rows(ti, tj);
      if (rm.nrows <= 0) continue;
      for (int l = 1; l < ne; ++l) {
        const LayerDesc& L = m.emb[(size_t)net * ne + l];
        const R* W = params + L.w_off;
        DP_CUDA_TRY(launch_dense_fwd<R>(rm, Ye[l - 1], L.n_in, W, W + (long)L.n_in * L.n_out, L.n_out, L.skip, 1,
                                        Ye[l], Te[l], st));
        dim3 g(nb(rm.nrows, BM), nb(L.n_out, BN));
        k_dense_tan<R><<<g, 256, 0, st>>>(rm, Yed[l - 1], L.n_in, W, L.n_out, L.skip, 1, Te[l], Yed[l], Zed[l]);
      }
    }
  k_contract_tan<R><<<(unsigned)N, 128, sizeof(R) * M * 8, st>>>(pc, Ye[ne - 1], Yed[ne - 1], Renv, Rdot, Tm, Tmd, D,
                                                                   Dd);
  for (int t = 0; t < nt; ++t) {
    const RowMap rm{0, io.type_start[t], 0, 0, 0, 0, io.type_start[t + 1] - io.type_start[t]};
    if (rm.nrows <= 0) continue;
    const R* X = D;
    const R* Xd = Dd;
    for (int l = 0; l < nfl - 1; ++l) {
      const LayerDesc& L = m.fit[(size_t)t * nfl + l];
      const R* W = params + L.w_off;
      DP_CUDA_TRY(launch_dense_fwd<R>(rm, X, L.n_in, W, W + (long)L.n_in * L.n_out, L.n_out, L.skip, 1, Yf[l], Tf[l],
                                      st));
      dim3 g(nb(rm.nrows, BM), nb(L.n_out, BN));
      k_dense_tan<R><<<g, 256, 0, st>>>(rm, Xd, L.n_in, W, L.n_out, L.skip, 1, Tf[l], Yfd[l], Zfd[l]);
      X = Yf[l];
      Xd = Yfd[l];
    }
  }
  // ---- reverse: fitting net ----
  {
    // per type (the output weights differ): gx = a w, gxd = b w at the last hidden output
    for (int t = 0; t < nt; ++t) {
      const RowMap rm{0, io.type_start[t], 0, 0, 0, 0, io.type_start[t + 1] - io.type_start[t]};
      if (rm.nrows <= 0) continue;
      const LayerDesc& L = m.fit[(size_t)t * nfl + nfl - 1];
      const long r0 = io.type_start[t];
      k_fit_last_rev<R><<<nb((long)rm.nrows * L.n_in, 256), 256, 0, st>>>(
          rm.nrows, io.perm + r0, pc.atom_frame, a_dev, b, params + L.w_off, L.n_in, fa + r0 * L.n_in,
          fad + r0 * L.n_in, fz + r0, fzd + r0);
      // output layer weight/bias gradients: x = last hidden output, gz = a, gzd = b
      const R* X = nfl >= 2 ? Yf[nfl - 2] : D;
      const R* Xd = nfl >= 2 ? Yfd[nfl - 2] : Dd;
      launch_wgrad<R>(rm, X, Xd, L.n_in, fz, fzd, 1, grad + L.w_off, grad + L.w_off + L.n_in, st);
    }
  }
  R* gy = fa;
  R* gyd = fad;
  R* gx = fb;
  R* gxd = fbd;
  for (int l = nfl - 2; l >= 0; --l) {
    for (int t = 0; t < nt; ++t) {
      const RowMap rm{0, io.type_start[t], 0, 0, 0, 0, io.type_start[t + 1] - io.type_start[t]};
      if (rm.nrows <= 0) continue;
      const LayerDesc& L = m.fit[(size_t)t * nfl + l];
      const R* W = params + L.w_off;
      k_rev_tanh<R><<<nb((long)rm.nrows * L.n_out, 256), 256, 0, st>>>(rm, L.n_out, gy, gyd, Tf[l], Zfd[l], fz, fzd);
      dim3 g(nb(rm.nrows, BM), nb(L.n_in, BN));
      k_dense_bx<R><<<g, 256, 0, st>>>(rm, fz, gy, L.n_in, W, L.n_out, L.skip, gx);
      k_dense_bx<R><<<g, 256, 0, st>>>(rm, fzd, gyd, L.n_in, W, L.n_out, L.skip, gxd);
      const R* X = l > 0 ? Yf[l - 1] : D;
      const R* Xd = l > 0 ? Yfd[l - 1] : Dd;
      launch_wgrad<R>(rm, X, Xd, L.n_in, fz, fzd, L.n_out, grad + L.w_off, grad + L.w_off + (long)L.n_in * L.n_out,
                      st);
    }
    std::swap(gy, gx);
    std::swap(gyd, gxd);
  }
  // gy, gyd now hold dPhi/dD, dPhi/dDd
  {
    const size_t sm = sizeof(R) * M * 16;
    k_descr_rev<R><<<(unsigned)N, 128, sm, st>>>(pc, Tm, Tmd, gy, gyd, Renv, Rdot, ea, ead);
  }
  // ---- reverse: embedding nets ----
  R* egy = ea;
  R* egyd = ead;
  R* egx = eb;
  R* egxd = ebd;
  for (int l = ne - 1; l >= 1; --l) {
    for (int ti = 0; ti < nt; ++ti)
      for (int tj = 0; tj < nt; ++tj) {
        const RowMap rm = emb_rows(ti, tj);
        if (rm.nrows <= 0) continue;
        const LayerDesc& L = m.emb[(size_t)net_index(pc, ti, tj) * ne + l];
        const R* W = params + L.w_off;
        k_rev_tanh<R><<<nb((long)rm.nrows * L.n_out, 256), 256, 0, st>>>(rm, L.n_out, egy, egyd, Te[l], Zed[l], ez,
                                                                        ezd);
        dim3 g(nb(rm.nrows, BM), nb(L.n_in, BN));
        k_dense_bx<R><<<g, 256, 0, st>>>(rm, ez, egy, L.n_in, W, L.n_out, L.skip, egx);
        k_dense_bx<R><<<g, 256, 0, st>>>(rm, ezd, egyd, L.n_in, W, L.n_out, L.skip, egxd);
        launch_wgrad<R>(rm, Ye[l - 1], Yed[l - 1], L.n_in, ez, ezd, L.n_out, grad + L.w_off,
                        grad + L.w_off + (long)L.n_in * L.n_out, st);
      }
    std::swap(egy, egx);
    std::swap(egyd, egxd);
  }
  {
    const long rpb = 2048;
    const size_t sm = sizeof(R) * (size_t)m.n_embed_nets * w1 * 2;
    k_emb0_rev<R><<<nb(rows, (int)rpb), 256, sm, st>>>(pc, tsorted, Renv, Rdot, w1, egy, egyd, Te[0], Zed[0], rpb,
                                                      grad, off);
  }
  DP_CUDA_TRY(cudaGetLastError());
  *grad_out = grad;
  return DP_OK;
}

int run_param_grad(const DeviceModel& m, const PathConst& pc, const PathIO& io, const double* w_dev,
                   const double* a_dev, const double* gv_dev, double b, double* grad, Arena& ar, cudaStream_t st) {
  if (m.compressed || (m.precision != DP_PREC_FP64 && m.precision != DP_PREC_FP32)) {
    set_error("parameter gradients need an uncompressed FP64 or FP32 model");
    return DP_E_UNSUPPORTED;
  }
  if (m.precision == DP_PREC_FP64) {
    double* g = nullptr;
    const int rc = run_grad<double>(m, pc, m.p64, io, w_dev, a_dev, gv_dev, b, ar, st, &g);
    if (rc != DP_OK || ar.measure) return rc;
    DP_CUDA_TRY(cudaMemcpyAsync(grad, g, sizeof(double) * m.n_params, cudaMemcpyDeviceToDevice, st));
    return DP_OK;
  }
  float* g = nullptr;
  const int rc = run_grad<float>(m, pc, m.p32, io, w_dev, a_dev, gv_dev, b, ar, st, &g);
  if (rc != DP_OK || ar.measure) return rc;
  k_to_double<float><<<nb(m.n_params, 256), 256, 0, st>>>(g, m.n_params, grad);
  DP_CUDA_TRY(cudaGetLastError());
  return DP_OK;
}

}  // namespace dpgb
