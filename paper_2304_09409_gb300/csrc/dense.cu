// Dense layer of Eq. (NN) on CUDA cores, forward and input-gradient, for FP64 and FP32.
//
//   forward : Y = phi(X W + b) + skip(X)      (skip: none, +x, +{x,x}); Tact = phi(X W + b)
//   backward: GX = (GY * phi'(.)) W^T + skip^T(GY),   phi' = 1 - Tact^2 for tanh
//
// Rows are either a contiguous range or a (atom range) x (type block of slots) window of the
// [N, Nc] slot matrix, so one launch covers all rows that share one embedding net.  A 64x64
// output tile per 256-thread block, 4x4 outputs per thread, K staged through shared memory
// in chunks of 16.  The FP64 pipe of GB300 is narrow, so this simple tiling already keeps it
// the limiter; the mixed-precision path uses the tensor-core kernels instead.
#include "dp_internal.cuh"

namespace dpgb {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

__device__ __forceinline__ long row_index(const RowMap& m, int r) {
  if (m.kind == 0) return m.r0 + r;
  return (long)(m.p0 + r / m.nk) * m.nc + m.k0 + r % m.nk;
}

// A row whose environment row has s = 0 (padding slot), when the map carries environment rows.
template <class R>
__device__ __forceinline__ bool zero_row(const RowMap& m, long row) {
  return m.zrow != nullptr && reinterpret_cast<const R*>(m.zrow)[row * 4] == R(0);
}
// True for every thread when the block's BM rows from r0 are all zero rows (a tile of padding).
template <class R>
__device__ __forceinline__ bool zero_tile(const RowMap& m, int r0) {
  if (m.zrow == nullptr) return false;
  const int r = r0 + (int)threadIdx.x;
  const bool live = threadIdx.x < BM && r < m.nrows && !zero_row<R>(m, row_index(m, r));
  return !__syncthreads_or(live);
}

__device__ __forceinline__ double act_tanh(double z) { return tanh(z); }
__device__ __forceinline__ float act_tanh(float z) { return tanhf(z); }

template <class R>
__global__ void __launch_bounds__(256)
    k_dense_fwd(RowMap rm, const R* __restrict__ X, int n_in, const R* __restrict__ W, const R* __restrict__ b,
                int n_out, int skip, int tanh_act, R* __restrict__ Y, R* __restrict__ Tact) {
  // FP32: the transposed A tile's rows padded to 68 values, so that a thread's four rows (and
  // its four B columns) load as one 16-byte vector each
  __shared__ __align__(16) R As[BK][BM + (sizeof(R) == 4 ? 4 : 1)];
  __shared__ __align__(16) R Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int r0 = blockIdx.x * BM, c0 = blockIdx.y * BN;
  if (zero_tile<R>(rm, r0)) return;  // block-uniform
  R acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = R(0);
  for (int k0 = 0; k0 < n_in; k0 += BK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int e = tid + q * 256;  // 0..1023
      int r = e / BK, kk = e % BK;
      R v = R(0);
      if (r0 + r < rm.nrows && k0 + kk < n_in) v = X[row_index(rm, r0 + r) * n_in + k0 + kk];
      As[kk][r] = v;
      int kb = e / BN, cb = e % BN;
      R w = R(0);
      if (k0 + kb < n_in && c0 + cb < n_out) w = W[(long)(k0 + kb) * n_out + c0 + cb];
      Bs[kb][cb] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      R a[4], bb[4];
      if constexpr (sizeof(R) == 4) {
        const float4 av = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
        const float4 bv = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
        a[0] = av.x; a[1] = av.y; a[2] = av.z; a[3] = av.w;
        bb[0] = bv.x; bb[1] = bv.y; bb[2] = bv.z; bb[3] = bv.w;
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          a[q] = As[kk][ty * 4 + q];
          bb[q] = Bs[kk][tx * 4 + q];
        }
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] += a[p] * bb[q];
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int r = r0 + ty * 4 + p;
    if (r >= rm.nrows) continue;
    const long row = row_index(rm, r);
    if (zero_row<R>(rm, row)) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = c0 + tx * 4 + q;
      if (c >= n_out) continue;
      R z = acc[p][q] + b[c];
      R t = tanh_act ? act_tanh(z) : z;
      R y = t;
      if (skip == 1) y += X[row * n_in + c];
      if (skip == 2) y += X[row * n_in + (c % n_in)];
      Y[row * n_out + c] = y;
      if (Tact) Tact[row * n_out + c] = t;
    }
  }
}

template <class R>
__global__ void __launch_bounds__(256)
    k_dense_bwd(RowMap rm, const R* __restrict__ GY, const R* __restrict__ Tact, int n_in,
                const R* __restrict__ W, int n_out, int skip, R* __restrict__ GX) {
  // FP32: the transposed A tile's rows padded to 68 values, so that a thread's four rows (and
  // its four B columns) load as one 16-byte vector each
  __shared__ __align__(16) R As[BK][BM + (sizeof(R) == 4 ? 4 : 1)];
  __shared__ __align__(16) R Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int r0 = blockIdx.x * BM, c0 = blockIdx.y * BN;  // columns are input features
  if (zero_tile<R>(rm, r0)) return;  // block-uniform
  R acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = R(0);
  for (int k0 = 0; k0 < n_out; k0 += BK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int e = tid + q * 256;
      int r = e / BK, kk = e % BK;
      R v = R(0);
      if (r0 + r < rm.nrows && k0 + kk < n_out) {
        long idx = row_index(rm, r0 + r) * n_out + k0 + kk;
        v = GY[idx];
        if (Tact) {
          R t = Tact[idx];
          v *= (R(1) - t * t);
        }
      }
      As[kk][r] = v;
      int kb = e / BN, cb = e % BN;
      R w = R(0);
      if (k0 + kb < n_out && c0 + cb < n_in) w = W[(long)(c0 + cb) * n_out + k0 + kb];
      Bs[kb][cb] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      R a[4], bb[4];
      if constexpr (sizeof(R) == 4) {
        const float4 av = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
        const float4 bv = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
        a[0] = av.x; a[1] = av.y; a[2] = av.z; a[3] = av.w;
        bb[0] = bv.x; bb[1] = bv.y; bb[2] = bv.z; bb[3] = bv.w;
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          a[q] = As[kk][ty * 4 + q];
          bb[q] = Bs[kk][tx * 4 + q];
        }
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] += a[p] * bb[q];
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int r = r0 + ty * 4 + p;
    if (r >= rm.nrows) continue;
    const long row = row_index(rm, r);
    if (zero_row<R>(rm, row)) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = c0 + tx * 4 + q;
      if (c >= n_in) continue;
      R g = acc[p][q];
      if (skip == 1) g += GY[row * n_out + c];
      if (skip == 2) g += GY[row * n_out + c] + GY[row * n_out + c + n_in];
      GX[row * n_in + c] = g;
    }
  }
}

}  // namespace

template <class R>
cudaError_t launch_dense_fwd(const RowMap& rm, const R* X, int n_in, const R* W, const R* b, int n_out, int skip,
                             int tanh_act, R* Y, R* Tact, cudaStream_t st) {
  if (rm.nrows <= 0) return cudaSuccess;
  dim3 grid((rm.nrows + BM - 1) / BM, (n_out + BN - 1) / BN);
  k_dense_fwd<R><<<grid, 256, 0, st>>>(rm, X, n_in, W, b, n_out, skip, tanh_act, Y, Tact);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_dense_bwd(const RowMap& rm, const R* GY, const R* Tact, int n_in, const R* W, int n_out,
                             int skip, R* GX, cudaStream_t st) {
  if (rm.nrows <= 0) return cudaSuccess;
  dim3 grid((rm.nrows + BM - 1) / BM, (n_in + BN - 1) / BN);
  k_dense_bwd<R><<<grid, 256, 0, st>>>(rm, GY, Tact, n_in, W, n_out, skip, GX);
  return cudaGetLastError();
}

template cudaError_t launch_dense_fwd<double>(const RowMap&, const double*, int, const double*, const double*, int,
                                              int, int, double*, double*, cudaStream_t);
template cudaError_t launch_dense_fwd<float>(const RowMap&, const float*, int, const float*, const float*, int, int,
                                             int, float*, float*, cudaStream_t);
template cudaError_t launch_dense_bwd<double>(const RowMap&, const double*, const double*, int, const double*, int,
                                              int, double*, cudaStream_t);
template cudaError_t launch_dense_bwd<float>(const RowMap&, const float*, const float*, int, const float*, int, int,
                                             float*, cudaStream_t);

}  // namespace dpgb
