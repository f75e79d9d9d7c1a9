// Fitting-net GEMMs on the 5th-generation tensor cores of GB300 (sm_103a).
//
// One CTA (8 warps) computes a 128 x BN output tile.  Thread 0 streams 128 x 64 (A) and
// BN x 64 (B) BF16 tiles into a shared-memory ring (4 stages for long reductions, 2 for short
// ones so that several CTAs share an SM) with TMA (128-byte swizzle); thread 32 issues
// tcgen05.mma (M = 128, N = BN, K = 16 per instruction) from the ring into an FP32 accumulator
// in tensor memory and releases each stage with tcgen05.commit; after the last stage the eight
// warps read the accumulator back with tcgen05.ld (two warps per 32-row lane quadrant, taking
// alternate 16-column chunks) and apply the layer's epilogue (bias, tanh, ResNet skip, the
// 1 - t^2 gate of the backward pass, the final linear layer) in registers, so every layer of
// the fitting net -- forward and backward -- is a single launch.  All atom types go into one launch: their rows are contiguous and each
// tile picks its type's weight tensor map.  Every mbarrier wait is bounded: on time-out the
// CTA records an error, waits (bounded) for its outstanding copies, frees its tensor memory
// and returns.
#include <cudaTypedefs.h>

#include <mutex>

#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace dpgb {

namespace {

constexpr int kStages = 4;  // ring stages at most
constexpr int kThreads = 256;
constexpr int BM = 128;
constexpr int BK = 64;  // 64 BF16 = 128 bytes = one swizzle atom per row

using namespace ptx;

__host__ __device__ inline int ring_stages(int K) { return (K + BK - 1) / BK >= 8 ? kStages : 2; }

template <int EPI>
__global__ void __launch_bounds__(kThreads)
    k_tc_gemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ TcMaps tb, const TcArgs g) {
  __shared__ float s_e[2][BM];  // FWD_LAST: energy partial of each row from each column half
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int BN = g.BN;
  const uint32_t a_bytes = BM * BK * 2;
  const uint32_t b_bytes = (uint32_t)BN * BK * 2;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  const int NS = ring_stages(g.K);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NS * stage_bytes);
  uint64_t* empty = full + kStages;
  uint64_t* accf = empty + kStages;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(accf + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int t = 0;
  while (t + 1 < g.ntypes && (int)blockIdx.x >= g.tile_start[t + 1]) ++t;
  const int row0 = g.row_start[t] + ((int)blockIdx.x - g.tile_start[t]) * BM;
  const int row_end = g.row_start[t + 1];
  const int col0 = blockIdx.y * BN;
  const int nk = (g.K + BK - 1) / BK;
  uint32_t ncols = 32;
  while ((int)ncols < BN) ncols <<= 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    mbar_fence_init();
  }
  if (warp == 0) {
    tmem_alloc(tmem_holder, ncols);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ----
    int nissued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % NS;
      if (kb >= NS && !mbar_wait(&empty[s], ((kb / NS) - 1) & 1, g.err)) break;
      unsigned char* st = smem + s * stage_bytes;
      mbar_expect_tx(&full[s], stage_bytes);
      tma_load_2d(st, &ta, &full[s], kb * BK, row0);
      tma_load_2d(st + a_bytes, &tb.m[t], &full[s], kb * BK, col0);
      nissued = kb + 1;
    }
    // every copy this thread started has landed before the CTA may exit: the last block issued
    // to stage s is s + NS * ((nissued - 1 - s) / NS)
    for (int s = 0; s < NS && s < nissued; ++s) {
      const int last = s + NS * ((nissued - 1 - s) / NS);
      mbar_wait(&full[s], (last / NS) & 1, g.err);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    const uint32_t idesc = idesc_f16(BM, BN, 1);
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % NS;
      if (!mbar_wait(&full[s], (kb / NS) & 1, g.err)) break;
      tc_fence_after();
      const uint32_t sa = su32(smem + s * stage_bytes);
      const uint64_t ad = sdesc_sw128(sa), bd = sdesc_sw128(sa + a_bytes);
#pragma unroll
      for (int k = 0; k < BK / 16; ++k) mma_f16(tmem, ad + 2 * k, bd + 2 * k, idesc, (kb | k) != 0);
      mma_commit(&empty[s]);
    }
    mma_commit(accf);
  }
  __syncwarp();

  // ---- epilogue: warps w and w + 4 own accumulator rows 32(w % 4) .. +31, alternate chunks ----
  mbar_wait(accf, 0, g.err);
  tc_fence_after();
  const int quad = warp & 3, half = warp >> 2;
  const int row = row0 + quad * 32 + lane;
  const bool rv = row < row_end;
  const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16);
  float e_acc = 0.f;
  for (int c = half * 16; c < BN; c += 32) {
    float v[16];
    tmem_ld16(tbase + c, v);
    const int cb = col0 + c;
    if (!rv || cb >= g.N) continue;
    const long ro = (long)row * g.N;
    // rows of 16-byte-aligned chunks take vector loads/stores; a ragged last chunk goes scalar
    const bool vec = (cb + 16 <= g.N) && ((g.N & 7) == 0);
    float o[16], aux[16];
    if (EPI == TC_EPI_PLAIN) {
#pragma unroll
      for (int i = 0; i < 16; ++i) o[i] = v[i];
    } else if (EPI == TC_EPI_FWD || EPI == TC_EPI_FWD_LAST) {
      float sk[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) sk[i] = 0.f;
      if (g.skip_kind && vec && (g.skip_ld & 15) == 0) {
        const int sc = (g.skip_kind == 1) ? cb : (cb % g.skip_ld);
        const float4* s4 = reinterpret_cast<const float4*>(g.skip_mat + (long)row * g.skip_ld + sc);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 x = s4[q];
          sk[4 * q] = x.x;
          sk[4 * q + 1] = x.y;
          sk[4 * q + 2] = x.z;
          sk[4 * q + 3] = x.w;
        }
      } else if (g.skip_kind) {
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (cb + i < g.N)
            sk[i] = g.skip_mat[(long)row * g.skip_ld + (g.skip_kind == 1 ? cb + i : (cb + i) % g.skip_ld)];
      }
      const float* bias = g.bias[t];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int col = cb + i < g.N ? cb + i : g.N - 1;
        const float th = tanhf(v[i] + bias[col]);
        if (EPI == TC_EPI_FWD) {
          o[i] = th + sk[i];
          aux[i] = th;
        } else {
          const float wl = g.w_last[t][col];
          if (cb + i < g.N) e_acc += (th + sk[i]) * wl;
          aux[i] = wl * (1.f - th * th);
        }
      }
    } else {  // TC_EPI_BWD
      float tb[16];
      if (vec) {
        const float4* t4 = reinterpret_cast<const float4*>(g.tact + ro + cb);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 x = t4[q];
          tb[4 * q] = x.x;
          tb[4 * q + 1] = x.y;
          tb[4 * q + 2] = x.z;
          tb[4 * q + 3] = x.w;
        }
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) tb[i] = cb + i < g.N ? g.tact[ro + cb + i] : 0.f;
      }
      const float* sv = g.skip_vec ? g.w_last[t] : (g.skip_mat ? g.skip_mat + (long)row * g.skip_ld : nullptr);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int col = cb + i < g.N ? cb + i : g.N - 1;
        float gy = v[i];
        if (sv) {
          if (g.skip_kind == 1) gy += sv[col];
          if (g.skip_kind == 2) gy += sv[col] + sv[col + g.N];
        }
        o[i] = gy;
        aux[i] = gy * (1.f - tb[i] * tb[i]);
      }
    }
    // ---- stores ----
    float* of = (EPI == TC_EPI_FWD_LAST) ? nullptr : g.out_f32;
    float* ot = (EPI == TC_EPI_FWD) ? g.out_t : nullptr;
    const float* bsrc = (EPI == TC_EPI_FWD) ? o : aux;  // values stored as BF16
    if (vec) {
      if (of) {
        float4* d4 = reinterpret_cast<float4*>(of + ro + cb);
#pragma unroll
        for (int q = 0; q < 4; ++q) d4[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
      }
      if (ot) {
        float4* d4 = reinterpret_cast<float4*>(ot + ro + cb);
#pragma unroll
        for (int q = 0; q < 4; ++q) d4[q] = make_float4(aux[4 * q], aux[4 * q + 1], aux[4 * q + 2], aux[4 * q + 3]);
      }
      if (EPI != TC_EPI_PLAIN) {
        uint4 pk[2];
        uint32_t* w = reinterpret_cast<uint32_t*>(pk);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const __nv_bfloat162 h2 = __floats2bfloat162_rn(bsrc[2 * q], bsrc[2 * q + 1]);
          w[q] = *reinterpret_cast<const uint32_t*>(&h2);
        }
        uint4* d = reinterpret_cast<uint4*>(g.out_bf16 + ro + cb);
        d[0] = pk[0];
        d[1] = pk[1];
      }
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        if (cb + i >= g.N) break;
        if (of) of[ro + cb + i] = o[i];
        if (ot) ot[ro + cb + i] = aux[i];
        if (EPI != TC_EPI_PLAIN) g.out_bf16[ro + cb + i] = __float2bfloat16_rn(bsrc[i]);
      }
    }
  }
  if (EPI == TC_EPI_FWD_LAST) s_e[half][quad * 32 + lane] = e_acc;
  tc_fence_before();
  __syncthreads();
  if (EPI == TC_EPI_FWD_LAST && half == 0 && rv)
    g.e_out[(long)blockIdx.y * g.e_ld + row] =
        s_e[0][quad * 32 + lane] + s_e[1][quad * 32 + lane] + (blockIdx.y == 0 ? g.b_last[t] : 0.f);
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_encode_mu;

}  // namespace

int make_tmap_bf16(CUtensorMap* map, const void* base, long rows, long cols, int box_rows) {
  {
    std::lock_guard<std::mutex> lk(g_encode_mu);
    if (!g_encode) {
      cudaDriverEntryPointQueryResult q;
      void* fn = nullptr;
      cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
      if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return DP_E_CUDA;
      }
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
  }
  if ((cols * 2) % 16 != 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0 || box_rows < 1 || box_rows > 256) {
    set_error("tensor map: row pitch and base must be 16-byte aligned, box rows in [1, 256]");
    return DP_E_UNSUPPORTED;
  }
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(cols * 2)};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return DP_E_CUDA;
  }
  return DP_OK;
}

int tc_pick_bn(int N, int row_tiles) {
  int bn = ((N + 15) / 16) * 16;
  if (bn > 256) bn = 256;
  while (bn > 64 && (long)row_tiles * ((N + bn - 1) / bn) < 2L * 152) bn = ((bn / 2 + 15) / 16) * 16;
  return bn;
}

cudaError_t launch_tc_gemm(int epi, const CUtensorMap& ta, const TcMaps& tb, const TcArgs& a, cudaStream_t st) {
  const int tiles = a.tile_start[a.ntypes];
  if (tiles <= 0) return cudaSuccess;
  dim3 grid(tiles, (a.N + a.BN - 1) / a.BN);
  const size_t smem = (size_t)ring_stages(a.K) * (BM * BK * 2 + (size_t)a.BN * BK * 2) + 1024 + 256;
  cudaError_t e = cudaSuccess;
  switch (epi) {
    case TC_EPI_PLAIN:
      e = cudaFuncSetAttribute(k_tc_gemm<TC_EPI_PLAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) k_tc_gemm<TC_EPI_PLAIN><<<grid, kThreads, smem, st>>>(ta, tb, a);
      break;
    case TC_EPI_FWD:
      e = cudaFuncSetAttribute(k_tc_gemm<TC_EPI_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) k_tc_gemm<TC_EPI_FWD><<<grid, kThreads, smem, st>>>(ta, tb, a);
      break;
    case TC_EPI_FWD_LAST:
      e = cudaFuncSetAttribute(k_tc_gemm<TC_EPI_FWD_LAST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) k_tc_gemm<TC_EPI_FWD_LAST><<<grid, kThreads, smem, st>>>(ta, tb, a);
      break;
    default:
      e = cudaFuncSetAttribute(k_tc_gemm<TC_EPI_BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) k_tc_gemm<TC_EPI_BWD><<<grid, kThreads, smem, st>>>(ta, tb, a);
      break;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace dpgb
