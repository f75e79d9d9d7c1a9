// Fitting-net GEMMs on the 5th-generation tensor cores of GB300 (sm_103a).
//
// One CTA (4 warps) computes a 128 x BN output tile.  Thread 0 streams 128 x 64 (A) and
// BN x 64 (B) BF16 tiles into a 4-stage shared-memory ring with TMA (128-byte swizzle);
// thread 32 issues tcgen05.mma (M = 128, N = BN, K = 16 per instruction) from the ring into
// an FP32 accumulator in tensor memory and releases each stage with tcgen05.commit; after the
// last stage all four warps read their 32 accumulator rows back with tcgen05.ld and apply the
// layer's epilogue (bias, tanh, ResNet skip, the 1 - t^2 gate of the backward pass, the final
// linear layer) in registers, so every layer of the fitting net -- forward and backward --
// is a single launch.  All atom types go into one launch: their rows are contiguous and each
// tile picks its type's weight tensor map.  Every mbarrier wait is bounded: on time-out the
// CTA records an error, waits (bounded) for its outstanding copies, frees its tensor memory
// and returns.
#include <cudaTypedefs.h>

#include <mutex>

#include "tc_gemm.cuh"

namespace dpgb {

namespace {

constexpr int kStages = 4;
constexpr int BM = 128;
constexpr int BK = 64;  // 64 BF16 = 128 bytes = one swizzle atom per row
constexpr long kSpin = 1L << 24;

__device__ __forceinline__ uint32_t su32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* err) {
  for (long it = 0; it < kSpin; ++it)
    if (mbar_try(b, parity)) return true;
  atomicExch(err, 1);
  return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(su32(bar)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle: rows of 128 bytes,
// 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;              // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;              // descriptor version
  d |= (uint64_t)2 << 61;              // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t addr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int EPI>
__global__ void __launch_bounds__(128, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ TcMaps tb, const TcArgs g) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int BN = g.BN;
  const uint32_t a_bytes = BM * BK * 2;
  const uint32_t b_bytes = (uint32_t)BN * BK * 2;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * stage_bytes);
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
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_holder)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ----
    int issued[kStages] = {0, 0, 0, 0};
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kStages;
      if (kb >= kStages && !mbar_wait(&empty[s], ((kb / kStages) - 1) & 1, g.err)) break;
      unsigned char* st = smem + s * stage_bytes;
      mbar_expect_tx(&full[s], stage_bytes);
      tma_load_2d(st, &ta, &full[s], kb * BK, row0);
      tma_load_2d(st + a_bytes, &tb.m[t], &full[s], kb * BK, col0);
      issued[s]++;
    }
    // every copy this thread started has landed before the CTA may exit
    for (int s = 0; s < kStages; ++s)
      if (issued[s] > 0) mbar_wait(&full[s], (issued[s] - 1) & 1, g.err);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kStages;
      if (!mbar_wait(&full[s], (kb / kStages) & 1, g.err)) break;
      tc_fence_after();
      const uint32_t sa = su32(smem + s * stage_bytes);
      const uint64_t ad = sdesc_sw128(sa), bd = sdesc_sw128(sa + a_bytes);
#pragma unroll
      for (int k = 0; k < BK / 16; ++k) mma_bf16(tmem, ad + 2 * k, bd + 2 * k, idesc, (kb | k) != 0);
      mma_commit(&empty[s]);
    }
    mma_commit(accf);
  }
  __syncwarp();

  // ---- epilogue: warp w owns accumulator rows 32w .. 32w+31 ----
  mbar_wait(accf, 0, g.err);
  tc_fence_after();
  const int row = row0 + warp * 32 + lane;
  const bool rv = row < row_end;
  const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
  float e_acc = 0.f;
  for (int c = 0; c < BN; c += 16) {
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
  if (EPI == TC_EPI_FWD_LAST && rv) g.e_out[row] = e_acc + g.b_last[t];
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
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

int tc_pick_bn(int N, int row_tiles, bool full_row) {
  int bn = ((N + 15) / 16) * 16;
  if (bn > 256) bn = 256;
  if (full_row) return bn;
  while (bn > 64 && (long)row_tiles * ((N + bn - 1) / bn) < 2L * 152) bn = ((bn / 2 + 15) / 16) * 16;
  return bn;
}

cudaError_t launch_tc_gemm(int epi, const CUtensorMap& ta, const TcMaps& tb, const TcArgs& a, cudaStream_t st) {
  const int tiles = a.tile_start[a.ntypes];
  if (tiles <= 0) return cudaSuccess;
  dim3 grid(tiles, (a.N + a.BN - 1) / a.BN);
  const size_t smem = (size_t)kStages * (BM * BK * 2 + (size_t)a.BN * BK * 2) + 1024 + 256;
  cudaError_t e = cudaSuccess;
  switch (epi) {
    case TC_EPI_PLAIN:
      e = cudaFuncSetAttribute(k_tc_gemm<TC_EPI_PLAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) k_tc_gemm<TC_EPI_PLAIN><<<grid, 128, smem, st>>>(ta, tb, a);
      break;
    case TC_EPI_FWD:
      e = cudaFuncSetAttribute(k_tc_gemm<TC_EPI_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) k_tc_gemm<TC_EPI_FWD><<<grid, 128, smem, st>>>(ta, tb, a);
      break;
    case TC_EPI_FWD_LAST:
      e = cudaFuncSetAttribute(k_tc_gemm<TC_EPI_FWD_LAST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) k_tc_gemm<TC_EPI_FWD_LAST><<<grid, 128, smem, st>>>(ta, tb, a);
      break;
    default:
      e = cudaFuncSetAttribute(k_tc_gemm<TC_EPI_BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) k_tc_gemm<TC_EPI_BWD><<<grid, 128, smem, st>>>(ta, tb, a);
      break;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace dpgb
