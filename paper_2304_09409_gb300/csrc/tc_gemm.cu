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

// Ring depth: kStages for long reductions, two for short ones so that several CTAs (and their
// epilogues) share an SM.  Split operands (NP = 3) carry high and low parts of both tiles per
// stage (48 KB at BN = 64): two stages, so that two CTAs share an SM and one's epilogue runs
// while the other's operands stream in.
__host__ __device__ inline uint32_t stage_bytes_of(int BN, int NP) {
  return (uint32_t)(NP == 3 ? 2 : 1) * (uint32_t)(BM * BK * 2 + BN * BK * 2);
}
__host__ __device__ inline int ring_stages(int K, int BN, int NP) {
  if (NP == 3) return 2;
  return (K + BK - 1) / BK >= 8 ? kStages : 2;
}

// Shared-memory staging of the epilogue (all but the plain epilogue): FP32 tiles [128][BN] as
// 32-column boxes of 16 KB laid out by the TMA 128-byte swizzle (row r at r * 128 B, 16-byte
// chunk q at position q ^ (r & 7)), so a thread that owns a row reads and writes its 16-byte
// chunks without bank conflicts; BF16 tiles as 64-column boxes of the same layout.
//   slot 0: the skip input (in place: the FP32 output y or g), slot 1: tanh output t (forward)
//   or the gate input t_below (backward), then the BF16 output (split operands: its high part,
//   then its low part).
__host__ __device__ inline uint32_t epi_f32_bytes(int BN) { return (uint32_t)(BN / 32) * 16384u; }
__host__ __device__ inline uint32_t epi_bf16_bytes(int BN) { return (uint32_t)((BN + 63) / 64) * 16384u; }
__host__ __device__ inline uint32_t epi_bytes(int epi, int BN, int NP) {
  if (epi == TC_EPI_PLAIN) return 0;
  const uint32_t f = epi_f32_bytes(BN), h = epi_bf16_bytes(BN) * (NP == 3 ? 2u : 1u);
  return epi == TC_EPI_FWD_LAST ? f + h : 2 * f + h;
}
__device__ __forceinline__ uint32_t sw_off(int r, int q) { return (uint32_t)(r * 128 + ((q ^ (r & 7)) << 4)); }

// High and low BF16 parts of x (x = hi + lo up to the rounding of lo).
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

template <int EPI, int NP>
__global__ void __launch_bounds__(kThreads)
    k_tc_gemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ TcMaps tb,
              const __grid_constant__ TcEpiMaps em, const TcArgs g, const __grid_constant__ TcLo lo) {
  __shared__ float s_e[2][BM];  // FWD_LAST: energy partial of each row from each column half
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int BN = g.BN;
  const uint32_t a_bytes = BM * BK * 2;
  const uint32_t b_bytes = (uint32_t)BN * BK * 2;
  const uint32_t stage_bytes = stage_bytes_of(BN, NP);  // [A hi | B hi (| A lo | B lo)]
  const int NS = ring_stages(g.K, BN, NP);
  const uint32_t ring = (uint32_t)NS * stage_bytes, ep = epi_bytes(EPI, BN, NP);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (ring > ep ? ring : ep));
  uint64_t* empty = full + kStages;
  uint64_t* accf = empty + kStages;
  uint64_t* efull = accf + 1;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(efull + 1);
  unsigned char* S0 = smem;                           // epilogue slots reuse the ring
  unsigned char* S1 = smem + epi_f32_bytes(BN);
  unsigned char* SB = smem + (EPI == TC_EPI_FWD_LAST ? 1 : 2) * epi_f32_bytes(BN);
  unsigned char* SBL = SB + epi_bf16_bytes(BN);  // split operands: low part of the BF16 output

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int t = 0;
  while (t + 1 < g.ntypes && (int)blockIdx.x >= g.tile_start[t + 1]) ++t;
  const int row0 = g.row_start[t] + ((int)blockIdx.x - g.tile_start[t]) * BM;
  const int row_end = g.row_start[t + 1];
  const int col0 = blockIdx.y * BN;
  const int nk = (g.K + BK - 1) / BK;
  uint32_t ncols = 32;
  while ((int)ncols < BN) ncols <<= 1;
  const bool has_skip = (EPI != TC_EPI_PLAIN) && g.skip_kind == 1 && g.skip_mat != nullptr;
  const bool has_tact = (EPI == TC_EPI_BWD);
  const int nb = BN / 32;  // 32-column boxes

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    mbar_init(efull, 1);
    mbar_fence_init();
  }
  if (warp == 0) tmem_alloc(tmem_holder, ncols);
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
      if (NP == 3) {
        tma_load_2d(st + a_bytes + b_bytes, &lo.a, &full[s], kb * BK, row0);
        tma_load_2d(st + 2 * a_bytes + b_bytes, &lo.b.m[t], &full[s], kb * BK, col0);
      }
      nissued = kb + 1;
    }
    // every copy this thread started has landed before the CTA may exit: the last block issued
    // to stage s is s + NS * ((nissued - 1 - s) / NS)
    for (int s = 0; s < NS && s < nissued; ++s) {
      const int last = s + NS * ((nissued - 1 - s) / NS);
      mbar_wait(&full[s], (last / NS) & 1, g.err);
    }
    // epilogue inputs into the ring once the MMAs have read it
    if (has_skip || has_tact) {
      bool ok = mbar_wait(accf, 0, g.err);
      tc_fence_after();
      if (ok) {
        mbar_expect_tx(efull, (uint32_t)((has_skip ? 1 : 0) + (has_tact ? 1 : 0)) * epi_f32_bytes(BN));
        for (int b = 0; b < nb; ++b) {
          if (has_skip) tma_load_2d(S0 + b * 16384, &em.skip, efull, col0 + 32 * b, row0);
          if (has_tact) tma_load_2d(S1 + b * 16384, &em.tact, efull, col0 + 32 * b, row0);
        }
        mbar_wait(efull, 0, g.err);
      } else {
        mbar_arrive(efull);  // release the epilogue of a failed CTA
      }
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
      const uint64_t adl = sdesc_sw128(sa + a_bytes + b_bytes), bdl = sdesc_sw128(sa + 2 * a_bytes + b_bytes);
#pragma unroll
      for (int k = 0; k < BK / 16; ++k) {
        if (NP == 3) {  // small terms first: lo.hi, hi.lo, then hi.hi
          mma_f16(tmem, adl + 2 * k, bd + 2 * k, idesc, (kb | k) != 0);
          mma_f16(tmem, ad + 2 * k, bdl + 2 * k, idesc, 1);
          mma_f16(tmem, ad + 2 * k, bd + 2 * k, idesc, 1);
        } else {
          mma_f16(tmem, ad + 2 * k, bd + 2 * k, idesc, (kb | k) != 0);
        }
      }
      mma_commit(&empty[s]);
    }
    mma_commit(accf);
  }
  __syncwarp();

  // ---- epilogue: warps w and w + 4 own accumulator rows 32(w % 4) .. +31 ----
  mbar_wait(accf, 0, g.err);
  tc_fence_after();
  const int quad = warp & 3, half = warp >> 2;
  const int rl = quad * 32 + lane;  // row within the tile
  const int row = row0 + rl;
  const bool rv = row < row_end;
  const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16);
  float e_acc = 0.f;
  if (EPI == TC_EPI_PLAIN) {
    for (int c = half * 16; c < BN; c += 32) {
      float v[16];
      tmem_ld16(tbase + c, v);
      const int cb = col0 + c;
      if (!rv || cb >= g.N) continue;
      if (g.out_bf16) {  // BF16 output, tile-blocked (8-column groups, rows of the tile contiguous)
        const int nr = min(BM, row_end - row0);
        __nv_bfloat16* tile = g.out_bf16 + (long)row0 * g.N;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int col = cb + i;
          if (col < g.N) tile[((long)(col >> 3) * nr + (row - row0)) * 8 + (col & 7)] = __float2bfloat16_rn(v[i]);
        }
        continue;
      }
      float* dst = g.out_f32 + (long)row * g.N + cb;
      if (cb + 16 <= g.N && (g.N & 3) == 0) {
        float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
        for (int q = 0; q < 4; ++q) d4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (cb + i < g.N) dst[i] = v[i];
      }
    }
  } else {
    if (has_skip || has_tact) mbar_wait(efull, 0, g.err);
    const float* bias = g.bias[t];
    const float* sv = (EPI == TC_EPI_BWD && g.skip_vec) ? g.w_last[t] : nullptr;
    for (int b = half; b < nb; b += 2) {  // one 32-column box at a time
      float v[32];
      {
        uint32_t raw[32];
        tmem_ld16_async(tbase + 32 * b, raw);
        tmem_ld16_async(tbase + 32 * b + 16, raw + 16);
        tmem_wait_ld();
#pragma unroll
        for (int e = 0; e < 32; ++e) v[e] = __uint_as_float(raw[e]);
      }
      unsigned char* s0 = S0 + b * 16384;
      unsigned char* s1 = S1 + b * 16384;
      float o[32], aux[32];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float4 x0 = make_float4(0.f, 0.f, 0.f, 0.f), x1 = x0;
        if (has_skip) x0 = *reinterpret_cast<const float4*>(s0 + sw_off(rl, q));
        if (has_tact) x1 = *reinterpret_cast<const float4*>(s1 + sw_off(rl, q));
        const float sk[4] = {x0.x, x0.y, x0.z, x0.w}, tb4[4] = {x1.x, x1.y, x1.z, x1.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int i = 4 * q + k;
          const int col = min(col0 + 32 * b + i, g.N - 1);
          if (EPI == TC_EPI_FWD || EPI == TC_EPI_FWD_LAST) {
            const float th = tanhf(v[i] + __ldg(bias + col));
            if (EPI == TC_EPI_FWD) {
              o[i] = th + sk[k];
              aux[i] = th;
            } else {
              const float wl = __ldg(g.w_last[t] + col);
              if (col0 + 32 * b + i < g.N) e_acc += (th + sk[k]) * wl;
              aux[i] = wl * (1.f - th * th);
            }
          } else {  // BWD
            float gy = v[i] + sk[k];
            if (sv) gy += __ldg(sv + col);
            o[i] = gy;
            aux[i] = gy * (1.f - tb4[k] * tb4[k]);
          }
        }
      }
      // FP32 outputs in place, BF16 output into its own box
      if (EPI == TC_EPI_FWD || (EPI == TC_EPI_BWD && g.out_f32)) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
          *reinterpret_cast<float4*>(s0 + sw_off(rl, q)) = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
      }
      if (EPI == TC_EPI_FWD) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
          *reinterpret_cast<float4*>(s1 + sw_off(rl, q)) =
              make_float4(aux[4 * q], aux[4 * q + 1], aux[4 * q + 2], aux[4 * q + 3]);
      }
      const float* bsrc = (EPI == TC_EPI_FWD) ? o : aux;
      unsigned char* sb = SB + (b >> 1) * 16384;
      unsigned char* sbl = SBL + (b >> 1) * 16384;
#pragma unroll
      for (int k = 0; k < 4; ++k) {  // 8 BF16 per 16-byte chunk
        uint32_t w[4], wl[4];
#pragma unroll
        for (int h2 = 0; h2 < 4; ++h2) {
          __nv_bfloat162 pr, pl;
          if (NP == 3) {
            split_bf16(bsrc[8 * k + 2 * h2], pr.x, pl.x);
            split_bf16(bsrc[8 * k + 2 * h2 + 1], pr.y, pl.y);
            wl[h2] = *reinterpret_cast<const uint32_t*>(&pl);
          } else {
            pr = __floats2bfloat162_rn(bsrc[8 * k + 2 * h2], bsrc[8 * k + 2 * h2 + 1]);
          }
          w[h2] = *reinterpret_cast<const uint32_t*>(&pr);
        }
        *reinterpret_cast<uint4*>(sb + sw_off(rl, 4 * (b & 1) + k)) = make_uint4(w[0], w[1], w[2], w[3]);
        if (NP == 3)
          *reinterpret_cast<uint4*>(sbl + sw_off(rl, 4 * (b & 1) + k)) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
      }
    }
  }
  if (EPI == TC_EPI_FWD_LAST) s_e[half][rl] = e_acc;
  tc_fence_before();
  __syncthreads();
  if (EPI == TC_EPI_FWD_LAST && half == 0 && rv)
    g.e_out[(long)blockIdx.y * g.e_ld + row] = s_e[0][rl] + s_e[1][rl] + (blockIdx.y == 0 ? g.b_last[t] : 0.f);
  if (EPI != TC_EPI_PLAIN) {
    // ---- coalesced copy-out of the staged tiles (rows of this type only) ----
    const int c4n = BN / 4, c8n = BN / 8;
    float* of0 = (EPI == TC_EPI_FWD || EPI == TC_EPI_BWD) ? g.out_f32 : nullptr;
    float* of1 = (EPI == TC_EPI_FWD) ? g.out_t : nullptr;
    for (int u = threadIdx.x; u < BM * c4n; u += kThreads) {
      const int r = u / c4n, c4 = u - r * c4n;
      const int col = col0 + 4 * c4;
      if (row0 + r >= row_end || col >= g.N) continue;
      const uint32_t so = (uint32_t)((c4 >> 3) * 16384) + sw_off(r, c4 & 7);
      const long go = (long)(row0 + r) * g.N + col;
      if (of0) *reinterpret_cast<float4*>(of0 + go) = *reinterpret_cast<const float4*>(S0 + so);
      if (of1) *reinterpret_cast<float4*>(of1 + go) = *reinterpret_cast<const float4*>(S1 + so);
    }
    for (int u = threadIdx.x; u < BM * c8n; u += kThreads) {
      const int r = u / c8n, c8 = u - r * c8n;
      const int col = col0 + 8 * c8;
      if (row0 + r >= row_end || col >= g.N) continue;
      const uint32_t so = (uint32_t)((c8 >> 3) * 16384) + sw_off(r, c8 & 7);
      *reinterpret_cast<uint4*>(g.out_bf16 + (long)(row0 + r) * g.N + col) = *reinterpret_cast<const uint4*>(SB + so);
      if (NP == 3)
        *reinterpret_cast<uint4*>(g.out_bf16_lo + (long)(row0 + r) * g.N + col) =
            *reinterpret_cast<const uint4*>(SBL + so);
    }
  }
  tc_fence_before();
  __syncthreads();
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

int make_tmap_2d(CUtensorMap* map, const void* base, int elem_bytes, long rows, long cols, int box_cols,
                 int box_rows) {
  if (!g_encode) {  // load the encoder (a map of a dummy aligned address; nothing is accessed)
    CUtensorMap tmp;
    if (make_tmap_bf16(&tmp, reinterpret_cast<const void*>(uintptr_t(256)), 1, 64, 1) != DP_OK || !g_encode)
      return DP_E_CUDA;
  }
  if ((cols * elem_bytes) % 16 != 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0 || box_rows < 1 ||
      box_rows > 256 || box_cols * elem_bytes != 128) {
    set_error("tensor map: 16-byte aligned base and row pitch, 128-byte box rows, box rows in [1, 256]");
    return DP_E_UNSUPPORTED;
  }
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(cols * elem_bytes)};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(map, elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                        const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return DP_E_CUDA;
  }
  return DP_OK;
}

int tc_pick_bn(int N, int row_tiles) {
  int bn = ((N + 31) / 32) * 32;
  if (bn > 256) bn = 256;
  while (bn > 64 && (long)row_tiles * ((N + bn - 1) / bn) < 2L * 152) bn = ((bn / 2 + 31) / 32) * 32;
  return bn;
}

int make_tmap_f32(CUtensorMap* map, const void* base, long rows, long cols) {
  CUtensorMap tmp;
  if (make_tmap_bf16(&tmp, base, rows, cols, 128) != DP_OK) return DP_E_CUDA;  // loads the encoder
  if ((cols * 4) % 16 != 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0) {
    set_error("tensor map: FP32 row pitch and base must be 16-byte aligned");
    return DP_E_UNSUPPORTED;
  }
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(cols * 4)};
  cuuint32_t box[2] = {32, (cuuint32_t)BM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled (FP32) failed (" + std::to_string((int)r) + ")");
    return DP_E_CUDA;
  }
  return DP_OK;
}

template <int EPI, int NP>
cudaError_t launch_one(dim3 grid, size_t smem, const CUtensorMap& ta, const TcMaps& tb, const TcEpiMaps& em,
                       const TcArgs& a, const TcLo& lo, cudaStream_t st) {
  cudaError_t e = allow_max_smem(k_tc_gemm<EPI, NP>);
  if (e == cudaSuccess) k_tc_gemm<EPI, NP><<<grid, kThreads, smem, st>>>(ta, tb, em, a, lo);
  return e;
}

template <int NP>
cudaError_t launch_np(int epi, dim3 grid, size_t smem, const CUtensorMap& ta, const TcMaps& tb, const TcEpiMaps& em,
                      const TcArgs& a, const TcLo& lo, cudaStream_t st) {
  switch (epi) {
    case TC_EPI_PLAIN:
      return launch_one<TC_EPI_PLAIN, NP>(grid, smem, ta, tb, em, a, lo, st);
    case TC_EPI_FWD:
      return launch_one<TC_EPI_FWD, NP>(grid, smem, ta, tb, em, a, lo, st);
    case TC_EPI_FWD_LAST:
      return launch_one<TC_EPI_FWD_LAST, NP>(grid, smem, ta, tb, em, a, lo, st);
    default:
      return launch_one<TC_EPI_BWD, NP>(grid, smem, ta, tb, em, a, lo, st);
  }
}

cudaError_t launch_tc_gemm(int epi, const CUtensorMap& ta, const TcMaps& tb, const TcArgs& a, cudaStream_t st,
                           const TcLo* lo) {
  const int tiles = a.tile_start[a.ntypes];
  if (tiles <= 0) return cudaSuccess;
  if (epi != TC_EPI_PLAIN && (a.BN % 32 != 0 || a.skip_kind == 2)) {
    set_error("tensor-core GEMM epilogue: output blocks of 32 columns, skips of kind 0 or 1 only");
    return cudaErrorInvalidValue;
  }
  const int NP = lo ? 3 : 1;
  if (NP == 3 && epi != TC_EPI_PLAIN && !a.out_bf16_lo) {
    set_error("split tensor-core GEMM: the epilogue needs a low-part output");
    return cudaErrorInvalidValue;
  }
  dim3 grid(tiles, (a.N + a.BN - 1) / a.BN);
  const size_t ring = (size_t)ring_stages(a.K, a.BN, NP) * stage_bytes_of(a.BN, NP);
  const size_t ep = epi_bytes(epi, a.BN, NP);
  const size_t smem = (ring > ep ? ring : ep) + 1024 + 256;
  // epilogue inputs (skip, gate) as TMA maps over all rows
  TcEpiMaps em;
  std::memset(&em, 0, sizeof(em));
  const long rows = a.row_start[a.ntypes];
  if (epi != TC_EPI_PLAIN && a.skip_kind == 1 && a.skip_mat &&
      make_tmap_f32(&em.skip, a.skip_mat, rows, a.skip_ld) != DP_OK)
    return cudaErrorInvalidValue;
  if (epi == TC_EPI_BWD && make_tmap_f32(&em.tact, a.tact, rows, a.N) != DP_OK) return cudaErrorInvalidValue;
  TcLo none;
  std::memset(&none, 0, sizeof(none));
  cudaError_t e = NP == 3 ? launch_np<3>(epi, grid, smem, ta, tb, em, a, *lo, st)
                          : launch_np<1>(epi, grid, smem, ta, tb, em, a, none, st);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace dpgb
