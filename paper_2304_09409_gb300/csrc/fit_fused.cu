// The whole fitting net of the mixed mode -- forward through every hidden layer to E_i and the
// backward to dE/dD -- in one tcgen05 kernel per 128-atom tile (Eq. (fitting_energy), layers of
// Eq. (NN)).
//
// Per tile the CTA runs a chain of GEMMs whose intermediate activations never leave the SM:
//   forward  z_l = y_{l-1} W_l + b_l,  t_l = tanh z_l,  y_l = t_l (+ y_{l-1}),  E = y_last . w + b
//   backward gz_last = w (1 - t_last^2),  gy_{l-1} = gz_l W_l^T (+ gy_l),  gz_{l-1} = gy_{l-1} (1 - t_{l-1}^2),
//            dE/dD = gz_0 W_0^T
// D streams in by TMA (first layer), the weights of every layer stream through a three-stage
// TMA ring, the accumulator lives in tensor memory columns [0, 256), and the FP32 residual stream
// (y_l forward, gy_l backward) in columns [256, 512).  Eight epilogue warps read the accumulator
// (two per 32-row lane quadrant, alternate 16-column chunks), apply tanh / skip / gate, and write
// the next layer's A operand straight into shared memory in the 128-byte-swizzled K-major layout
// the tensor cores read.  The tanh gates 1 - t^2 of the inner layers go to an L2-resident scratch
// array and come back in the backward; dE/dD leaves in 256-column chunks from two alternating
// accumulator buffers.  One producer thread issues TMA, one thread issues tcgen05.mma; every
// mbarrier wait is bounded (on time-out the CTA records an error and finishes).
#include <cuda_bf16.h>

#include <cstring>

#include "fit_tc.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace dpgb {

namespace {

using namespace ptx;

constexpr int kFL = 4;             // hidden layers at most
constexpr int kEpiThreads = 256;   // eight epilogue warps
constexpr int kFThreads = kEpiThreads + 64;  // + producer warp + MMA warp
constexpr int FBM = 128, FBK = 64;
constexpr int kRing = 3;
constexpr uint32_t kAStage = FBM * FBK * 2;  // 16 KB: a 128 x 64 BF16 block
constexpr uint32_t kBStage = 256 * FBK * 2;  // 32 KB: up to 256 weight rows
constexpr uint32_t kStage = kAStage + kBStage;
constexpr uint32_t kAb = 4 * kAStage;  // A operand of the inner GEMMs: 128 rows x 256 (K)
constexpr int kGateLd = 256;

struct FusedMaps {
  CUtensorMap d;                          // D [rows][KD], box {64, 128}
  CUtensorMap w[DP_MAX_TYPES][2 * kFL];   // forward W_l^T (slot l), backward W_l (slot nh + l)
};

struct FusedArgs {
  int ntypes, nh;
  int width[kFL + 1];  // width[0] = KD (descriptor), width[l + 1] = outputs of hidden layer l
  int skip[kFL];       // 1: y_l = t_l + y_{l-1}
  int row_start[DP_MAX_TYPES + 1];
  int tile_start[DP_MAX_TYPES + 1];
  const float* bias[DP_MAX_TYPES][kFL];
  const float* w_last[DP_MAX_TYPES];
  float b_last[DP_MAX_TYPES];
  float* gate;          // [nh - 1][rows * kGateLd]: 1 - t_l^2 of the inner hidden layers, tile-blocked
                        // (4-column groups, the tile's rows contiguous)
  const int* perm;      // sorted row -> atom
  double* atom_e;       // [atoms] atomic energies, input order
  __nv_bfloat16* gD;    // dE/dD, BF16, tile-blocked (fit_tc.cuh)
  int* err;
};

// tanh by the hardware approximation (relative error about 2^-11): the activations leave the
// epilogue as BF16 operands (2^-9), so its error does not survive into the next layer.
__device__ __forceinline__ float tanh_hw(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void ab_store16(unsigned char* Ab, int rl, int col, const float* x) {
  uint32_t w[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const __nv_bfloat162 pr = __floats2bfloat162_rn(x[2 * q], x[2 * q + 1]);
    w[q] = *reinterpret_cast<const uint32_t*>(&pr);
  }
  const int kb = col >> 6, q0 = (col & 63) >> 3;
  unsigned char* base = Ab + kb * kAStage + rl * 128;
  *reinterpret_cast<uint4*>(base + ((q0 ^ (rl & 7)) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
  *reinterpret_cast<uint4*>(base + (((q0 + 1) ^ (rl & 7)) << 4)) = make_uint4(w[4], w[5], w[6], w[7]);
}

__global__ void __launch_bounds__(kFThreads, 1) k_fit_fused(const __grid_constant__ FusedMaps mp, const FusedArgs g) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char* ring = smem;
  unsigned char* Ab = smem + kRing * kStage;
  uint64_t* full = reinterpret_cast<uint64_t*>(Ab + kAb);
  uint64_t* empty = full + kRing;
  uint64_t* accf = empty + kRing;   // MMA -> epilogue: accumulator of an inner phase ready
  uint64_t* afree = accf + 1;       // epilogue -> MMA: next A operand written, accumulator read
  uint64_t* bfull = afree + 1;      // [2] dE/dD chunk buffers
  uint64_t* bempty = bfull + 2;     // [2]
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bempty + 2);
  float* s_e = reinterpret_cast<float*>(tmem_holder + 4);  // [2][128]
  float* s_bias = s_e + 2 * FBM;                           // [kFL][256] biases of the hidden layers
  float* s_wl = s_bias + kFL * 256;                        // [256] weights of the output layer

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int t = 0;
  while (t + 1 < g.ntypes && (int)blockIdx.x >= g.tile_start[t + 1]) ++t;
  const int row0 = g.row_start[t] + ((int)blockIdx.x - g.tile_start[t]) * FBM;
  const int row_end = g.row_start[t + 1];
  const long rows = g.row_start[g.ntypes];
  const int nh = g.nh, KD = g.width[0];
  const int nch = (KD + 255) / 256;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kRing; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    mbar_init(afree, kEpiThreads);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bfull[b], 1);
      mbar_init(&bempty[b], kEpiThreads);
    }
    mbar_fence_init();
  }
  if (warp == 8) tmem_alloc(tmem_holder, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 8) {
    if (lane == 0) {
      // ---- TMA producer: D and W_0^T blocks, then the weights of every later phase ----
      int it = 0;
      bool ok = true;
      auto push = [&](const CUtensorMap* bm, int bx, int by, uint32_t bbytes, bool with_a) -> bool {
        const int s = it % kRing;
        if (it >= kRing && !mbar_wait(&empty[s], ((it / kRing) - 1) & 1, g.err)) return false;
        unsigned char* st = ring + s * kStage;
        mbar_expect_tx(&full[s], (with_a ? kAStage : 0u) + bbytes);
        if (with_a) tma_load_2d(st, &mp.d, &full[s], bx, row0);
        tma_load_2d(st + kAStage, bm, &full[s], bx, by);
        ++it;
        return true;
      };
      for (int l = 0; ok && l < nh; ++l) {
        const int nkb = (g.width[l] + FBK - 1) / FBK;
        for (int kb = 0; ok && kb < nkb; ++kb)
          ok = push(&mp.w[t][l], kb * FBK, 0, (uint32_t)g.width[l + 1] * 128u, l == 0);
      }
      for (int l = nh - 1; ok && l >= 1; --l) {
        const int nkb = (g.width[l + 1] + FBK - 1) / FBK;
        for (int kb = 0; ok && kb < nkb; ++kb) ok = push(&mp.w[t][nh + l], kb * FBK, 0, (uint32_t)g.width[l] * 128u, false);
      }
      {
        const int nkb = (g.width[1] + FBK - 1) / FBK;
        for (int c = 0; ok && c < nch; ++c)
          for (int kb = 0; ok && kb < nkb; ++kb) ok = push(&mp.w[t][nh], kb * FBK, c * 256, 256u * 128u, false);
      }
      // every copy this thread started has landed before the CTA may exit
      for (int s = 0; s < kRing && s < it; ++s) {
        const int last = s + kRing * ((it - 1 - s) / kRing);
        mbar_wait(&full[s], (last / kRing) & 1, g.err);
      }
    }
  } else if (warp == 9) {
    if (lane == 0) {
      // ---- MMA issuer ----
      int it = 0, afr = 0;
      bool ok = true;
      auto gemm = [&](int K, int N, bool a_ring, uint32_t dcol) -> bool {
        const uint32_t idesc = idesc_f16(FBM, N, 1);
        const int nkb = (K + FBK - 1) / FBK;
        for (int kb = 0; kb < nkb; ++kb) {
          const int s = it % kRing;
          if (!mbar_wait(&full[s], (it / kRing) & 1, g.err)) return false;
          tc_fence_after();
          const uint32_t sa = su32(ring + s * kStage);
          const uint64_t ad = sdesc_sw128(a_ring ? sa : su32(Ab + kb * kAStage));
          const uint64_t bd = sdesc_sw128(sa + kAStage);
#pragma unroll
          for (int k = 0; k < FBK / 16; ++k) mma_f16(tmem + dcol, ad + 2 * k, bd + 2 * k, idesc, (kb | k) != 0);
          mma_commit(&empty[s]);
          ++it;
        }
        return true;
      };
      auto wait_free = [&]() -> bool {
        const bool r = mbar_wait(afree, afr & 1, g.err);
        ++afr;
        tc_fence_after();
        return r;
      };
      for (int l = 0; ok && l < nh; ++l) {
        if (l > 0) ok = wait_free();
        if (ok) ok = gemm(g.width[l], g.width[l + 1], l == 0, 0);
        mma_commit(accf);
      }
      for (int l = nh - 1; ok && l >= 1; --l) {
        ok = wait_free();
        if (ok) ok = gemm(g.width[l + 1], g.width[l], false, 0);
        mma_commit(accf);
      }
      if (ok) ok = wait_free();
      for (int c = 0; ok && c < nch; ++c) {
        const int buf = c & 1;
        if (c >= 2 && !mbar_wait(&bempty[buf], ((c >> 1) - 1) & 1, g.err)) break;
        tc_fence_after();
        ok = gemm(g.width[1], min(256, KD - c * 256), false, (uint32_t)(buf * 256));
        mma_commit(&bfull[buf]);
      }
    }
  } else {
    // ---- epilogue: warps w and w + 4 own rows 32(w % 4) .. +31, alternate 16-column chunks ----
    const int quad = warp & 3, half = warp >> 2;
    const int rl = quad * 32 + lane;
    const int row = row0 + rl;
    const bool rv = row < row_end;
    const int nr = min(FBM, row_end - row0);  // rows of this tile (tile-blocked scratch and dE/dD)
    // gate of (row, col) in layer l's scratch: 4-column groups of the tile's rows, contiguous
    auto gate_at = [&](int l, int col) -> float* {
      return g.gate + (long)l * rows * kGateLd + (long)row0 * kGateLd + ((long)(col >> 2) * nr + rl) * 4;
    };
    const uint32_t tb = tmem + ((uint32_t)(quad * 32) << 16);
    int acf = 0;
    auto wait_acc = [&]() {
      mbar_wait(accf, acf & 1, g.err);
      ++acf;
      __syncwarp();
      tc_fence_after();
    };
    auto pad = [&](int N) {  // zero K columns [N, next multiple of 64) of the next A operand
      if (half != 1) return;
      for (int col = N; col < ((N + 63) & ~63); col += 8) {
        const int kb = col >> 6, q = (col & 63) >> 3;
        *reinterpret_cast<uint4*>(Ab + kb * kAStage + rl * 128 + ((q ^ (rl & 7)) << 4)) = make_uint4(0u, 0u, 0u, 0u);
      }
    };
    auto release = [&](bool stored) {
      if (stored) tmem_wait_st();
      tc_fence_before();
      fence_async_smem();  // the A operand written here is read by the tensor cores next
      mbar_arrive(afree);
    };
    // biases and output weights of this tile's type into shared memory (while the first GEMM runs)
    for (int l = 0; l < nh; ++l)
      for (int c = threadIdx.x; c < g.width[l + 1]; c += kEpiThreads) s_bias[l * 256 + c] = __ldg(g.bias[t][l] + c);
    for (int c = threadIdx.x; c < g.width[nh]; c += kEpiThreads) s_wl[c] = __ldg(g.w_last[t] + c);
    bar_sync(1, kEpiThreads);
    const float* wl = s_wl;
    // forward
    for (int l = 0; l < nh; ++l) {
      wait_acc();
      const int N = g.width[l + 1];
      const bool last = (l == nh - 1), sk = g.skip[l] == 1;
      const float* bias = s_bias + l * 256;
      float e_acc = 0.f;
      const int nq = N / 16;
      for (int q0 = half; q0 < nq; q0 += 4) {  // two 16-column pieces per wait
        uint32_t rab[2][16], ryb[2][16];
#pragma unroll
        for (int u = 0; u < 2; ++u)
          if (q0 + 2 * u < nq) {
            tmem_ld16_async(tb + (q0 + 2 * u) * 16, rab[u]);
            if (sk) tmem_ld16_async(tb + 256 + (q0 + 2 * u) * 16, ryb[u]);
          }
        tmem_wait_ld();
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          if (q0 + 2 * u >= nq) break;
          const int col = (q0 + 2 * u) * 16;
          float y[16], gt[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float th = tanh_hw(__uint_as_float(rab[u][i]) + bias[col + i]);
            y[i] = th + (sk ? __uint_as_float(ryb[u][i]) : 0.f);
            gt[i] = 1.f - th * th;
          }
          if (!last) {
            ab_store16(Ab, rl, col, y);
            tmem_st16(tb + 256 + col, y);  // the residual stream of the next layer
            if (rv) {
#pragma unroll
              for (int q = 0; q < 4; ++q)
                *reinterpret_cast<float4*>(gate_at(l, col + 4 * q)) =
                    make_float4(gt[4 * q], gt[4 * q + 1], gt[4 * q + 2], gt[4 * q + 3]);
            }
          } else {
            float gz[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const float w = wl[col + i];
              e_acc += y[i] * w;
              gz[i] = w * gt[i];
            }
            ab_store16(Ab, rl, col, gz);
          }
        }
      }
      pad(N);
      if (last) {
        s_e[half * FBM + rl] = e_acc;
        bar_sync(1, kEpiThreads);
        if (half == 0 && rv) g.atom_e[g.perm[row]] = (double)(s_e[rl] + s_e[FBM + rl] + g.b_last[t]);
      }
      release(!last);
    }
    // backward of layers nh-1 .. 1: gz_{l-1} into the A operand, gy_{l-1} kept for the next skip
    for (int l = nh - 1; l >= 1; --l) {
      const int N = g.width[l];
      const bool top = (l == nh - 1), sk = g.skip[l] == 1, keep = (l - 1 >= 1);
      if (rv)  // this row's gates towards L1 while the GEMM of this phase runs
        for (int q16 = half; q16 < N / 16; q16 += 2)
#pragma unroll
          for (int q = 0; q < 4; ++q) prefetch_l1(gate_at(l - 1, q16 * 16 + 4 * q));
      wait_acc();
      const int nq = N / 16;
      for (int q0 = half; q0 < nq; q0 += 4) {  // two 16-column pieces per wait
        uint32_t rab[2][16], ryb[2][16];
#pragma unroll
        for (int u = 0; u < 2; ++u)
          if (q0 + 2 * u < nq) {
            tmem_ld16_async(tb + (q0 + 2 * u) * 16, rab[u]);
            if (sk && !top) tmem_ld16_async(tb + 256 + (q0 + 2 * u) * 16, ryb[u]);
          }
        tmem_wait_ld();
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          if (q0 + 2 * u >= nq) break;
          const int col = (q0 + 2 * u) * 16;
          float gt[16];
          if (rv) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float4 x = *reinterpret_cast<const float4*>(gate_at(l - 1, col + 4 * q));
              gt[4 * q] = x.x;
              gt[4 * q + 1] = x.y;
              gt[4 * q + 2] = x.z;
              gt[4 * q + 3] = x.w;
            }
          } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) gt[i] = 0.f;
          }
          float gy[16], gz[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            float v = __uint_as_float(rab[u][i]);
            if (sk) v += top ? wl[col + i] : __uint_as_float(ryb[u][i]);
            gy[i] = v;
            gz[i] = v * gt[i];
          }
          ab_store16(Ab, rl, col, gz);
          if (keep) tmem_st16(tb + 256 + col, gy);
        }
      }
      pad(N);
      release(keep);
    }
    // dE/dD = gz_0 W_0^T in 256-column chunks from two alternating accumulators
    for (int c = 0; c < nch; ++c) {
      const int buf = c & 1;
      mbar_wait(&bfull[buf], (c >> 1) & 1, g.err);
      __syncwarp();
      tc_fence_after();
      const int N = min(256, KD - c * 256);
      const int nq = N / 16;  // 16-column pieces; this warp takes every other one, four loads per wait
      __nv_bfloat16* gtile = g.gD + (long)row0 * KD;
      for (int q0 = half; q0 < nq; q0 += 8) {
        uint32_t ra[4][16];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (q0 + 2 * u < nq) tmem_ld16_async(tb + (uint32_t)(buf * 256) + (q0 + 2 * u) * 16, ra[u]);
        tmem_wait_ld();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (q0 + 2 * u >= nq || !rv) continue;
          uint32_t w[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const __nv_bfloat162 pr =
                __floats2bfloat162_rn(__uint_as_float(ra[u][2 * q]), __uint_as_float(ra[u][2 * q + 1]));
            w[q] = *reinterpret_cast<const uint32_t*>(&pr);
          }
          // two 8-column groups: consecutive rows of the warp write consecutive 16-byte chunks
          const int g8 = (c * 256 + (q0 + 2 * u) * 16) >> 3;
          uint4* d0 = reinterpret_cast<uint4*>(gtile + ((long)g8 * nr + rl) * 8);
          uint4* d1 = reinterpret_cast<uint4*>(gtile + ((long)(g8 + 1) * nr + rl) * 8);
          *d0 = make_uint4(w[0], w[1], w[2], w[3]);
          *d1 = make_uint4(w[4], w[5], w[6], w[7]);
        }
      }
      tc_fence_before();
      mbar_arrive(&bempty[buf]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 8) tmem_dealloc(tmem, 512);
}

size_t fused_smem() {
  return (size_t)kRing * kStage + kAb + 16 * 8 + 16 + (2 * FBM + kFL * 256 + 256) * 4 + 1024;
}

}  // namespace

bool fit_fused_supported(const DeviceModel& m) {
  const int nfl = m.n_fit_layers, nh = nfl - 1;
  if (nh < 1 || nh > kFL) return false;
  const int KD = m.M * m.A;
  if (KD % 16 != 0) return false;
  for (int t = 0; t < m.cfg.ntypes; ++t)
    for (int l = 0; l < nh; ++l) {
      const LayerDesc& L = m.fit[(size_t)t * nfl + l];
      const LayerDesc& L0 = m.fit[l];
      if (L.n_in != L0.n_in || L.n_out != L0.n_out || L.skip != L0.skip) return false;
      if (L.n_out % 16 || L.n_out > 256 || L.skip > 1 || (l == 0 && L.skip)) return false;
    }
  return m.fit[0].n_in == KD;
}

int run_fitting_fused(const DeviceModel& m, const PathConst& pc, const __nv_bfloat16* Dbf, const PathIO& io,
                      Arena& ar, cudaStream_t st, const __nv_bfloat16** gDh_out) {
  const long N = pc.natoms;
  const int nfl = m.n_fit_layers, nh = nfl - 1;
  const int nt = pc.ntypes;
  const int KD = pc.M * pc.A;
  float* gate = ar.get<float>((long)(nh > 1 ? nh - 1 : 1) * N * kGateLd);
  __nv_bfloat16* gD = ar.get<__nv_bfloat16>(N * KD);
  if (ar.measure) return DP_OK;
  if (!ar.ok()) {
    set_error("scratch allocation failed");
    return DP_E_OOM;
  }
  FusedArgs a;
  std::memset(&a, 0, sizeof(a));
  a.ntypes = nt;
  a.nh = nh;
  a.width[0] = KD;
  for (int l = 0; l < nh; ++l) {
    a.width[l + 1] = m.fit[l].n_out;
    a.skip[l] = m.fit[l].skip;
  }
  int tiles = 0;
  for (int t = 0; t <= nt; ++t) {
    a.row_start[t] = io.type_start[t];
    a.tile_start[t] = tiles;
    if (t < nt) tiles += (io.type_start[t + 1] - io.type_start[t] + FBM - 1) / FBM;
  }
  FusedMaps mp;
  std::memset(&mp, 0, sizeof(mp));
  int rc = make_tmap_bf16(&mp.d, Dbf, N, KD, FBM);
  if (rc != DP_OK) return rc;
  const float* p32 = m.p32;
  for (int t = 0; t < nt; ++t) {
    for (int l = 0; l < nh; ++l) {
      const LayerDesc& L = m.fit[(size_t)t * nfl + l];
      a.bias[t][l] = p32 + L.w_off + (long)L.n_in * L.n_out;
      const CUtensorMap* f = fit_weight_map(m, t, l, 0, L.n_out);
      const CUtensorMap* b = fit_weight_map(m, t, l, 1, l == 0 ? 256 : L.n_in);
      if (!f || !b) return DP_E_CUDA;
      mp.w[t][l] = *f;
      mp.w[t][nh + l] = *b;
    }
    const LayerDesc& Lo = m.fit[(size_t)t * nfl + nh];
    a.w_last[t] = p32 + Lo.w_off;
    a.b_last[t] = m.fit_out_bias[t];
  }
  a.gate = gate;
  a.perm = io.perm;
  a.atom_e = io.atom_energy;
  a.gD = gD;
  a.err = &io.status->timeout;  // bounded waits that give up are reported by the call
  if (tiles > 0) {
    ProfScope _ps(io.prof, "fit_fused_tc", st);
    const size_t smem = fused_smem();
    DP_CUDA_TRY(allow_max_smem(k_fit_fused));
    k_fit_fused<<<tiles, kFThreads, smem, st>>>(mp, a);
    DP_CUDA_TRY(cudaGetLastError());
  }
  *gDh_out = gD;
  return DP_OK;
}

}  // namespace dpgb
