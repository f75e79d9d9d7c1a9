// The whole fitting net of the FP32 mode -- forward to E_i and backward to dE/dD -- in one tcgen05
// kernel per 128-atom tile, on split BF16 operands (x = hi + lo, every product formed as
// hi.hi + hi.lo + lo.hi: about 16 significant bits per operand, FP32 accumulation), Eq.
// (fitting_energy) with the layers of Eq. (NN).
//
// Per tile the CTA runs the chain of GEMMs of the net: forward layers z_l = y_{l-1} W_l + b_l,
// t_l = tanh z_l, y_l = t_l (+ y_{l-1}), E = y_last . w + b; backward gz_last = w (1 - t_last^2),
// gy_{l-1} = gz_l W_l^T (+ gy_l), gz_{l-1} = gy_{l-1} (1 - t_{l-1}^2), dE/dD = gz_0 W_0^T.  Each GEMM
// streams its A operand (the descriptor, or the previous phase's activations) and its weights
// through one two-stage TMA ring of high and low halves (96 KB a stage); the accumulator lives in
// tensor memory.  Activations go from each epilogue to the next phase through a per-tile scratch
// that stays in L2 (high and low BF16 halves for the next A operand, FP32 for the gates): the
// epilogue writes the next A operand into the idle ring in the swizzled layout of the TMA box and
// stores it with four tiled TMA stores per half (coalesced), clipped at the end of the tile's
// type; the FP32 residual stream stays in tensor memory; dE/dD leaves in 256-column chunks from two
// alternating accumulators, so that one chunk's epilogue overlaps the next chunk's MMAs.  One
// thread issues TMA, one issues tcgen05.mma, sixteen warps run the epilogues; every mbarrier wait
// is bounded (on time-out the CTA records an error and finishes).
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "fit_tc.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace dpgb {

namespace {

using namespace ptx;

constexpr int kSL = 4;  // hidden layers at most
constexpr int kSEpi = 256;               // eight epilogue warps: two per 32-row quarter of the tile
constexpr int kSThreads = kSEpi + 64;    // + a TMA producer warp and an MMA warp
constexpr int kProd = kSEpi / 32, kMmaW = kProd + 1;  // their warp indices
constexpr int kParts = kSEpi / 128;      // epilogue warps sharing a row quarter, interleaved by 16 columns
constexpr int kStep = 16 * kParts;       // column stride of one epilogue thread
constexpr int SBM = 128, SBK = 64;
constexpr int kSRing = 2;
constexpr uint32_t kSA = SBM * SBK * 2;   // 16 KB: one 128 x 64 BF16 block of A
constexpr uint32_t kSB = 256 * SBK * 2;   // 32 KB: up to 256 weight rows
constexpr uint32_t kSStage = 2 * (kSA + kSB);  // [A hi | A lo | B hi | B lo]
constexpr int kSLd = 256;  // row pitch of the activation scratch (elements)

struct SplitMaps {
  CUtensorMap d[2];                       // D hi / lo [rows][KD], box {64, 128}
  CUtensorMap x[2][2];                    // activation scratch buffer b (hi / lo) [rows][kSLd], box {64, 128}
  CUtensorMap xt[DP_MAX_TYPES][2][2];     // the same per type, over the type's rows only (stores)
  CUtensorMap w[DP_MAX_TYPES][2 * kSL][2];  // per type: forward W_l^T (slot l), backward W_l (slot nh + l); hi / lo
};

struct SplitArgs {
  int ntypes, nh;
  int width[kSL + 1];  // width[0] = KD, width[l + 1] = outputs of hidden layer l
  int skip[kSL];
  int row_start[DP_MAX_TYPES + 1];
  int tile_start[DP_MAX_TYPES + 1];
  const float* bias[DP_MAX_TYPES][kSL];
  const float* w_last[DP_MAX_TYPES];
  float b_last[DP_MAX_TYPES];
  __nv_bfloat16* xs[2][2];  // activation scratch [2 buffers][hi, lo] [rows][kSLd]
  float* gate;              // 1 - t_l^2 of the inner hidden layers [nh][rows][kSLd]
  const int* perm;
  double* atom_e;
  float* gD;                // dE/dD FP32 [rows][KD], or null when gT is formed instead
  // dE/dT of the se_e2_a contraction (M_< = 16), formed from each dE/dD chunk in the epilogue:
  // gT[m][c] = sum_l gD[m][l] T[l][c] + [m < 16] sum_q gD[q][m] T[q][c], stored m-major
  // [M][rows][4] FP32 (consecutive rows of one m are contiguous)
  float* gT;
  const float* Tm;          // T [rows][M][4] FP32
  int M;
  int* err;
};

// 32-byte global accesses (one full sector per lane): half the instructions and no partial-sector
// writes where each lane owns a row of the tile.
__device__ __forceinline__ void st_v8(float* p, const float* v) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]),
               "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
               : "memory");
}
__device__ __forceinline__ void ld_v8(const float* p, float* v) {
  asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
               : "l"(p));
}

// tanh from the exponential, tanh x = 1 - 2 / (1 + e^{2x}) (x clamped to +-15, where tanh is 1 to
// FP32): absolute error a few 1e-7, below the ~2^-17 relative rounding the next GEMM's split
// operands apply anyway.  Only the exponential goes to the special-function unit, the epilogues'
// narrowest pipe: 1/d comes from the bit pattern of d (first guess within 5.1 %, the constant
// fitted to the mantissa range [1, 2)) and three Newton steps y <- y (2 - d y) on the FMA pipe.
__device__ __forceinline__ float tanh_ex(float x) {
  const float e = __expf(2.f * fminf(fmaxf(x, -15.f), 15.f));
  const float d = 1.f + e;  // [1, 1 + e^30]: a normal number
  float y = __int_as_float(0x7EF311C0 - __float_as_int(d));
  y = y * (2.f - d * y);
  y = y * (2.f - d * y);
  y = y * (2.f - d * y);
  return 1.f - 2.f * y;
}

__device__ __forceinline__ void split2(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

__global__ void __launch_bounds__(kSThreads, 1) k_fit_split(const __grid_constant__ SplitMaps mp, const SplitArgs g) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kSRing * kSStage);
  uint64_t* empty = full + kSRing;
  uint64_t* accf = empty + kSRing;  // [2] accumulator buffer ready (MMA -> epilogue)
  uint64_t* accfree = accf + 2;     // [2] accumulator read and phase outputs written (epilogue -> MMA, TMA)
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(accfree + 2);
  float* s_e = reinterpret_cast<float*>(tmem_holder + 4);  // [kParts][128]
  float* s_bias = s_e + kParts * SBM;                      // [kSL][256] biases of the hidden layers
  float* s_wl = s_bias + kSL * 256;                        // [256] weights of the output layer

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int t = 0;
  while (t + 1 < g.ntypes && (int)blockIdx.x >= g.tile_start[t + 1]) ++t;
  const int row0 = g.row_start[t] + ((int)blockIdx.x - g.tile_start[t]) * SBM;
  const int row_end = g.row_start[t + 1];
  const long rows = g.row_start[g.ntypes];
  const int nh = g.nh, KD = g.width[0];
  const int nch = (KD + 255) / 256;
  // phases: forward layers 0 .. nh-1, backward layers nh-1 .. 1, then the nch dE/dD chunks
  const int nphase = nh + (nh - 1) + nch;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kSRing; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&accfree[b], kSEpi);
    }
    mbar_fence_init();
  }
  if (warp == kProd) tmem_alloc(tmem_holder, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  // phase p: its GEMM (K, N), the A map pair, the weight slot, the accumulator buffer, and
  // whether its A operand was written by the phase before (the producer then waits for it)
  auto phase_info = [&](int p, int& K, int& N, const CUtensorMap*& ah, const CUtensorMap*& al, int& wslot, int& wrow,
                        int& buf) {
    buf = 0;
    wrow = 0;
    if (p < nh) {  // forward layer p: A = D (p == 0) or the scratch the previous layer wrote
      K = g.width[p];
      N = g.width[p + 1];
      ah = p == 0 ? &mp.d[0] : &mp.x[(p - 1) & 1][0];
      al = p == 0 ? &mp.d[1] : &mp.x[(p - 1) & 1][1];
      wslot = p;
    } else if (p < 2 * nh - 1) {  // backward layer l = nh - 1 - (p - nh): A = gz_l
      const int l = nh - 1 - (p - nh);
      K = g.width[l + 1];
      N = g.width[l];
      const int xb = (p - 1) & 1;
      ah = &mp.x[xb][0];
      al = &mp.x[xb][1];
      wslot = nh + l;
    } else {  // dE/dD chunk c = gz_0 W_0^T, columns [256 c, 256 c + 256)
      const int c = p - (2 * nh - 1);
      K = g.width[1];
      N = min(256, KD - 256 * c);
      const int xb = (2 * nh - 2) & 1;
      ah = &mp.x[xb][0];
      al = &mp.x[xb][1];
      wslot = nh;
      wrow = 256 * c;
      buf = c & 1;
    }
  };

  if (warp == kProd) {
    if (lane == 0) {
      // ---- TMA producer ----
      int it = 0;
      bool ok = true;
      int fr[2] = {0, 0};  // accumulator-free phases waited for, per buffer
      for (int p = 0; ok && p < nphase; ++p) {
        int K, N, wslot, wrow, buf;
        const CUtensorMap *ah, *al;
        phase_info(p, K, N, ah, al, wslot, wrow, buf);
        // the A operand of phases after the first was written by the previous phase's epilogue
        if (p >= 1 && p <= 2 * nh - 1) {
          const int pb = 0;  // chain phases use accumulator buffer 0
          ok = mbar_wait(&accfree[pb], fr[pb] & 1, g.err);
          ++fr[pb];
          if (!ok) break;
        }
        const int nkb = (K + SBK - 1) / SBK;
        for (int kb = 0; ok && kb < nkb; ++kb) {
          const int s = it % kSRing;
          if (it >= kSRing && !mbar_wait(&empty[s], ((it / kSRing) - 1) & 1, g.err)) {
            ok = false;
            break;
          }
          unsigned char* st = smem + s * kSStage;
          // the weight boxes hold N rows (chain layers) or 256 (dE/dD chunks; rows beyond W_0 are zero-filled)
          const uint32_t brows = p < 2 * nh - 1 ? (uint32_t)N : 256u;
          mbar_expect_tx(&full[s], 2 * kSA + 2 * brows * 128u);
          tma_load_2d(st, ah, &full[s], kb * SBK, row0);
          tma_load_2d(st + kSA, al, &full[s], kb * SBK, row0);
          tma_load_2d(st + 2 * kSA, &mp.w[t][wslot][0], &full[s], kb * SBK, wrow);
          tma_load_2d(st + 2 * kSA + kSB, &mp.w[t][wslot][1], &full[s], kb * SBK, wrow);
          ++it;
        }
      }
      // every copy this thread started has landed before the CTA may exit
      for (int s = 0; s < kSRing && s < it; ++s) {
        const int last = s + kSRing * ((it - 1 - s) / kSRing);
        mbar_wait(&full[s], (last / kSRing) & 1, g.err);
      }
    }
  } else if (warp == kMmaW) {
    if (lane == 0) {
      // ---- MMA issuer ----
      int it = 0;
      bool ok = true;
      int fr[2] = {0, 0};
      for (int p = 0; ok && p < nphase; ++p) {
        int K, N, wslot, wrow, buf;
        const CUtensorMap *ah, *al;
        phase_info(p, K, N, ah, al, wslot, wrow, buf);
        // the accumulator buffer must have been read by the epilogue of its previous phase
        if (p >= 1) {
          int need;
          if (p <= 2 * nh - 1) {
            need = 1;  // chain: the previous phase's epilogue
          } else {
            const int c = p - (2 * nh - 1);
            need = (buf == 0) ? 1 : (c >= 2 ? 1 : 0);  // buffer 0 follows the chain; buffer 1 from chunk 3 on
          }
          if (need) {
            ok = mbar_wait(&accfree[buf], fr[buf] & 1, g.err);
            ++fr[buf];
            if (!ok) break;
          }
        }
        tc_fence_after();
        const uint32_t idesc = idesc_f16(SBM, N <= 256 ? ((N + 15) & ~15) : 256, 1);
        const uint32_t acc = tmem + (uint32_t)(buf * 256);
        const int nkb = (K + SBK - 1) / SBK;
        for (int kb = 0; kb < nkb; ++kb) {
          const int s = it % kSRing;
          if (!mbar_wait(&full[s], (it / kSRing) & 1, g.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = su32(smem + s * kSStage);
          const uint64_t ah_ = sdesc_sw128(sa), al_ = sdesc_sw128(sa + kSA);
          const uint64_t bh_ = sdesc_sw128(sa + 2 * kSA), bl_ = sdesc_sw128(sa + 2 * kSA + kSB);
#pragma unroll
          for (int k = 0; k < SBK / 16; ++k) {  // small terms first: lo.hi, hi.lo, then hi.hi
            mma_f16(acc, al_ + 2 * k, bh_ + 2 * k, idesc, (kb | k) != 0);
            mma_f16(acc, ah_ + 2 * k, bl_ + 2 * k, idesc, 1);
            mma_f16(acc, ah_ + 2 * k, bh_ + 2 * k, idesc, 1);
          }
          mma_commit(&empty[s]);
          ++it;
        }
        mma_commit(&accf[buf]);
      }
    }
  } else {
  // ---- epilogues: warps w and w + 4 own rows 32(w % 4) .. +31 and take 16-column pieces in turn ----
  // The FP32 residual stream (y_l forward, gy_l backward) stays in tensor-memory columns
  // [256, 512) of the thread's row, which the chain phases leave free.
  const int quad = warp & 3, part = warp >> 2;
  const int rl = quad * 32 + lane;
  const long row = row0 + rl;
  const bool rv = row < row_end;
  const uint32_t tq = tmem + ((uint32_t)(quad * 32) << 16);
  int af[2] = {0, 0};  // accumulator-ready phases waited for, per buffer
  bool dead = false;   // after a timed-out wait: stop waiting, keep arriving
  auto wait_acc = [&](int buf) {
    if (!dead && !mbar_wait(&accf[buf], af[buf] & 1, g.err)) dead = true;
    ++af[buf];
    __syncwarp();
    tc_fence_after();
  };
  auto release = [&](int buf, bool stored) {
    if (stored) tmem_wait_st();
    fence_async_global();  // this phase's global writes, read next by TMA
    tc_fence_before();
    mbar_arrive(&accfree[buf]);
  };
  auto gate_at = [&](int l, int col) -> float* { return g.gate + ((long)l * rows + row) * kSLd + col; };
  // the next A operand, staged in the idle ring: 64-column block kb of half hl at (2 kb + hl) * kSA,
  // row rl at rl * 128 bytes, 16-byte chunk j at (j ^ (rl % 8)) * 16 (the TMA box's 128-byte swizzle)
  auto put_x = [&](int c, const float* x) {
    __align__(16) __nv_bfloat16 hi[16], lo[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) split2(x[i], hi[i], lo[i]);
    const int kb = c >> 6, j = (c & 63) >> 3;
    unsigned char* bh = smem + (2 * kb) * kSA + rl * 128;
    unsigned char* bl = bh + kSA;
    *reinterpret_cast<uint4*>(bh + ((j ^ (rl & 7)) << 4)) = *reinterpret_cast<const uint4*>(hi);
    *reinterpret_cast<uint4*>(bh + (((j + 1) ^ (rl & 7)) << 4)) = *reinterpret_cast<const uint4*>(hi + 8);
    *reinterpret_cast<uint4*>(bl + ((j ^ (rl & 7)) << 4)) = *reinterpret_cast<const uint4*>(lo);
    *reinterpret_cast<uint4*>(bl + (((j + 1) ^ (rl & 7)) << 4)) = *reinterpret_cast<const uint4*>(lo + 8);
  };
  // the staged operand to scratch buffer xb, one 64-column block at a time: after its second pieces
  // of block kb (loop iteration k odd) every thread has staged its part of the block, and one
  // thread starts the block's two TMA stores while the epilogue goes on; all complete before the
  // phase is released
  auto store_block = [&](int k, int xb) {
    if (!(k & 1)) return;
    const int kb = k >> 1;
    fence_async_smem();
    bar_sync(1, kSEpi);
    if (threadIdx.x == 0) {
      for (int hl = 0; hl < 2; ++hl)
        tma_store_2d(&mp.xt[t][xb][hl], smem + (2 * kb + hl) * kSA, kb * 64, row0 - g.row_start[t]);
      bulk_commit();
    }
  };
  auto flush_wait = [&]() {
    if (threadIdx.x == 0) bulk_wait0();
  };
  // biases and output weights of this tile's type into shared memory
  for (int l = 0; l < nh; ++l)
    for (int c = threadIdx.x; c < 256; c += kSEpi)
      s_bias[l * 256 + c] = c < g.width[l + 1] ? __ldg(g.bias[t][l] + c) : 0.f;
  for (int c = threadIdx.x; c < 256; c += kSEpi) s_wl[c] = c < g.width[nh] ? __ldg(g.w_last[t] + c) : 0.f;
  bar_sync(1, kSEpi);
  // forward
  for (int l = 0; l < nh; ++l) {
    wait_acc(0);
    const int N = g.width[l + 1];
    const bool last = (l == nh - 1), sk = g.skip[l] == 1;
    const float* bias = s_bias + l * 256;
    const int xb = l & 1;
    float e_acc = 0.f;
    // the accumulator (and residual) pieces load one ahead of the piece being processed
    uint32_t na[16], ny[16];
    tmem_ld16_async(tq + part * 16, na);
    if (sk) tmem_ld16_async(tq + 256 + part * 16, ny);
    tmem_wait_ld();
    for (int c = part * 16, k = 0; c < kSLd; c += kStep, ++k) {  // zeros beyond N: the next A operand's K padding
      uint32_t ra[16], ry[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        ra[i] = na[i];
        ry[i] = ny[i];
      }
      if (c + kStep < kSLd) {
        tmem_ld16_async(tq + c + kStep, na);
        if (sk) tmem_ld16_async(tq + 256 + c + kStep, ny);
      }
      float out[16], y[16], gt[16];
      if (c < N) {  // widths are multiples of 16: a piece is all real columns or all padding
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int col = c + i;
          const float th = tanh_ex(__uint_as_float(ra[i]) + bias[col]);
          y[i] = th + (sk ? __uint_as_float(ry[i]) : 0.f);
          gt[i] = 1.f - th * th;
          if (last) {
            const float w = s_wl[col];
            e_acc += y[i] * w;
            out[i] = w * gt[i];
          } else {
            out[i] = y[i];
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) out[i] = y[i] = gt[i] = 0.f;
      }
      tmem_wait_ld();                          // the next piece has landed
      if (!last) tmem_st16(tq + 256 + c, y);  // the residual stream of the next layer
      put_x(c, out);
      if (rv && !last && c < N) {
        st_v8(gate_at(l, c), gt);
        st_v8(gate_at(l, c + 8), gt + 8);
      }
      store_block(k, xb);
    }
    if (last) {
      s_e[part * SBM + rl] = e_acc;
      bar_sync(1, kSEpi);
      if (part == 0 && rv) {
        float e = 0.f;
#pragma unroll
        for (int q = 0; q < kParts; ++q) e += s_e[q * SBM + rl];
        g.atom_e[g.perm[row]] = (double)(e + g.b_last[t]);
      }
    }
    flush_wait();
    release(0, !last);
  }
  // backward of layers nh-1 .. 1: gz_{l-1} into the scratch, gy_{l-1} kept for the next skip
  for (int l = nh - 1; l >= 1; --l) {
    const int N = g.width[l];
    if (rv)  // this row's gates towards L1 while the GEMM of this phase runs
      for (int c = part * 16; c < N; c += kStep)
#pragma unroll
        for (int q = 0; q < 4; ++q) prefetch_l1(gate_at(l - 1, c + 4 * q));
    wait_acc(0);
    const bool top = (l == nh - 1), sk = g.skip[l] == 1, keep = (l - 1 >= 1);
    const int p = nh + (nh - 1 - l);  // phase index
    const int xb = p & 1;
    const bool ldy = sk && !top;
    uint32_t na[16], ny[16];
    tmem_ld16_async(tq + part * 16, na);
    if (ldy) tmem_ld16_async(tq + 256 + part * 16, ny);
    tmem_wait_ld();
    for (int c = part * 16, k = 0; c < kSLd; c += kStep, ++k) {  // zeros beyond N: the next A operand's K padding
      uint32_t ra[16], ry[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        ra[i] = na[i];
        ry[i] = ny[i];
      }
      if (c + kStep < kSLd) {
        tmem_ld16_async(tq + c + kStep, na);
        if (ldy) tmem_ld16_async(tq + 256 + c + kStep, ny);
      }
      float gt[16];
      if (rv && c < N) {
        ld_v8(gate_at(l - 1, c), gt);
        ld_v8(gate_at(l - 1, c + 8), gt + 8);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) gt[i] = 0.f;
      }
      float gy[16], gz[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int col = c + i;
        float v = col < N ? __uint_as_float(ra[i]) : 0.f;
        if (sk && col < N) v += top ? s_wl[col] : __uint_as_float(ry[i]);
        gy[i] = v;
        gz[i] = v * gt[i];
      }
      tmem_wait_ld();
      if (keep) tmem_st16(tq + 256 + c, gy);
      put_x(c, gz);
      store_block(k, xb);
    }
    flush_wait();
    release(0, keep);
  }
  // dE/dD in 256-column chunks from the two alternating accumulators: stored, or (gT mode, 16-column
  // pieces = one m) folded at once into dE/dT, term 1 per piece and term 2 accumulated per row
  const bool gtm = g.gT != nullptr;
  float ext[16][4];
#pragma unroll
  for (int l = 0; l < 16; ++l)
#pragma unroll
    for (int q = 0; q < 4; ++q) ext[l][q] = 0.f;
  // T_< of the tile's rows in shared memory over the forward's dead biases and energies: row rl's
  // float4 l at rl * 16 + (l ^ (rl % 8)), so that the 32 rows of a warp read without conflicts
  float4* s_tl = reinterpret_cast<float4*>(s_e);
  if (gtm) {
    for (int e = threadIdx.x; e < SBM * 16; e += kSEpi) {
      const int r = e >> 4, l = e & 15;
      const long rr = row0 + r;
      s_tl[r * 16 + (l ^ (r & 7))] = rr < row_end ? __ldg(reinterpret_cast<const float4*>(g.Tm + (rr * g.M + l) * 4))
                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    bar_sync(1, kSEpi);
  }
  for (int c = 0; c < nch; ++c) {
    const int buf = c & 1;
    wait_acc(buf);
    const int N = min(256, KD - 256 * c);
    float* dst = gtm ? nullptr : g.gD + row * KD + 256 * c;
    const uint32_t tb = tq + (uint32_t)(buf * 256);
    for (int q = part * 16; q < N; q += kStep) {
      float v[16];
      tmem_ld16(tb + q, v);
      if (rv) {
        if (gtm) {
          const int m = (256 * c + q) >> 4;
          const float4 tm = __ldg(reinterpret_cast<const float4*>(g.Tm + (row * g.M + m) * 4));
          float t1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int l = 0; l < 16; ++l) {
            const float4 tl = s_tl[rl * 16 + (l ^ (rl & 7))];
            t1[0] += v[l] * tl.x;
            t1[1] += v[l] * tl.y;
            t1[2] += v[l] * tl.z;
            t1[3] += v[l] * tl.w;
            ext[l][0] += v[l] * tm.x;
            ext[l][1] += v[l] * tm.y;
            ext[l][2] += v[l] * tm.z;
            ext[l][3] += v[l] * tm.w;
          }
          reinterpret_cast<float4*>(g.gT)[(long)m * rows + row] = make_float4(t1[0], t1[1], t1[2], t1[3]);
        } else {
          st_v8(dst + q, v);
          st_v8(dst + q + 8, v + 8);
        }
      }
    }
    tc_fence_before();
    mbar_arrive(&accfree[buf]);
  }
  if (gtm) {
    // term 2 of the rows' first 16 m: the parts' partial sums meet in the idle ring (every load and
    // MMA of the tile completed before the last chunk's accumulator became ready)
    float* s_ext = reinterpret_cast<float*>(smem);  // [kParts][128][64]
#pragma unroll
    for (int l = 0; l < 16; ++l)
      *reinterpret_cast<float4*>(s_ext + ((part * SBM) + rl) * 64 + l * 4) =
          make_float4(ext[l][0], ext[l][1], ext[l][2], ext[l][3]);
    bar_sync(1, kSEpi);
    if (rv)
      for (int l = part; l < 16; l += kParts) {
        float4 a = reinterpret_cast<float4*>(g.gT)[(long)l * rows + row];
        for (int pp = 0; pp < kParts; ++pp) {
          const float4 e = *reinterpret_cast<const float4*>(s_ext + ((pp * SBM) + rl) * 64 + l * 4);
          a.x += e.x;
          a.y += e.y;
          a.z += e.z;
          a.w += e.w;
        }
        reinterpret_cast<float4*>(g.gT)[(long)l * rows + row] = a;
      }
  }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kProd) tmem_dealloc(tmem, 512);
}

// ring, barriers, then either the forward's energies, biases and output weights or (dE/dT mode) T_< rows
size_t split_smem() {
  const size_t tail = std::max<size_t>((kParts * SBM + kSL * 256 + 256) * 4, (size_t)SBM * 16 * 16);
  return (size_t)kSRing * kSStage + 16 * 8 + 16 + tail + 1024;
}

}  // namespace

bool fit_split_supported(const DeviceModel& m) {
  const int nfl = m.n_fit_layers, nh = nfl - 1;
  if (nh < 1 || nh > kSL) return false;
  const int KD = m.M * m.A;
  if (KD % 16 != 0) return false;
  for (int t = 0; t < m.cfg.ntypes; ++t)
    for (int l = 0; l < nh; ++l) {
      const LayerDesc& L = m.fit[(size_t)t * nfl + l];
      const LayerDesc& L0 = m.fit[l];
      if (L.n_in != L0.n_in || L.n_out != L0.n_out || L.skip != L0.skip) return false;
      if (L.n_out % 16 || L.n_out > 256 || L.skip > 1 || (l == 0 && L.skip)) return false;
    }
  return m.fit[0].n_in == KD && m.fit_wt_bf16_lo != nullptr;
}

int run_fitting_split(const DeviceModel& m, const PathConst& pc, const __nv_bfloat16* Dhi, const __nv_bfloat16* Dlo,
                      const PathIO& io, Arena& ar, cudaStream_t st, const float** gD_out, const float* Tm,
                      float* gT) {
  const long N = pc.natoms;
  const int nfl = m.n_fit_layers, nh = nfl - 1;
  const int nt = pc.ntypes;
  const int KD = pc.M * pc.A;
  const bool gtm = gT != nullptr && Tm != nullptr && pc.A == 16;
  __nv_bfloat16* xs = ar.get<__nv_bfloat16>(4 * N * kSLd);
  float* gate = ar.get<float>((long)nh * N * kSLd);
  float* gD = gtm ? nullptr : ar.get<float>(N * KD);
  if (ar.measure) return DP_OK;
  if (!ar.ok()) {
    set_error("scratch allocation failed");
    return DP_E_OOM;
  }
  SplitArgs a;
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
    if (t < nt) tiles += (io.type_start[t + 1] - io.type_start[t] + SBM - 1) / SBM;
  }
  SplitMaps mp;
  std::memset(&mp, 0, sizeof(mp));
  int rc = make_tmap_bf16(&mp.d[0], Dhi, N, KD, SBM);
  if (rc == DP_OK) rc = make_tmap_bf16(&mp.d[1], Dlo, N, KD, SBM);
  for (int b = 0; rc == DP_OK && b < 2; ++b)
    for (int hl = 0; rc == DP_OK && hl < 2; ++hl) {
      a.xs[b][hl] = xs + (long)(2 * b + hl) * N * kSLd;
      rc = make_tmap_bf16(&mp.x[b][hl], a.xs[b][hl], N, kSLd, SBM);
      for (int t = 0; rc == DP_OK && t < nt; ++t) {
        const long n_t = io.type_start[t + 1] - io.type_start[t];
        if (n_t > 0)
          rc = make_tmap_bf16(&mp.xt[t][b][hl], a.xs[b][hl] + (long)io.type_start[t] * kSLd, n_t, kSLd, SBM);
      }
    }
  if (rc != DP_OK) return rc;
  const float* p32 = m.p32;
  for (int t = 0; t < nt; ++t) {
    for (int l = 0; l < nh; ++l) {
      const LayerDesc& L = m.fit[(size_t)t * nfl + l];
      a.bias[t][l] = p32 + L.w_off + (long)L.n_in * L.n_out;
      for (int hl = 0; hl < 2; ++hl) {
        const CUtensorMap* f = fit_weight_map(m, t, l, 0, L.n_out, hl == 1);
        const CUtensorMap* b = fit_weight_map(m, t, l, 1, l == 0 ? 256 : L.n_in, hl == 1);
        if (!f || !b) return DP_E_CUDA;
        mp.w[t][l][hl] = *f;
        mp.w[t][nh + l][hl] = *b;
      }
    }
    const LayerDesc& Lo = m.fit[(size_t)t * nfl + nh];
    a.w_last[t] = p32 + Lo.w_off;
    a.b_last[t] = m.fit_out_bias[t];
  }
  a.gate = gate;
  a.perm = io.perm;
  a.atom_e = io.atom_energy;
  a.gD = gD;
  a.gT = gtm ? gT : nullptr;
  a.Tm = Tm;
  a.M = pc.M;
  a.err = &io.status->timeout;
  if (tiles > 0) {
    ProfScope _ps(io.prof, "fit_split_tc", st);
    const size_t smem = split_smem();
    DP_CUDA_TRY(allow_max_smem(k_fit_split));
    k_fit_split<<<tiles, kSThreads, smem, st>>>(mp, a);
    DP_CUDA_TRY(cudaGetLastError());
  }
  *gD_out = gD;
  return DP_OK;
}

}  // namespace dpgb
