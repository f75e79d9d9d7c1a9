// Uncompressed path with the embedding and fitting GEMMs on the 5th-generation tensor cores:
// BF16 (DP_PREC_BF16) or TF32 (DP_PREC_TF32) operands, FP32 accumulation in tensor memory
// (Eqs. (G2), (NN), (fitting_energy)).
//
// Every dense layer after the scalar first embedding layer, forward and backward, is one launch
// of k_dense_tc: a 128-row tile per CTA, operands streamed by TMA through a shared-memory ring
// (128-byte swizzle), one thread issuing tcgen05.mma into a TMEM accumulator, eight epilogue
// warps applying the layer's bias, tanh, ResNet skip ({x,x} included), the 1 - t^2 gate of the
// backward pass, or the final linear layer of the fitting net.  The rows of one launch belong to
// several nets (one per (centre type, neighbour type) pair for the embedding, one per centre type
// for the fitting net): each tile takes its group's weight map.
//
// Per-slot arrays use a block-major order: row = N * sel_off[t] + p * sel[t] + (k - sel_off[t])
// for slot k (neighbour-type block t) of the p-th atom in type-sorted order, so the rows of one
// embedding net (atoms of one centre type, slots of one neighbour block) are contiguous.  The
// scalar first layer with the environment matrix, the contraction T = G^T R / Nc with
// D = T T_<^T, dE/dT -> dE/dG and dE/dR, and the first layer's backward with the force and
// virial scatter run on the CUDA cores (FP32; FP64 for the pair displacement and the scatter).
// Activation widths are padded to multiples of 16 with zero columns (zero weight rows), so that
// every operand row is 16-byte aligned for TMA.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "env.cuh"
#include "fit_tc.cuh"
#include "path.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace dpgb {

namespace {

using namespace ptx;

constexpr int kDThreads = 256;
constexpr int DBM = 128;
constexpr int kDStages = 4;
constexpr int kDGroups = DP_MAX_TYPES;

enum DenseMode : int { DM_FWD = 0, DM_FWD_LAST = 1, DM_BWD = 2, DM_PLAIN = 3 };

inline int pad16(int n) { return (n + 15) & ~15; }

struct DenseMaps {
  CUtensorMap a;
  CUtensorMap b[kDGroups];
};

struct DenseArgs {
  int ngroups;
  int row_start[kDGroups + 1];
  int tile_start[kDGroups + 1];
  int K, N, BN;  // reduction length, output width, output columns per CTA
  int ldo;       // row pitch (elements) of the outputs
  const float* bias[kDGroups];
  const float* wlast[kDGroups];
  float blast[kDGroups];
  int skip;  // FWD: 0, 1 (x[c]), 2 (x[c mod n_in]); BWD: 0, 1 (gy[c]), 2 (gy[c] + gy[c + N]), 3 (wlast[c])
  const float* skip_in;
  int ld_skip, n_in_skip;
  const float* tbelow;  // BWD: tanh outputs of the layer below (gate 1 - t^2), or null
  int ld_tb;
  float* out_y;  // FWD: y; BWD: g (or null); PLAIN: the product
  float* out_t;  // FWD: t
  void* out_a;   // next A operand (EB-byte elements), or null
  float* e_out;  // FWD_LAST: energy partial per column block [col blocks][e_ld]
  long e_ld;
  // embedding layers: the slot rows' environment rows; a row whose s is zero (padding) gets no
  // epilogue, and its outputs are left as they are (null: every row)
  const float4* zrow;
  int* err;
};

template <int EB>
__device__ __forceinline__ void store_a(void* base, long idx, float x) {
  if (EB == 2)
    reinterpret_cast<__nv_bfloat16*>(base)[idx] = __float2bfloat16_rn(x);
  else
    reinterpret_cast<float*>(base)[idx] = x;
}

// 16 consecutive values of one row (64-byte aligned: row pitches and column pieces are multiples
// of 16) as two 32-byte accesses, one full sector each: an epilogue thread owns a row, so scalar
// accesses would touch a different line per lane and per element.
__device__ __forceinline__ void ld16f(const float* p, float* v) {
  asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
               : "l"(p));
  asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15])
               : "l"(p + 8));
}
__device__ __forceinline__ void st16f(float* p, const float* v) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]),
               "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
               : "memory");
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p + 8), "f"(v[8]), "f"(v[9]),
               "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15])
               : "memory");
}
// 16 values of the next A operand at element index idx (a multiple of 16)
template <int EB>
__device__ __forceinline__ void store16_a(void* base, long idx, const float* x) {
  if (EB == 2) {
    uint32_t w[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
      w[i] = *reinterpret_cast<const uint32_t*>(&h);
    }
    __nv_bfloat16* p = reinterpret_cast<__nv_bfloat16*>(base) + idx;
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(w[0]), "r"(w[1]),
                 "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
                 : "memory");
  } else {
    st16f(reinterpret_cast<float*>(base) + idx, x);
  }
}

// tanh x = 1 - 2 / (1 + e^{2x}), x clamped to +-15 (where tanh is 1 to FP32): absolute error a few
// 1e-7, below the BF16 / TF32 rounding of the operands these layers feed.  The exponential takes
// the special-function unit; 1/d comes from the bit pattern of d (first guess within 5.1 %) and
// three Newton steps on the FMA pipe.
__device__ __forceinline__ float tanh_op(float x) {
  const float e = __expf(2.f * fminf(fmaxf(x, -15.f), 15.f));
  const float d = 1.f + e;
  float y = __int_as_float(0x7EF311C0 - __float_as_int(d));
  y = y * (2.f - d * y);
  y = y * (2.f - d * y);
  y = y * (2.f - d * y);
  return 1.f - 2.f * y;
}

// One dense layer (or its backward) on a 128-row tile: C = A . B^T on the tensor cores, then the
// epilogue of MODE.  A: [rows][K] (EB-byte elements), B^T: [N][K] per group.
template <int EB, int MODE>
__global__ void __launch_bounds__(kDThreads, 3)  // three CTAs per SM: the epilogues are latency-bound
    k_dense_tc(const __grid_constant__ DenseMaps mp, const DenseArgs g) {
  __shared__ float s_e[2][DBM];
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  constexpr int BK = 128 / EB;  // elements of one 128-byte row
  const int BN = g.BN;
  const uint32_t a_bytes = DBM * 128, b_bytes = (uint32_t)BN * 128, stage = a_bytes + b_bytes;
  const int nk = (g.K + BK - 1) / BK;
  const int NS = nk >= kDStages ? kDStages : (nk < 2 ? 2 : nk);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NS * stage);
  uint64_t* empty = full + kDStages;
  uint64_t* accf = empty + kDStages;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(accf + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int grp = 0;
  while (grp + 1 < g.ngroups && (int)blockIdx.x >= g.tile_start[grp + 1]) ++grp;
  const int row0 = g.row_start[grp] + ((int)blockIdx.x - g.tile_start[grp]) * DBM;
  const int row_end = g.row_start[grp + 1];
  const int col0 = blockIdx.y * BN;
  uint32_t ncols = 32;
  while ((int)ncols < BN) ncols <<= 1;
  if (g.zrow != nullptr) {  // a tile of zero environment rows only (padding) has nothing to compute
    const long r = row0 + threadIdx.x;
    const bool live = threadIdx.x < DBM && r < row_end && g.zrow[r].x != 0.f;
    if (!__syncthreads_or(live)) return;  // block-uniform
  }

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    mbar_fence_init();
  }
  if (warp == 0) tmem_alloc(tmem_holder, ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ----
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % NS;
      if (kb >= NS && !mbar_wait(&empty[s], ((kb / NS) - 1) & 1, g.err)) break;
      unsigned char* st = smem + s * stage;
      mbar_expect_tx(&full[s], stage);
      tma_load_2d(st, &mp.a, &full[s], kb * BK, row0);
      tma_load_2d(st + a_bytes, &mp.b[grp], &full[s], kb * BK, col0);
      issued = kb + 1;
    }
    // every copy this thread started has landed before the CTA may exit
    for (int s = 0; s < NS && s < issued; ++s) {
      const int last = s + NS * ((issued - 1 - s) / NS);
      mbar_wait(&full[s], (last / NS) & 1, g.err);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: four 32-byte K steps per 128-byte row ----
    const uint32_t idesc = EB == 2 ? idesc_f16(DBM, BN, 1) : idesc_tf32(DBM, BN);
    bool ok = true;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % NS;
      if (!mbar_wait(&full[s], (kb / NS) & 1, g.err)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t sa = su32(smem + s * stage);
      const uint64_t ad = sdesc_sw128(sa), bd = sdesc_sw128(sa + a_bytes);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (EB == 2)
          mma_f16(tmem, ad + 2 * k, bd + 2 * k, idesc, (kb | k) != 0);
        else
          mma_tf32(tmem, ad + 2 * k, bd + 2 * k, idesc, (kb | k) != 0);
      }
      mma_commit(&empty[s]);
    }
    if (ok && nk > 0)
      mma_commit(accf);
    else
      mbar_arrive(accf);
  }
  __syncwarp();

  // ---- epilogue: warps w and w + 4 own accumulator rows 32(w % 4) .. +31, alternate 16 columns ----
  mbar_wait(accf, 0, g.err);
  __syncwarp();
  tc_fence_after();
  const int quad = warp & 3, half = warp >> 2;
  const int rl = quad * 32 + lane;
  const long row = row0 + rl;
  const bool rv = row < row_end;
  const uint32_t tb = tmem + ((uint32_t)(quad * 32) << 16);
  const float* bias = g.bias[grp];
  const float* wl = g.wlast[grp];
  float e_acc = 0.f;
  // a zero environment row (padding) is read by nobody downstream: the contraction and the
  // descriptor backward stop at or skip zero rows, and the first layer's backward does not read the
  // rows of a pair whose s is zero
  const bool rz = rv && g.zrow != nullptr && g.zrow[row].x == 0.f;
  for (int c = half * 16; c < BN; c += 32) {
    float v[16];
    tmem_ld16(tb + c, v);
    const int cg0 = col0 + c;  // a piece is all inside the padded width or all beyond it
    if (!rv || rz || cg0 >= g.ldo) continue;
    const long o = row * g.ldo + cg0;
    if (MODE == DM_PLAIN) {
      float y[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) y[i] = cg0 + i < g.N ? v[i] : 0.f;
      st16f(g.out_y + o, y);
    } else if (MODE == DM_FWD || MODE == DM_FWD_LAST) {
      float xs[16];
      // n_out = n_in: the same padded width; {x, x} with n_in a multiple of 16: the piece's inputs are
      // 16 consecutive values too
      const bool xv = g.skip == 1 || (g.skip == 2 && (g.n_in_skip & 15) == 0);
      if (xv) ld16f(g.skip_in + row * g.ld_skip + (g.skip == 1 ? cg0 : cg0 % g.n_in_skip), xs);
      float y[16], t[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int cg = cg0 + i;
        float tt = 0.f, yy = 0.f;
        if (cg < g.N) {
          tt = tanh_op(v[i] + __ldg(bias + cg));
          yy = tt;
          if (xv) yy += xs[i];
          else if (g.skip == 2) yy += __ldg(g.skip_in + row * g.ld_skip + cg % g.n_in_skip);
        }
        y[i] = yy;
        t[i] = tt;
      }
      if (MODE == DM_FWD) {
        st16f(g.out_y + o, y);
        if (g.out_t) st16f(g.out_t + o, t);
        if (g.out_a) store16_a<EB>(g.out_a, o, y);
      } else {
        float ga[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int cg = cg0 + i;
          const float w = cg < g.N ? __ldg(wl + cg) : 0.f;
          e_acc += y[i] * w;
          ga[i] = w * (1.f - t[i] * t[i]);
        }
        store16_a<EB>(g.out_a, o, ga);
      }
    } else {  // DM_BWD
      float xs[16], tb16[16];
      if (g.skip == 1 || g.skip == 2) ld16f(g.skip_in + row * g.ld_skip + cg0, xs);  // gy[c]: the wider width
      const bool x2v = g.skip == 2 && (g.N & 15) == 0;  // gy[c + N] as 16 consecutive values too
      if (x2v) {
        float x2[16];
        ld16f(g.skip_in + row * g.ld_skip + cg0 + g.N, x2);
#pragma unroll
        for (int i = 0; i < 16; ++i) xs[i] += x2[i];
      }
      if (g.tbelow) ld16f(g.tbelow + row * g.ld_tb + cg0, tb16);
      float gyv[16], gzv[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int cg = cg0 + i;
        float gy = 0.f, gz = 0.f;
        if (cg < g.N) {
          gy = v[i];
          if (g.skip == 1) gy += xs[i];
          if (g.skip == 2) gy += xs[i] + (x2v ? 0.f : __ldg(g.skip_in + row * g.ld_skip + cg + g.N));
          if (g.skip == 3) gy += __ldg(wl + cg);
          gz = g.tbelow ? gy * (1.f - tb16[i] * tb16[i]) : gy;
        }
        gyv[i] = gy;
        gzv[i] = gz;
      }
      if (g.out_y) st16f(g.out_y + o, gyv);
      if (g.out_a) store16_a<EB>(g.out_a, o, gzv);
    }
  }
  if (MODE == DM_FWD_LAST) {
    s_e[half][rl] = e_acc;
    __syncthreads();
    if (half == 0 && rv)
      g.e_out[(long)blockIdx.y * g.e_ld + row] = s_e[0][rl] + s_e[1][rl] + (blockIdx.y == 0 ? g.blast[grp] : 0.f);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

size_t dense_smem(int K, int BN, int EB) {
  const int BK = 128 / EB;
  const int nk = (K + BK - 1) / BK;
  const int NS = nk >= kDStages ? kDStages : (nk < 2 ? 2 : nk);
  return (size_t)NS * (DBM * 128 + (size_t)BN * 128) + 1024 + 256;
}

template <int EB, int MODE>
cudaError_t launch_dense_mode(dim3 grid, size_t smem, const DenseMaps& mp, const DenseArgs& a, cudaStream_t st) {
  cudaError_t e = allow_max_smem(k_dense_tc<EB, MODE>);
  if (e == cudaSuccess) k_dense_tc<EB, MODE><<<grid, kDThreads, smem, st>>>(mp, a);
  return e;
}

template <int EB>
cudaError_t launch_dense(int mode, const DenseMaps& mp, const DenseArgs& a, cudaStream_t st) {
  const int tiles = a.tile_start[a.ngroups];
  if (tiles <= 0) return cudaSuccess;
  dim3 grid(tiles, (a.ldo + a.BN - 1) / a.BN);
  const size_t smem = dense_smem(a.K, a.BN, EB);
  cudaError_t e;
  switch (mode) {
    case DM_FWD:
      e = launch_dense_mode<EB, DM_FWD>(grid, smem, mp, a, st);
      break;
    case DM_FWD_LAST:
      e = launch_dense_mode<EB, DM_FWD_LAST>(grid, smem, mp, a, st);
      break;
    case DM_BWD:
      e = launch_dense_mode<EB, DM_BWD>(grid, smem, mp, a, st);
      break;
    default:
      e = launch_dense_mode<EB, DM_PLAIN>(grid, smem, mp, a, st);
      break;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// Columns per CTA: the padded width in one block when that gives enough CTAs, else blocks of a
// multiple of 16 so that the grid covers the SMs about twice.
int pick_bn(int ldo, int tiles) {
  int bn = std::min(ldo, 256);
  while (bn > 64 && (long)tiles * ((ldo + bn - 1) / bn) < 2L * 152) bn = ((bn / 2) + 15) & ~15;
  return bn;
}

// ---- block-major slot rows -------------------------------------------------------------------
__device__ __forceinline__ long brow(const PathConst& pc, int p, int k, int t) {
  return (long)pc.natoms * pc.sel_off[t] + (long)p * pc.sel[t] + (k - pc.sel_off[t]);
}
__device__ __forceinline__ int block_of_slot(const PathConst& pc, int k) {
  int t = 0;
  while (t + 1 < pc.ntypes && k >= pc.sel_off[t + 1]) ++t;
  return t;
}

// R of every slot and the scalar first embedding layer (1 -> w1): y0 = tanh(s w + b) (+ s).
template <int EB>
__global__ void k_env_l0(PathConst pc, const double* __restrict__ coord, const int* __restrict__ perm,
                         const int* __restrict__ tsorted, const int* __restrict__ nl_j, const int* __restrict__ nl_code,
                         NetPtrs<float> nets, int w1, int ld1, int skip, float4* __restrict__ Renv,
                         float* __restrict__ Y0, float* __restrict__ T0, void* __restrict__ A0) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)pc.natoms * pc.nc) return;
  const int p = (int)(e / pc.nc), k = (int)(e % pc.nc);
  const int t = block_of_slot(pc, k);
  const long row = brow(pc, p, k, t);
  const int i = perm[p];
  const int j = nl_j[(long)i * pc.nc + k];
  float o[4] = {0.f, 0.f, 0.f, 0.f};
  if (j >= 0) {
    double d0, d1, d2;
    listed_disp(coord + 3 * i, coord + 3 * j, nl_code[(long)i * pc.nc + k], pc, frame_of(pc, i), d0, d1, d2);
    float r, s, ds, u[3];
    pair_env<float>(d0, d1, d2, norm2_exact(d0, d1, d2), pc.rs, pc.rc, pc.near2, r, s, ds, u);
    o[0] = s;
    o[1] = s * u[0];
    o[2] = s * u[1];
    o[3] = s * u[2];
  }
  Renv[row] = make_float4(o[0], o[1], o[2], o[3]);
  if (o[0] == 0.f) return;  // a zero row: its layer outputs are read by nobody (see k_dense_tc)
  const int net = pc.type_one_side ? t : tsorted[p] * pc.ntypes + t;
  const float* w = nets.w0[net];
  const float* b = nets.b0[net];
  for (int c0 = 0; c0 < ld1; c0 += 16) {  // ld1 is a multiple of 16: 16-value vector stores per row
    float tv[16], yv[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int c = c0 + q;
      float tt = 0.f, y = 0.f;
      if (c < w1) {
        tt = tanh_op(o[0] * __ldg(w + c) + __ldg(b + c));
        y = tt + (skip ? o[0] : 0.f);
      }
      tv[q] = tt;
      yv[q] = y;
    }
    st16f(Y0 + row * ld1 + c0, yv);
    st16f(T0 + row * ld1 + c0, tv);
    if (A0) store16_a<EB>(A0, row * ld1 + c0, yv);
  }
}

// T = G^T R / Nc and D = T T_<^T, one block per atom; D also as the fitting net's A operand.
template <int EB>
__global__ void k_contract_b(PathConst pc, const float* __restrict__ G, int ldg, const float4* __restrict__ Renv,
                             float4* __restrict__ Tm, float* __restrict__ D, void* __restrict__ Da) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  float* Ts = reinterpret_cast<float*>(sm_raw);  // [M][4]
  const int p = blockIdx.x;
  const int M = pc.M, A = pc.A;
  const float inv_nc = 1.f / (float)pc.nc;
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    for (int t = 0; t < pc.ntypes; ++t)
      for (int k = pc.sel_off[t]; k < pc.sel_off[t + 1]; ++k) {
        const long row = brow(pc, p, k, t);
        const float4 r4 = Renv[row];
        // the block's real neighbours come first, nearest first, and s falls with r: past the first
        // zero row (padding, or s rounded to zero just inside r_c) every row adds zero
        if (r4.x == 0.f) break;
        const float gv = G[row * ldg + m];
        a0 += gv * r4.x;
        a1 += gv * r4.y;
        a2 += gv * r4.z;
        a3 += gv * r4.w;
      }
    a0 *= inv_nc;
    a1 *= inv_nc;
    a2 *= inv_nc;
    a3 *= inv_nc;
    Ts[m * 4] = a0;
    Ts[m * 4 + 1] = a1;
    Ts[m * 4 + 2] = a2;
    Ts[m * 4 + 3] = a3;
    Tm[(long)p * M + m] = make_float4(a0, a1, a2, a3);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < M * A; idx += blockDim.x) {
    const int m = idx / A, l = idx % A;
    const float d = Ts[m * 4] * Ts[l * 4] + Ts[m * 4 + 1] * Ts[l * 4 + 1] + Ts[m * 4 + 2] * Ts[l * 4 + 2] +
                    Ts[m * 4 + 3] * Ts[l * 4 + 3];
    D[(long)p * M * A + idx] = d;
    if (Da) store_a<EB>(Da, (long)p * M * A + idx, d);
  }
}

// dE/dT from dE/dD, then per slot dE/dR (gR) and dE/dG (gG, FP32) and the last embedding layer's
// backward operand gz = dE/dG (1 - t^2) (EB-byte elements); one block per atom.
template <int EB>
__global__ void k_descr_bwd_b(PathConst pc, const float4* __restrict__ Tm, const float* __restrict__ gD,
                              const float* __restrict__ G, const float* __restrict__ Tlast, int ldg,
                              const float4* __restrict__ Renv, float* __restrict__ gG, void* __restrict__ gZ,
                              float4* __restrict__ gR) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int M = pc.M, A = pc.A;
  float* Ts = reinterpret_cast<float*>(sm_raw);  // [M][4]
  float* gTs = Ts + M * 4;                       // [M][4]
  float* gDs = gTs + M * 4;                      // [M][A]
  const int p = blockIdx.x;
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    const float4 t4 = Tm[(long)p * M + m];
    Ts[m * 4] = t4.x;
    Ts[m * 4 + 1] = t4.y;
    Ts[m * 4 + 2] = t4.z;
    Ts[m * 4 + 3] = t4.w;
  }
  for (int e = threadIdx.x; e < M * A; e += blockDim.x) gDs[e] = gD[(long)p * M * A + e];
  __syncthreads();
  for (int e = threadIdx.x; e < M * 4; e += blockDim.x) {
    const int m = e / 4, c = e % 4;
    float acc = 0.f;
    for (int l = 0; l < A; ++l) acc += gDs[m * A + l] * Ts[l * 4 + c];
    if (m < A)
      for (int q = 0; q < M; ++q) acc += gDs[q * A + m] * Ts[q * 4 + c];
    gTs[e] = acc;
  }
  __syncthreads();
  const float inv_nc = 1.f / (float)pc.nc;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int k = warp; k < pc.nc; k += nw) {
    const int t = block_of_slot(pc, k);
    const long row = brow(pc, p, k, t);
    const float4 r4 = Renv[row];
    // a zero row (padding, or s rounded to zero within ~1e-15 of r_c) is read by nobody downstream:
    // the embedding layers' backward epilogues skip it and the first layer's backward does not read
    // the rows of a pair whose s is zero
    if (r4.x == 0.f) continue;  // warp-uniform
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    for (int m = lane; m < ldg; m += 32) {
      float gg = 0.f, gz = 0.f;
      if (m < M) {
        const float gv = G[row * ldg + m];
        a0 += gTs[m * 4] * gv;
        a1 += gTs[m * 4 + 1] * gv;
        a2 += gTs[m * 4 + 2] * gv;
        a3 += gTs[m * 4 + 3] * gv;
        gg = (gTs[m * 4] * r4.x + gTs[m * 4 + 1] * r4.y + gTs[m * 4 + 2] * r4.z + gTs[m * 4 + 3] * r4.w) * inv_nc;
        const float tt = Tlast[row * ldg + m];
        gz = gg * (1.f - tt * tt);
      }
      gG[row * ldg + m] = gg;
      store_a<EB>(gZ, row * ldg + m, gz);
    }
    for (int off = 16; off > 0; off >>= 1) {
      a0 += __shfl_xor_sync(0xffffffffu, a0, off);
      a1 += __shfl_xor_sync(0xffffffffu, a1, off);
      a2 += __shfl_xor_sync(0xffffffffu, a2, off);
      a3 += __shfl_xor_sync(0xffffffffu, a3, off);
    }
    if (lane == 0) gR[row] = make_float4(a0 * inv_nc, a1 * inv_nc, a2 * inv_nc, a3 * inv_nc);
  }
}

// Backward of the scalar first layer (dE/ds from dE/dy0), then dE/dr_ij and the FP64 force and
// virial scatter.
__global__ void __launch_bounds__(256)
    k_l0_bwd_force(PathConst pc, const double* __restrict__ coord, const int* __restrict__ perm,
                   const int* __restrict__ tsorted, const int* __restrict__ nl_j, const int* __restrict__ nl_code,
                   NetPtrs<float> nets, int w1, int ld1, int skip, const float* __restrict__ G0,
                   const float* __restrict__ T0, const float4* __restrict__ gR, double* __restrict__ force,
                   double* __restrict__ avir) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long)pc.natoms * pc.nc) return;
  const int p = (int)(e / pc.nc), k = (int)(e % pc.nc);
  const int i = perm[p];
  const int j = nl_j[(long)i * pc.nc + k];
  if (j < 0) return;
  const int t = block_of_slot(pc, k);
  const long row = brow(pc, p, k, t);
  const int net = pc.type_one_side ? t : tsorted[p] * pc.ntypes + t;
  const float* w = nets.w0[net];
  double d[3];
  listed_disp(coord + 3 * i, coord + 3 * j, nl_code[(long)i * pc.nc + k], pc, frame_of(pc, i), d[0], d[1], d[2]);
  float r, s, ds, u[3];
  pair_env<float>(d[0], d[1], d[2], norm2_exact(d[0], d[1], d[2]), pc.rs, pc.rc, pc.near2, r, s, ds, u);
  // a pair whose s rounded to zero (within ~1e-15 of r_c) had no layer epilogues: its rows are not
  // read, and its force terms (s = 0, |ds/dr| below 1e-29) are zero
  if (s == 0.f) return;
  float gs = 0.f;
  for (int c = 0; c < w1; ++c) {
    const float gy = G0[row * ld1 + c], tt = T0[row * ld1 + c];
    gs += gy * (1.f - tt * tt) * __ldg(w + c);
    if (skip) gs += gy;
  }
  const float4 g4 = gR[row];
  const float gvu = g4.y * u[0] + g4.z * u[1] + g4.w * u[2];
  const float a = ds * (gs + g4.x + gvu), b = s / r;
  const float gv[3] = {g4.y, g4.z, g4.w};
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

__global__ void k_types_of_sorted(const int* __restrict__ type, const int* __restrict__ perm, int n,
                                  int* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) out[p] = type[perm[p]];
}

unsigned nblk(long n, int b) { return (unsigned)((n + b - 1) / b); }

// Weight operands of one layer: forward B^T = W^T [n_out][ld_in], backward B^T = W [n_in][ld_out]
// (zero-padded to multiples of 16), in EB-byte elements, into host buffers at `off`.
void put_layer(const double* W, int n_in, int n_out, int EB, std::vector<unsigned char>& fwd,
               std::vector<unsigned char>& bwd, long off) {
  const int li = pad16(n_in), lo = pad16(n_out);
  auto put = [&](std::vector<unsigned char>& v, long idx, double x) {
    if (EB == 2) {
      const float f = (float)x;
      uint32_t u;
      std::memcpy(&u, &f, 4);
      if ((u & 0x7F800000u) != 0x7F800000u) u += 0x7FFFu + ((u >> 16) & 1u);
      const uint16_t h = (uint16_t)(u >> 16);
      std::memcpy(&v[(size_t)(off + idx) * 2], &h, 2);
    } else {
      const float f = (float)x;
      std::memcpy(&v[(size_t)(off + idx) * 4], &f, 4);
    }
  };
  for (int i = 0; i < n_in; ++i)
    for (int o = 0; o < n_out; ++o) {
      put(fwd, (long)o * li + i, W[(long)i * n_out + o]);
      put(bwd, (long)i * lo + o, W[(long)i * n_out + o]);
    }
}

}  // namespace

bool tc_uncompressed_supported(const DeviceModel& m) {
  const int nt = m.cfg.ntypes;
  const int groups = m.cfg.type_one_side ? nt * nt : nt * nt;  // row groups of one launch: (centre, neighbour) pairs
  if (groups > kDGroups || m.cfg.n_embed < 2 || m.n_fit_layers < 2) return false;
  for (int l = 0; l < m.cfg.n_embed; ++l)
    if (m.cfg.embed[l] > 256) return false;
  for (int l = 0; l + 1 < m.n_fit_layers; ++l)
    if (m.fit[l].n_out > 256 || m.fit[l].skip == 2) return false;
  if ((m.M * m.A) % 16) return false;
  return true;
}

int tc_uncompressed_prepare(DeviceModel& m, const double* params_host) {
  const int EB = m.precision == DP_PREC_TF32 ? 4 : 2;
  const int ne = m.cfg.n_embed, nfl = m.n_fit_layers;
  // offsets (elements) of every layer's operands: embedding layers l >= 1 of every net, then the
  // hidden fitting layers of every type; each padded to 16 elements
  long total = 0;
  m.tc_off.clear();
  for (int n = 0; n < m.n_embed_nets; ++n)
    for (int l = 0; l < ne; ++l) {
      const LayerDesc& L = m.emb[(size_t)n * ne + l];
      m.tc_off.push_back(total);
      if (l > 0) total += (long)std::max(pad16(L.n_in) * L.n_out, pad16(L.n_out) * L.n_in) + 16;
    }
  for (int t = 0; t < m.cfg.ntypes; ++t)
    for (int l = 0; l < nfl; ++l) {
      const LayerDesc& L = m.fit[(size_t)t * nfl + l];
      m.tc_off.push_back(total);
      if (l + 1 < nfl) total += (long)std::max(pad16(L.n_in) * L.n_out, pad16(L.n_out) * L.n_in) + 16;
    }
  std::vector<unsigned char> fwd((size_t)total * EB, 0), bwd((size_t)total * EB, 0);
  size_t q = 0;
  for (int n = 0; n < m.n_embed_nets; ++n)
    for (int l = 0; l < ne; ++l, ++q) {
      const LayerDesc& L = m.emb[(size_t)n * ne + l];
      if (l > 0) put_layer(params_host + L.w_off, L.n_in, L.n_out, EB, fwd, bwd, m.tc_off[q]);
    }
  for (int t = 0; t < m.cfg.ntypes; ++t)
    for (int l = 0; l < nfl; ++l, ++q) {
      const LayerDesc& L = m.fit[(size_t)t * nfl + l];
      if (l + 1 < nfl) put_layer(params_host + L.w_off, L.n_in, L.n_out, EB, fwd, bwd, m.tc_off[q]);
    }
  DP_CUDA_TRY(cudaMalloc(&m.tc_wt, fwd.size()));
  DP_CUDA_TRY(cudaMalloc(&m.tc_w, bwd.size()));
  DP_CUDA_TRY(cudaMemcpy(m.tc_wt, fwd.data(), fwd.size(), cudaMemcpyHostToDevice));
  DP_CUDA_TRY(cudaMemcpy(m.tc_w, bwd.data(), bwd.size(), cudaMemcpyHostToDevice));
  return DP_OK;
}

namespace {

template <int EB>
int run_tc_impl(const DeviceModel& m, const PathConst& pc0, const PathIO& io, Arena& ar, cudaStream_t st) {
  PathConst pc = pc0;
  const long N = pc.natoms, nc = pc.nc, rows = N * nc;
  const int M = pc.M, A = pc.A, ne = m.cfg.n_embed, nfl = m.n_fit_layers, nh = nfl - 1, nt = pc.ntypes;
  const int KD = M * A;
  // ---- scratch ----
  float4* Renv = ar.get<float4>(rows);
  std::vector<float*> Ye(ne), Te(ne);
  std::vector<void*> Ae(ne);
  std::vector<int> ld(ne);
  for (int l = 0; l < ne; ++l) {
    ld[l] = pad16(m.cfg.embed[l]);
    Ye[l] = ar.get<float>(rows * ld[l]);
    Te[l] = ar.get<float>(rows * ld[l]);
    Ae[l] = EB == 2 ? (void*)ar.get<__nv_bfloat16>(rows * ld[l]) : (void*)Ye[l];
  }
  const int ldM = ld[ne - 1];
  float4* Tm = ar.get<float4>(N * M);
  float* D = ar.get<float>(N * KD);
  void* Da = EB == 2 ? (void*)ar.get<__nv_bfloat16>(N * KD) : (void*)D;
  // fitting
  std::vector<float*> Yf(nh), Tf(nh), gY(nh);
  std::vector<void*> Af(nh), gZ(nh);
  std::vector<int> ldf(nh);
  for (int l = 0; l < nh; ++l) {
    ldf[l] = pad16(m.fit[l].n_out);
    Yf[l] = ar.get<float>(N * ldf[l]);
    Tf[l] = ar.get<float>(N * ldf[l]);
    gY[l] = ar.get<float>(N * ldf[l]);
    Af[l] = EB == 2 ? (void*)ar.get<__nv_bfloat16>(N * ldf[l]) : (void*)Yf[l];
    gZ[l] = EB == 2 ? (void*)ar.get<__nv_bfloat16>(N * ldf[l]) : (void*)ar.get<float>(N * ldf[l]);
  }
  const int nEb = (ldf[nh - 1] + 63) / 64 + 4;  // energy partial blocks (upper bound)
  float* E = ar.get<float>(N * nEb);
  float* gD = ar.get<float>(N * KD);
  // embedding backward
  int maxld = 16;
  for (int l = 0; l < ne; ++l) maxld = std::max(maxld, ld[l]);
  float* gyA = ar.get<float>(rows * maxld);
  float* gyB = ar.get<float>(rows * maxld);
  void* gzA = EB == 2 ? (void*)ar.get<__nv_bfloat16>(rows * maxld) : (void*)ar.get<float>(rows * maxld);
  void* gzB = EB == 2 ? (void*)ar.get<__nv_bfloat16>(rows * maxld) : (void*)ar.get<float>(rows * maxld);
  float4* gR = ar.get<float4>(rows);
  int* tsorted = ar.get<int>(N);
  if (ar.measure) return DP_OK;
  if (!ar.ok()) {
    set_error("scratch allocation failed");
    return DP_E_OOM;
  }
  const float* p32 = m.p32;
  const unsigned char* wt = static_cast<const unsigned char*>(m.tc_wt);
  const unsigned char* wb = static_cast<const unsigned char*>(m.tc_w);
  auto off_emb = [&](int net, int l) { return m.tc_off[(size_t)net * ne + l]; };
  auto off_fit = [&](int t, int l) { return m.tc_off[(size_t)m.n_embed_nets * ne + (size_t)t * nfl + l]; };
  // row groups of the embedding launches: nets in block-major row order
  DenseArgs eg;
  std::memset(&eg, 0, sizeof(eg));
  std::vector<int> gnet;
  {
    int ng = 0, tiles = 0;
    for (int tj = 0; tj < nt; ++tj)
      for (int ti = 0; ti < nt; ++ti) {
        const long r0 = N * pc.sel_off[tj] + (long)io.type_start[ti] * pc.sel[tj];
        const long r1 = N * pc.sel_off[tj] + (long)io.type_start[ti + 1] * pc.sel[tj];
        eg.row_start[ng] = (int)r0;
        eg.tile_start[ng] = tiles;
        tiles += (int)((r1 - r0 + DBM - 1) / DBM);
        gnet.push_back(pc.type_one_side ? tj : ti * nt + tj);
        ++ng;
        eg.row_start[ng] = (int)r1;
      }
    eg.ngroups = ng;
    eg.tile_start[ng] = tiles;
  }
  if (rows >= (1L << 31) / 2) {
    set_error("tensor-core embedding: too many neighbour slots in one call");
    return DP_E_UNSUPPORTED;
  }
  eg.err = &io.status->timeout;
  eg.zrow = Renv;
  DenseArgs fg;
  std::memset(&fg, 0, sizeof(fg));
  {
    int tiles = 0;
    for (int t = 0; t <= nt; ++t) {
      fg.row_start[t] = io.type_start[t];
      fg.tile_start[t] = tiles;
      if (t < nt) tiles += (io.type_start[t + 1] - io.type_start[t] + DBM - 1) / DBM;
    }
    fg.ngroups = nt;
  }
  fg.err = &io.status->timeout;
  constexpr int BKE = 128 / EB;
  auto mapA = [&](CUtensorMap* mp, const void* base, long r, int cols) {
    return make_tmap_2d(mp, base, EB, r, cols, BKE, DBM);
  };
  auto mapB = [&](CUtensorMap* mp, const unsigned char* base, long off, int r, int cols, int box_rows) {
    return make_tmap_2d(mp, base + off * EB, EB, r, cols, BKE, box_rows);
  };
  // ---- forward: R and the first layer, then the GEMM layers of the embedding ----
  {
    ProfScope _ps(io.prof, "sorted_types", st);
    k_types_of_sorted<<<nblk(N, 256), 256, 0, st>>>(io.type, io.perm, (int)N, tsorted);
  }
  NetPtrs<float> nets;
  for (int n = 0; n < m.n_embed_nets; ++n) {
    const LayerDesc& L0 = m.emb[(size_t)n * ne];
    nets.w0[n] = p32 + L0.w_off;
    nets.b0[n] = p32 + L0.w_off + L0.n_out;
  }
  const int w1 = m.cfg.embed[0];
  {
    ProfScope _ps(io.prof, "env_l0", st);
    k_env_l0<EB><<<nblk(rows, 256), 256, 0, st>>>(pc, io.coord, io.perm, tsorted, io.nl_j, io.nl_code, nets, w1,
                                                   ld[0], m.emb[0].skip, Renv, Ye[0], Te[0], EB == 2 ? Ae[0] : nullptr);
  }
  for (int l = 1; l < ne; ++l) {
    DenseArgs a = eg;
    const LayerDesc& L = m.emb[l];
    a.K = L.n_in;
    a.N = L.n_out;
    a.ldo = ld[l];
    a.BN = pick_bn(a.ldo, a.tile_start[a.ngroups]);
    DenseMaps mp;
    std::memset(&mp, 0, sizeof(mp));
    int rc = mapA(&mp.a, Ae[l - 1], rows, ld[l - 1]);
    for (int q = 0; rc == DP_OK && q < a.ngroups; ++q) {
      const LayerDesc& Lq = m.emb[(size_t)gnet[q] * ne + l];
      rc = mapB(&mp.b[q], wt, off_emb(gnet[q], l), Lq.n_out, pad16(Lq.n_in), a.BN);
      a.bias[q] = p32 + Lq.w_off + (long)Lq.n_in * Lq.n_out;
    }
    if (rc != DP_OK) return rc;
    a.skip = L.skip;
    a.skip_in = Ye[l - 1];
    a.ld_skip = ld[l - 1];
    a.n_in_skip = L.n_in;
    a.out_y = Ye[l];
    a.out_t = Te[l];
    a.out_a = EB == 2 ? Ae[l] : nullptr;
    ProfScope _ps(io.prof, "emb_fwd_tc", st);
    DP_CUDA_TRY(launch_dense<EB>(DM_FWD, mp, a, st));
  }
  const float* G = Ye[ne - 1];
  {
    ProfScope _ps(io.prof, "contract", st);
    k_contract_b<EB><<<(unsigned)N, 128, sizeof(float) * M * 4, st>>>(pc, G, ldM, Renv, Tm, D,
                                                                      EB == 2 ? Da : nullptr);
  }
  // ---- fitting net, forward ----
  for (int l = 0; l < nh; ++l) {
    const bool last = (l == nh - 1);
    DenseArgs a = fg;
    const LayerDesc& L = m.fit[l];
    a.K = L.n_in;
    a.N = L.n_out;
    a.ldo = ldf[l];
    a.BN = pick_bn(a.ldo, a.tile_start[a.ngroups]);
    DenseMaps mp;
    std::memset(&mp, 0, sizeof(mp));
    int rc = mapA(&mp.a, l == 0 ? Da : Af[l - 1], N, l == 0 ? KD : ldf[l - 1]);
    for (int t = 0; rc == DP_OK && t < nt; ++t) {
      const LayerDesc& Lt = m.fit[(size_t)t * nfl + l];
      rc = mapB(&mp.b[t], wt, off_fit(t, l), Lt.n_out, pad16(Lt.n_in), a.BN);
      a.bias[t] = p32 + Lt.w_off + (long)Lt.n_in * Lt.n_out;
      const LayerDesc& Lo = m.fit[(size_t)t * nfl + nh];
      a.wlast[t] = p32 + Lo.w_off;
      a.blast[t] = m.fit_out_bias[t];
    }
    if (rc != DP_OK) return rc;
    a.skip = L.skip;
    a.skip_in = l > 0 ? Yf[l - 1] : nullptr;
    a.ld_skip = l > 0 ? ldf[l - 1] : 0;
    a.n_in_skip = L.n_in;
    if (!last) {
      a.out_y = Yf[l];
      a.out_t = Tf[l];
      a.out_a = EB == 2 ? Af[l] : nullptr;
    } else {
      a.out_a = gZ[l];
      a.e_out = E;
      a.e_ld = N;
    }
    ProfScope _ps(io.prof, last ? "fit_fwd_last_tc" : "fit_fwd_tc", st);
    DP_CUDA_TRY(launch_dense<EB>(last ? DM_FWD_LAST : DM_FWD, mp, a, st));
  }
  {
    ProfScope _ps(io.prof, "energy_sum", st);
    const int bn = pick_bn(ldf[nh - 1], fg.tile_start[nt]);
    DP_CUDA_TRY(launch_energy_f32(E, (ldf[nh - 1] + bn - 1) / bn, io.perm, (int)N, io.atom_energy, st));
  }
  // ---- fitting net, backward to dE/dD ----
  for (int l = nh - 1; l >= 0; --l) {
    DenseArgs a = fg;
    const LayerDesc& L = m.fit[l];
    a.K = L.n_out;
    a.N = L.n_in;
    a.ldo = l == 0 ? KD : ldf[l - 1];
    a.BN = pick_bn(a.ldo, a.tile_start[a.ngroups]);
    DenseMaps mp;
    std::memset(&mp, 0, sizeof(mp));
    int rc = mapA(&mp.a, gZ[l], N, ldf[l]);
    for (int t = 0; rc == DP_OK && t < nt; ++t) {
      const LayerDesc& Lt = m.fit[(size_t)t * nfl + l];
      rc = mapB(&mp.b[t], wb, off_fit(t, l), Lt.n_in, pad16(Lt.n_out), a.BN);
      const LayerDesc& Lo = m.fit[(size_t)t * nfl + nh];
      a.wlast[t] = p32 + Lo.w_off;
    }
    if (rc != DP_OK) return rc;
    if (l == 0) {
      a.out_y = gD;
      ProfScope _ps(io.prof, "fit_bwd_tc", st);
      DP_CUDA_TRY(launch_dense<EB>(DM_PLAIN, mp, a, st));
    } else {
      a.skip = (l == nh - 1) ? (L.skip ? 3 : 0) : L.skip;
      a.skip_in = (l == nh - 1) ? nullptr : gY[l];
      a.ld_skip = ldf[l];
      a.tbelow = Tf[l - 1];
      a.ld_tb = ldf[l - 1];
      a.out_y = gY[l - 1];
      a.out_a = gZ[l - 1];
      ProfScope _ps(io.prof, "fit_bwd_tc", st);
      DP_CUDA_TRY(launch_dense<EB>(DM_BWD, mp, a, st));
    }
  }
  // ---- descriptor backward, then the embedding backward ----
  {
    ProfScope _ps(io.prof, "descr_bwd", st);
    k_descr_bwd_b<EB><<<(unsigned)N, 128, sizeof(float) * (M * 8 + M * A), st>>>(pc, Tm, gD, G, Te[ne - 1], ldM, Renv,
                                                                                 gyA, gzA, gR);
  }
  float* gy = gyA;
  float* gyn = gyB;
  void* gz = gzA;
  void* gzn = gzB;
  for (int l = ne - 1; l >= 1; --l) {
    DenseArgs a = eg;
    const LayerDesc& L = m.emb[l];
    a.K = L.n_out;
    a.N = L.n_in;
    a.ldo = ld[l - 1];
    a.BN = pick_bn(a.ldo, a.tile_start[a.ngroups]);
    DenseMaps mp;
    std::memset(&mp, 0, sizeof(mp));
    int rc = mapA(&mp.a, gz, rows, ld[l]);
    for (int q = 0; rc == DP_OK && q < a.ngroups; ++q) {
      const LayerDesc& Lq = m.emb[(size_t)gnet[q] * ne + l];
      rc = mapB(&mp.b[q], wb, off_emb(gnet[q], l), Lq.n_in, pad16(Lq.n_out), a.BN);
    }
    if (rc != DP_OK) return rc;
    a.skip = L.skip;
    a.skip_in = gy;
    a.ld_skip = ld[l];
    a.tbelow = l - 1 >= 1 ? Te[l - 1] : nullptr;  // layer 0's gate is applied with its weights below
    a.ld_tb = ld[l - 1];
    a.out_y = gyn;
    a.out_a = l - 1 >= 1 ? gzn : nullptr;
    ProfScope _ps(io.prof, "emb_bwd_tc", st);
    DP_CUDA_TRY(launch_dense<EB>(DM_BWD, mp, a, st));
    std::swap(gy, gyn);
    std::swap(gz, gzn);
  }
  {
    ProfScope _ps(io.prof, "force", st);
    k_l0_bwd_force<<<nblk(rows, 256), 256, 0, st>>>(pc, io.coord, io.perm, tsorted, io.nl_j, io.nl_code, nets, w1,
                                                    ld[0], m.emb[0].skip, gy, Te[0], gR, io.force, io.atom_virial);
  }
  DP_CUDA_TRY(cudaGetLastError());
  return DP_OK;
}

}  // namespace

int run_tc_uncompressed(const DeviceModel& m, const PathConst& pc, const PathIO& io, Arena& ar, cudaStream_t st) {
  if (m.precision == DP_PREC_TF32) return run_tc_impl<4>(m, pc, io, ar, st);
  return run_tc_impl<2>(m, pc, io, ar, st);
}

}  // namespace dpgb
