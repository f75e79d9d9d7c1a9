// Tensor-core GEMM (tcgen05 MMA, TMA operand staging, TMEM accumulators) with the fused
// epilogues of the fitting-net layers, Eq. (NN).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include "dp_internal.cuh"

namespace dpgb {

enum TcEpilogue : int {
  TC_EPI_PLAIN = 0,     // C = acc                                          (fp32 or bf16 out)
  TC_EPI_FWD = 1,       // t = tanh(acc + b); y = t + skip(x)               (y fp32, y bf16, t fp32)
  TC_EPI_FWD_LAST = 2,  // as FWD, then E = y . w_last + b_last and the backward seed
                        //   gz = w_last * (1 - t^2) of the last hidden layer (E fp32, gz bf16)
  TC_EPI_BWD = 3,       // g = acc + skip^T(gy); gz = g * (1 - t_below^2)   (g fp32, gz bf16)
};

// One B operand (weights) per atom type: the rows of each type are contiguous.
struct TcMaps {
  CUtensorMap m[DP_MAX_TYPES];
};

struct TcArgs {
  int ntypes;
  int row_start[DP_MAX_TYPES + 1];   // rows of type t: [row_start[t], row_start[t+1])
  int tile_start[DP_MAX_TYPES + 1];  // prefix of 128-row tiles per type
  int K, N, BN;                      // reduction length, output width, output columns per CTA
  const float* bias[DP_MAX_TYPES];   // [N] per type
  const float* w_last[DP_MAX_TYPES];  // FWD_LAST: final linear layer weights [N] per type
  float b_last[DP_MAX_TYPES];
  const float* skip_mat;  // fwd: layer input x fp32 [rows][skip_ld]; bwd: gy fp32 [rows][skip_ld]
  int skip_vec;           // bwd of the last hidden layer: gy is the row vector w_last of the type
  int skip_kind;          // 0 none, 1 +x, 2 +{x,x} (Eq. NN)
  int skip_ld;
  const float* tact;        // bwd: tanh outputs of the layer below [rows][N]
  float* out_f32;           // [rows][N]
  __nv_bfloat16* out_bf16;  // [rows][N]
  __nv_bfloat16* out_bf16_lo;  // split operands: [rows][N] low part x - bf16(x) of the BF16 output
  float* out_t;             // [rows][N]
  float* e_out;             // FWD_LAST: per-row energy partial of each column block [col blocks][e_ld]
  long e_ld;
  int* err;                 // device error word (bounded waits)
};

// Epilogue inputs staged by TMA: the skip input and the gate input of the backward pass
// (row-major FP32 [rows][ld], boxes of 32 columns x 128 rows, 128-byte swizzle).
struct TcEpiMaps {
  CUtensorMap skip, tact;
};

// Low halves of split BF16 operands (x = hi + lo, hi = bf16(x), lo = bf16(x - hi)): with them
// every product is formed as hi.hi + hi.lo + lo.hi in three tensor-core passes, which keeps
// about 16 significant bits of each operand (relative error near 2^-17 per product).
struct TcLo {
  CUtensorMap a;  // A low part, same geometry as `ta`
  TcMaps b;       // B low parts, same geometry as `tb`
};

// Tensor map of a row-major [rows][cols] BF16 matrix, 128-byte swizzle, box {64, box_rows}.
int make_tmap_bf16(CUtensorMap* map, const void* base, long rows, long cols, int box_rows);
// Tensor map of a row-major [rows][cols] matrix of elem_bytes (2: BF16, 4: FP32) elements,
// 128-byte swizzle, box {box_cols, box_rows} with box_cols * elem_bytes = 128.
int make_tmap_2d(CUtensorMap* map, const void* base, int elem_bytes, long rows, long cols, int box_cols,
                 int box_rows);
// Tensor map of a row-major [rows][cols] FP32 matrix, 128-byte swizzle, box {32, 128}.
int make_tmap_f32(CUtensorMap* map, const void* base, long rows, long cols);

// C[rows][N] (+epilogue) = A[rows][K] . B_t[K][N]; A from `ta` ([rows][K] row-major), B_t from
// the type's map in `tb` (its transpose, [N][K] row-major); BF16 operands, FP32 accumulation.
// With `lo` the operands are split (three passes) and every BF16 output of the epilogue is
// written as its high part (out_bf16) and low part (out_bf16_lo).
cudaError_t launch_tc_gemm(int epi, const CUtensorMap& ta, const TcMaps& tb, const TcArgs& a, cudaStream_t st,
                           const TcLo* lo = nullptr);

// Output columns per CTA for an N-wide output with `row_tiles` 128-row tiles in total (a
// multiple of 32).
int tc_pick_bn(int N, int row_tiles);

}  // namespace dpgb
