// Compressed embedding on the tensor cores: interval moments (Sec. II.A.6, Eq. (compress)).
//
// With the tabulated embedding, G_m(s) on interval l is a quintic in t = s - x_l.  Writing
// tau = t / Delta_l and C_{(l,p),m} = a_{l,m,p} Delta_l^p (a_{l,m,p}: coefficient of t^p), the
// contraction of the se_e2_a descriptor becomes, for centre atom i,
//
//   T_{m,c} = (1/Nc) sum_j G_m(s_j) R_{j,c} = (1/Nc) sum_{(t,l,p)} C^{(t)}_{(l,p),m} mu_{(t,l,p),c},
//   mu_{(t,l,p),c} = sum_{j of type t in interval l} tau_j^p R_{j,c},
//
// exactly (up to rounding): a dense contraction over K = (neighbour type, interval, power) with
// a coefficient matrix shared by every centre atom of one type.  One CTA takes 32 atoms of one
// centre type, i.e. 128 rows (atom, c); its four builder warps form the moments of one
// 8-interval block (64 K columns, one 128-byte swizzle row per (atom, c)) in shared memory
// while the matching coefficient block arrives by TMA, and one thread issues tcgen05.mma into
// a TMEM accumulator [128 rows][M].  The epilogue scales by 1/Nc, stores T and forms
// D = T T_<^T per atom.
//
// The backward needs, per neighbour, dE/dR_{j,c} = (1/Nc) sum_m gT_{m,c} G_m(s_j) and
// dE/ds_j = (1/Nc) sum_c R_{j,c} sum_m gT_{m,c} G'_m(s_j), with gT = dE/dT.  With
//   P_{(t,l,p),c} = sum_m C^{(t)}_{(l,p),m} gT_{m,c}      (tensor cores: [128 rows] x [M] x [K blocks])
// both are short polynomials per neighbour: dE/dR_c = (1/Nc) sum_p tau^p P_{p,c} and
// dE/ds = (1/Nc) sum_c R_c sum_p p tau^{p-1} P_{p,c} / Delta_l.
//
// Neighbours of each type block are sorted by distance, so their intervals are non-increasing
// along the list and every (atom, interval) is a contiguous run; the few FP32 rounding
// inversions are folded into the run of the previous neighbour (its polynomial piece evaluated
// a rounding error beyond its end, where the pieces join with C^2 continuity).  Work is split
// by its shape: everything per neighbour runs in lane-per-slot kernels at full occupancy
// (k_env_mom forms the slot records and, by a segmented warp reduction, each run's moments;
// k_force_mom turns each slot's run P into the pair force), while the tensor-core kernels only
// move per-run data (a run's moments into the A tile, a run's P out of TMEM).
//
// Precision: FP16 operands in one pass (mixed mode), or BF16 operands split into high and low
// parts with three passes (hi.hi + hi.lo + lo.hi; FP32 mode); FP32 accumulation.  The rows of
// gT are scaled by a power of two so FP16 holds them without overflow.  Every mbarrier wait is
// bounded; on time-out the CTA records an error and leaves.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <climits>

#include "env.cuh"
#include "fit_tc.cuh"
#include "mom.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace dpgb {

namespace {

using namespace ptx;

constexpr int kAtoms = 32;        // centre atoms per CTA
constexpr int kRows = 128;        // accumulator rows: (atom, c)
constexpr int kMomThreads = 192;  // 4 builder / epilogue warps, an MMA warp and a TMA producer warp
constexpr int kABlock = kRows * 128;  // one 64-column K block of 128 rows (bytes)
constexpr int kGroupAtoms = 4;        // backward: atoms per staged group of dE/dD rows
// backward: 64-column TMEM accumulators in rotation, and the coefficient ring depth.  The one-pass
// (mixed) kernel keeps two of each so that three CTAs fit an SM (3 x 128 TMEM columns); the
// three-pass kernel runs one CTA per SM and takes four accumulators and three stages, so the MMAs
// of the next chunks run while the epilogue drains one.
template <int NPASS>
struct BwdDepth {
  static constexpr int acc = NPASS == 1 ? 2 : 4;
  static constexpr int stages = NPASS == 1 ? 2 : 3;
};

struct MomArgs {
  int ntypes, nc, M, A, lc, lcp, n1;
  float s0, stride1, stride2, inv1, inv2, split, smax, inv_nc;
  int sel_off[DP_MAX_TYPES + 1];
  int row_start[DP_MAX_TYPES + 1];
  int tile_start[DP_MAX_TYPES + 1];
  const int* perm;
  const int* nl_j;
  // per-slot records, rows in sorted atom order [N * nc]: (s, u), (ds/dr, r, tau, l), run index
  float4* envU;
  float4* envB;
  int* slot_run;
  // per-run records, run r of type block t of atom p at row p * nc + sel_off[t] + r
  int* run_l;      // interval of the run; -1 after the last run
  uint4* run_rec;  // moments as A-operand chunks [row][4 components][parts]
  float4* run_P;   // P of the run [row][4 components][2] FP32, or [row][4 components] 8 x BF16 when
                   // p_bf16 (mixed mode); shares memory with run_rec
  int p_bf16;
  float* Tm;          // [N][M][4]
  void* D;            // [N][M * A], BF16 or FP32 (d_bf16 = 2: BF16 high part)
  void* D_lo;         // d_bf16 = 2: [N][M * A] BF16 low part D - bf16(D)
  int d_bf16;
  const float* gD;            // [N][M * A] FP32, or
  const __nv_bfloat16* gDh;   // [N][M * A] BF16 (mixed mode)
  double* force;    // [N][3] input order
  double* avir;     // [N][9] input order
  unsigned char* gta;  // backward A operand per tile: the shared-memory image of dE/dT rows
  int* gtx;            // its row scales [tiles][128]
  // or, FP32 mode with the split fitting kernel, dE/dT itself, m-major [M][N][4] FP32: the backward
  // kernel then forms its A operand image in its prologue (no k_mom_gT)
  const float* gTt;
  int* table_range;
  int* err;
  unsigned int* mma_blocks;  // [2] blocks issued by the forward / backward MMA threads (work count)
  // mixed mode with the list built in the same call: FP32 displacements from cell-local positions
  const float4* atom_l;
  const int4* atom_m;
  const NlGeom* geoms;
  // mixed mode with the cell-centred list build: each slot's FP32 displacement, read in place of
  // the gathers above ([N][nc] in sorted order; w: 1 FP32 usable, 0 exact needed, -1 padding)
  const float4* disp;
};

// Interval of s (at most lcap: the list order caps it), tau = (s - x_l) / Delta_l, 1/Delta_l.
__device__ __forceinline__ int mom_interval(const MomArgs& g, float s, int lcap, float& tau, float& inv_d,
                                            bool& oor) {
  int l;
  if (s < g.split) {
    l = (int)floorf((s - g.s0) * g.inv1);
    l = l < 0 ? 0 : (l > g.n1 - 1 ? g.n1 - 1 : l);
  } else {
    l = g.n1 + (int)floorf((s - g.split) * g.inv2);
    if (l > g.lc - 1) l = g.lc - 1;
    if (s > g.smax) oor = true;
  }
  if (l > lcap) l = lcap;
  if (l < g.n1) {
    inv_d = g.inv1;
    tau = (s - (g.s0 + (float)l * g.stride1)) * g.inv1;
  } else {
    inv_d = g.inv2;
    tau = (s - (g.split + (float)(l - g.n1) * g.stride2)) * g.inv2;
  }
  return l;
}

// Block kb of the tile's schedule: neighbour types in order, 8-interval groups descending.
__device__ __forceinline__ void block_of(int kb, const int* ghi, int ntypes, int& t, int& grp) {
  t = 0;
  while (t < ntypes) {
    const int n = ghi[t] + 1;
    if (kb < n) break;
    kb -= n;
    ++t;
  }
  grp = ghi[t] - kb;
}

// tau of s on interval l (the list order lowered l below the interval of s by a rounding error).
__device__ __forceinline__ float tau_at(const MomArgs& g, float s, int l) {
  return l < g.n1 ? (s - (g.s0 + (float)l * g.stride1)) * g.inv1
                  : (s - (g.split + (float)(l - g.n1) * g.stride2)) * g.inv2;
}

__device__ __forceinline__ uint32_t pack_h2(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ uint32_t pack_b2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}
// 8 values as one 16-byte chunk: FP16 (one part) or BF16 high and low parts.
template <int NPASS>
__device__ __forceinline__ void store_chunk(unsigned char* hi, unsigned char* lo, const float* v) {
  if (NPASS == 1) {
    *reinterpret_cast<uint4*>(hi) = make_uint4(pack_h2(v[0], v[1]), pack_h2(v[2], v[3]), pack_h2(v[4], v[5]),
                                               pack_h2(v[6], v[7]));
  } else {
    float h[8], r[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      h[q] = __bfloat162float(__float2bfloat16_rn(v[q]));
      r[q] = v[q] - h[q];
    }
    *reinterpret_cast<uint4*>(hi) = make_uint4(pack_b2(h[0], h[1]), pack_b2(h[2], h[3]), pack_b2(h[4], h[5]),
                                               pack_b2(h[6], h[7]));
    *reinterpret_cast<uint4*>(lo) = make_uint4(pack_b2(r[0], r[1]), pack_b2(r[2], r[3]), pack_b2(r[4], r[5]),
                                               pack_b2(r[6], r[7]));
  }
}

// Byte offset of 16-byte chunk q of row r in a 128-byte-swizzled K-major block.
__device__ __forceinline__ uint32_t sw_off(int r, int q) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((q ^ (r & 7)) << 4));
}

// The run intervals of the tile's 32 atoms, every type block ([atom][nc], -1 past a tile's end),
// as 16-bit values (intervals are far below 2^15).  The tile's rows are one contiguous stretch of
// run_l: 16-byte loads where it is aligned, and each thread's loads all in flight before the first
// store.
__device__ __forceinline__ void stage_runs(const MomArgs& g, int row0, int row_end, short* runl_s, int tid,
                                           int nthreads) {
  const int n = kAtoms * g.nc;
  const int nv = min(kAtoms, row_end - row0) * g.nc;  // slots of the tile's real atoms
  const int* src = g.run_l + (long)row0 * g.nc;
  int done = 0;
  if ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
    const int n4 = nv >> 2;
    const int4* s4 = reinterpret_cast<const int4*>(src);
    short4* d4 = reinterpret_cast<short4*>(runl_s);
    for (int e0 = tid; e0 < n4; e0 += 8 * nthreads) {
      int4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * nthreads;
        if (e < n4) v[u] = __ldg(s4 + e);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = e0 + u * nthreads;
        if (e < n4) d4[e] = make_short4((short)v[u].x, (short)v[u].y, (short)v[u].z, (short)v[u].w);
      }
    }
    done = 4 * n4;
  }
  for (int e0 = done + tid; e0 < n; e0 += 16 * nthreads) {
    int v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = e0 + u * nthreads;
      v[u] = e < nv ? __ldg(src + e) : -1;
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = e0 + u * nthreads;
      if (e < n) runl_s[e] = (short)v[u];
    }
  }
}

// Ring depth of the forward's operand stages: two keep three CTAs (mixed mode) on an SM, one wave of
// tiles; the three-pass kernel (one CTA per SM, 60 KB stages) takes three, two blocks of run-record
// copies in flight per builder thread.
template <int NPASS>
struct MomStages {
  static constexpr int value = NPASS == 1 ? 2 : 3;
};


// Largest 8-interval group holding a neighbour of each type, over the tile's atoms (the first
// run of each list has the largest interval; runl_s holds the tile's run lists).
__device__ __forceinline__ void tile_groups(const MomArgs& g, const short* runl_s, int a, int* ghi) {
  for (int t = 0; t < g.ntypes; ++t) {
    const int l = runl_s[a * g.nc + g.sel_off[t]];
    if (l >= 0) atomicMax(&ghi[t], l >> 3);
  }
}

// =============================================================================================
// Per-slot records and per-run moments.  One warp takes one (atom, neighbour type) list, 32
// slots at a time: exact FP64 displacement, FP32 switch (Eq. (switch)), interval and tau; the
// interval is lowered to the running minimum along the list (a prefix-minimum scan) so that it
// never increases from slot to slot, even where FP32 rounding of s inverts two nearly equal
// distances.  Equal intervals then form contiguous runs, and a segmented reduction across the
// lanes sums each run's moments mu_{p,c} = sum tau^p R_c (runs that cross a 32-slot batch are
// carried to the next).  Each run's moments are written in the backward's A-operand chunk
// format (FP16, or BF16 high and low parts): the forward kernel copies them into its tiles
// without conversion.  Outputs, for slot k of atom p (row p * Nc + k):
//   envU (s, u), envB (ds/dr, r, tau, l) with l = -1 marking padding, slot_run (run index);
// and for run r of type block t (row p * Nc + sel_off[t] + r): run_l (-1 after the last run)
// and run_rec.
// =============================================================================================
template <int NPASS>
__global__ void __launch_bounds__(256, 3)
    k_env_mom(PathConst pc, MomArgs g, const double* __restrict__ coord, const int* __restrict__ nl_code) {
  constexpr int PARTS = NPASS == 1 ? 1 : 2;
  __shared__ float s_carry[8][24];  // moments of the run left open at a batch's end, per warp
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* carry = s_carry[warp];
  const long ntask = (long)pc.natoms * pc.ntypes;
  const long wstride = (long)gridDim.x * 8;
  // With the list build's displacements every slot is one coalesced load and no gather: the first
  // batch of the warp's next task is loaded while the current task runs, and each next batch of
  // a task while the current batch runs.
  auto disp_batch = [&](long tk, int base) -> float4 {
    float4 d = make_float4(0.f, 0.f, 0.f, -1.f);
    if (g.disp && tk < ntask) {
      const int pp = (int)(tk / pc.ntypes), tt = (int)(tk % pc.ntypes);
      if (base + lane < g.sel_off[tt + 1]) d = g.disp[(long)pp * pc.nc + base + lane];
    }
    return d;
  };
  const float frs = (float)pc.rs, frc = (float)pc.rc, inv_w = 1.0f / (frc - frs);
  long task = (long)blockIdx.x * 8 + warp;
  float4 dnext = disp_batch(task, task < ntask ? g.sel_off[task % pc.ntypes] : 0);
  for (; task < ntask; task += wstride) {  // warp-uniform
  const int p = (int)(task / pc.ntypes), t = (int)(task % pc.ntypes);
  const int kb0 = g.sel_off[t], kb1 = g.sel_off[t + 1];
  float4 dcur = dnext;
  dnext = disp_batch(task + wstride, task + wstride < ntask ? g.sel_off[(task + wstride) % pc.ntypes] : 0);
  const int i = g.disp ? -1 : g.perm[p];  // with displacements: read only for an exact pair
  const long rbase = (long)p * pc.nc + kb0;  // first run record of this list
  // Mixed mode: the displacement in FP32 as (l_j + delta . h_c) - l_i from the cell-local
  // positions of the list build (delta: the virtual-cell offset of the image of j), with the
  // list build's error bound; pairs within that bound of r_c take the exact FP64 displacement.
  // The cell-centred list build hands this same value over per slot (disp); the per-atom one
  // does not, and then it is formed here from the gathered positions, rounded the same way.
  const bool f32d = NPASS == 1 && g.atom_l != nullptr && g.disp == nullptr;
  float4 li = make_float4(0.f, 0.f, 0.f, 0.f);
  int4 mi = make_int4(0, 0, 0, 0);
  const NlGeom* G = nullptr;
  if (f32d) {
    li = g.atom_l[i];
    mi = g.atom_m[i];
    G = g.geoms + frame_of(pc, i);
  }
  int lmin = INT_MAX;                        // running minimum of the interval
  int carry_l = -1;                          // interval of the run open at the last batch's end
  int nruns = 0;
  bool oor = false;
  for (int base = kb0; base < kb1; base += 32) {
    const int k = base + lane;
    const bool in = k < kb1;
    const long row = (long)p * pc.nc + k;
    const float4 dd = dcur;
    if (g.disp && base + 32 < kb1) dcur = disp_batch(task, base + 32);
    int j = -1;
    if (!g.disp && in) j = g.nl_j[(long)i * pc.nc + k];
    const bool valid = g.disp ? dd.w >= 0.f : j >= 0;
    int l = INT_MAX;
    float r = 0.f, s = 0.f, ds = 0.f, u[3] = {0.f, 0.f, 0.f}, tau = 0.f;
    if (valid) {
      // the FP32 displacement: handed over by the list build, or formed from the gathered
      // cell-local positions, or (near r_c) rounded from the exact FP64 one; one call of the
      // switch below for all three, so that its rounding does not depend on the source
      float x0 = 0.f, x1 = 0.f, x2 = 0.f;
      bool have = false;
      if (g.disp) {
        if (dd.w > 0.5f) {  // FP32 r^2 certainly inside r_c
          x0 = dd.x;
          x1 = dd.y;
          x2 = dd.z;
          have = true;
        }
      } else if (f32d) {
        const int code = nl_code[(long)i * pc.nc + k];
        const float4 lj = g.atom_l[j];
        const int4 mj = g.atom_m[j];
        int n0, n1, n2;
        unpack_shift(code, n0, n1, n2);
        const int e0 = ((mj.w >> 20) & 1023) - ((mi.w >> 20) & 1023) + (n0 + mj.x - mi.x) * G->ncell[0];
        const int e1 = ((mj.w >> 10) & 1023) - ((mi.w >> 10) & 1023) + (n1 + mj.y - mi.y) * G->ncell[1];
        const int e2 = (mj.w & 1023) - (mi.w & 1023) + (n2 + mj.z - mi.z) * G->ncell[2];
        if (abs(e0) <= G->K[0] && abs(e1) <= G->K[1] && abs(e2) <= G->K[2]) {
          // (l_j + o) - l_i with o the FP32 offset of j's cell, rounded as the list build rounds it
          const float f0 = (float)e0, f1 = (float)e1, f2 = (float)e2;
          x0 = (lj.x + fmaf(f2, G->hc[6], fmaf(f1, G->hc[3], f0 * G->hc[0]))) - li.x;
          x1 = (lj.y + fmaf(f2, G->hc[7], fmaf(f1, G->hc[4], f0 * G->hc[1]))) - li.y;
          x2 = (lj.z + fmaf(f2, G->hc[8], fmaf(f1, G->hc[5], f0 * G->hc[2]))) - li.z;
          have = fmaf(x0, x0, fmaf(x1, x1, x2 * x2)) < G->rc2_in;
        }
      }
      if (!have) {
        const int ie = g.disp ? g.perm[p] : i;
        if (g.disp) j = g.nl_j[(long)ie * pc.nc + k];
        const int code = nl_code[(long)ie * pc.nc + k];
        double d0, d1, d2;
        listed_disp(coord + 3 * ie, coord + 3 * j, code, pc, frame_of(pc, ie), d0, d1, d2);
        x0 = (float)d0;
        x1 = (float)d1;
        x2 = (float)d2;
      }
      // a few ulps of FP32: the moments go on as FP16 or split-BF16 operands (2^-11, 2^-17)
      pair_env_f32_fast(x0, x1, x2, frs, frc, inv_w, r, s, ds, u);
      float invd;
      l = mom_interval(g, s, INT_MAX, tau, invd, oor);
    }
    {
      // the interval never increases along the list: a prefix minimum over the batch (and the
      // batches before), needed only where FP32 rounding inverted two nearly equal distances
      const int lp = __shfl_up_sync(0xffffffffu, l, 1);
      const bool inverted = valid && l > (lane == 0 ? lmin : lp);  // valid slots are a prefix
      if (__any_sync(0xffffffffu, inverted)) {
        int m = l;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const int o = __shfl_up_sync(0xffffffffu, m, off);
          if (lane >= off) m = min(m, o);
        }
        m = min(m, lmin);
        if (valid && m < l) {
          l = m;
          tau = tau_at(g, s, l);
        }
        lmin = __shfl_sync(0xffffffffu, m, 31);
      } else {
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        if (vm) lmin = __shfl_sync(0xffffffffu, l, 31 - __clz(vm));
      }
    }
    if (in) {
      if (valid) {
        g.envU[row] = make_float4(s, u[0], u[1], u[2]);
        g.envB[row] = make_float4(ds, r, tau, __int_as_float(l));
      } else {
        g.envB[row] = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
      }
    }
    // moments of this slot
    const int lk = valid ? l : -2;
    float v[24];
    {
      const float R[4] = {s, s * u[0], s * u[1], s * u[2]};
      float pw = 1.f;
#pragma unroll
      for (int pp = 0; pp < 6; ++pp) {
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c * 6 + pp] = valid ? pw * R[c] : 0.f;
        pw *= tau;
      }
    }
    // run structure of the batch: a head starts a new run (the first lane may continue the run
    // left open by the previous batch)
    const int lprev_lane = __shfl_up_sync(0xffffffffu, lk, 1);
    const int lprev = lane == 0 ? carry_l : lprev_lane;
    const bool head = valid && lk != lprev;
    const bool seg = valid && (lane == 0 || lk != lprev_lane);  // first lane of its run in this batch
    const unsigned headmask = __ballot_sync(0xffffffffu, head);
    const unsigned segmask = __ballot_sync(0xffffffffu, seg);
    const unsigned validmask = __ballot_sync(0xffffffffu, valid);
    // segmented sums towards the first lane of each run; after the step of distance off every lane
    // holds the sum over its run up to 2 off - 1 lanes ahead, so once no run reaches off lanes
    // ahead the heads hold their runs' sums (runs are short: one to a few slots)
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int lo = __shfl_down_sync(0xffffffffu, lk, off);
      const bool same = valid && lane + off < 32 && lo == lk;
      if (!__any_sync(0xffffffffu, same)) break;
#pragma unroll
      for (int e = 0; e < 24; ++e) {
        const float o = __shfl_down_sync(0xffffffffu, v[e], off);
        if (same) v[e] += o;
      }
    }
    const bool cont0 = __shfl_sync(0xffffffffu, valid && lk == carry_l, 0);  // lane 0 continues the open run
    if (lane == 0 && cont0)
#pragma unroll
      for (int e = 0; e < 24; ++e) v[e] += carry[e];
    if (carry_l >= 0 && !cont0 && lane == 0) {  // the open run ended exactly at the batch boundary
      const long rec = rbase + nruns - 1;
      g.run_l[rec] = carry_l;
      uint4* dst = g.run_rec + rec * 4 * PARTS;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float w8[8] = {carry[c * 6], carry[c * 6 + 1], carry[c * 6 + 2], carry[c * 6 + 3], carry[c * 6 + 4],
                             carry[c * 6 + 5], 0.f, 0.f};
        store_chunk<NPASS>(reinterpret_cast<unsigned char*>(dst + c * PARTS),
                           reinterpret_cast<unsigned char*>(dst + c * PARTS + 1), w8);
      }
    }
    // run index of every slot: runs so far + heads up to this lane - 1
    const int myrun = nruns + __popc(headmask & (0xffffffffu >> (31 - lane))) - 1;
    if (valid) g.slot_run[row] = myrun;
    // every run of the batch is complete except the one holding the last valid lane, unless
    // the list ends in this batch
    const int lastvalid = validmask ? 31 - __clz(validmask) : -1;
    const bool ends = lastvalid < 31 || base + 32 >= kb1;
    const int open = (!ends && lastvalid >= 0) ? 31 - __clz(segmask & (0xffffffffu >> (31 - lastvalid))) : -1;
    if (seg && lane != open) {
      const long rec = rbase + myrun;
      g.run_l[rec] = lk;
      uint4* dst = g.run_rec + rec * 4 * PARTS;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float w8[8] = {v[c * 6], v[c * 6 + 1], v[c * 6 + 2], v[c * 6 + 3], v[c * 6 + 4], v[c * 6 + 5], 0.f, 0.f};
        store_chunk<NPASS>(reinterpret_cast<unsigned char*>(dst + c * PARTS),
                           reinterpret_cast<unsigned char*>(dst + c * PARTS + 1), w8);
      }
    }
    __syncwarp();  // lane 0 has read the previous carry
    if (open >= 0) {
      carry_l = __shfl_sync(0xffffffffu, lk, open);
      if (lane == open)
#pragma unroll
        for (int e = 0; e < 24; ++e) carry[e] = v[e];
    } else {
      carry_l = -1;
    }
    __syncwarp();
    nruns += __popc(headmask);
    if (ends) break;  // warp-uniform: the rest of the block is padding
  }
  if (lane == 0 && nruns < kb1 - kb0) g.run_l[rbase + nruns] = -1;
  if (__any_sync(0xffffffffu, oor) && lane == 0) atomicOr(g.table_range, 1);
  }
}

// =============================================================================================
// Forward: T and D.  Thread r < 128 owns A row r = (atom r / 4, component r % 4): for every
// 8-interval block it copies the chunks of its atom's runs in the block from the run records
// (cp.async, already in operand format) and clears the chunks of empty intervals; the copies of
// block kb are released to the MMA once they have landed, up to S - 1 blocks later.
// =============================================================================================
template <int NPASS, int NPAD>
__global__ void __launch_bounds__(kMomThreads, NPASS == 1 ? 3 : 1)
    k_mom_fwd(const __grid_constant__ CUtensorMap bhi, const __grid_constant__ CUtensorMap blo, const MomArgs g) {
  constexpr int PARTS = NPASS == 1 ? 1 : 2;
  constexpr int S = MomStages<NPASS>::value;
  constexpr int D = S - 1;  // blocks in flight per builder thread
  constexpr int B_BYTES = NPAD * 128;
  constexpr int STAGE = PARTS * (kABlock + B_BYTES);
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  short* runl_s = reinterpret_cast<short*>(smem + S * STAGE);  // [32 atoms][nc] run intervals of the tile
  uint64_t* full = reinterpret_cast<uint64_t*>(runl_s + kAtoms * g.nc);
  uint64_t* empty = full + S;
  uint64_t* accf = empty + S;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(accf + 1);
  int* ghi = reinterpret_cast<int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int ti = 0;
  while (ti + 1 < g.ntypes && (int)blockIdx.x >= g.tile_start[ti + 1]) ++ti;
  const int row0 = g.row_start[ti] + ((int)blockIdx.x - g.tile_start[ti]) * kAtoms;
  const int row_end = g.row_start[ti + 1];

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], kRows + 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accf, 1);
    for (int t = 0; t < DP_MAX_TYPES; ++t) ghi[t] = -1;
    mbar_fence_init();
  }
  if (warp == 4) tmem_alloc(tmem_holder, 128);
  const int r = threadIdx.x;
  const int ae = r >> 2, c = r & 3;
  const int pe = row0 + ae;
  stage_runs(g, row0, row_end, runl_s, threadIdx.x, kMomThreads);
  __syncthreads();
  if (warp == 0) tile_groups(g, runl_s, lane, ghi);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  int nkb = 0;
  for (int t = 0; t < g.ntypes; ++t) nkb += ghi[t] + 1;

  if (warp == 5) {
    if (lane == 0) {
      // ---- TMA producer: a stage's coefficient block as soon as the stage is free ----
      int issued = 0;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % S;
        if (kb >= S && !mbar_wait(&empty[s], ((kb / S) - 1) & 1, g.err)) break;
        int t, grp;
        block_of(kb, ghi, g.ntypes, t, grp);
        unsigned char* bs = smem + s * STAGE + PARTS * kABlock;
        mbar_expect_tx(&full[s], PARTS * B_BYTES);
        const int x = (t * g.lcp + 8 * grp) * 8;
        tma_load_2d(bs, &bhi, &full[s], x, ti * NPAD);
        if (PARTS == 2) tma_load_2d(bs + B_BYTES, &blo, &full[s], x, ti * NPAD);
        issued = kb + 1;
      }
      // only the last S loads can still be in flight (each earlier stage was consumed before its
      // reuse): they must land before the CTA leaves
      for (int kb = max(0, issued - S); kb < issued; ++kb) mbar_wait(&full[kb % S], (kb / S) & 1, g.err);
    }
  } else if (warp == 4) {
    if (lane == 0) {
      // ---- MMA issuer ----
      const uint32_t idesc = idesc_f16(kRows, NPAD, NPASS == 1 ? 0 : 1);
      bool ok = true;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % S;
        if (!mbar_wait(&full[s], (kb / S) & 1, g.err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t sa = su32(smem + s * STAGE);
        const uint64_t ah = sdesc_sw128(sa), al = sdesc_sw128(sa + kABlock);
        const uint64_t bh = sdesc_sw128(sa + PARTS * kABlock), bl = sdesc_sw128(sa + PARTS * kABlock + B_BYTES);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          mma_f16(tmem, ah + 2 * k, bh + 2 * k, idesc, (kb | k) != 0);
          if (NPASS == 3) {
            mma_f16(tmem, ah + 2 * k, bl + 2 * k, idesc, 1);
            mma_f16(tmem, al + 2 * k, bh + 2 * k, idesc, 1);
          }
        }
        mma_commit(&empty[s]);
      }
      if (ok && nkb > 0)
        mma_commit(accf);
      else
        mbar_arrive(accf);
      if (ok && nkb > 0) atomicAdd(&g.mma_blocks[0], (unsigned)nkb);
    }
  } else {
    // ---- operand builders ----
    int cur_t = -1, ptr = 0, selt = 0;
    long rbase = 0;
    bool dead = false;  // after a timed-out wait: stop waiting, keep going through the blocks
    const uint32_t rowoff0 = (uint32_t)((r >> 3) * 1024 + (r & 7) * 128);
    for (int kb = 0; kb < nkb; ++kb) {
      int t, grp;
      block_of(kb, ghi, g.ntypes, t, grp);
      const int s = kb % S;
      if (kb >= D) {  // block kb - D: its copies have landed (the D - 1 later groups may still be in flight)
        cp_async_wait<D - 1>();
        fence_async_smem();
        mbar_arrive(&full[(kb - D) % S]);
      }
      if (kb >= S && !dead && !mbar_wait(&empty[s], ((kb / S) - 1) & 1, g.err)) dead = true;
      if (t != cur_t) {
        cur_t = t;
        selt = g.sel_off[t + 1] - g.sel_off[t];
        ptr = 0;
        rbase = (long)pe * g.nc + g.sel_off[t];
      }
      const short* myruns = runl_s + ae * g.nc + g.sel_off[t];
      unsigned char* ahi = smem + s * STAGE;
      unsigned char* alo = ahi + kABlock;
      unsigned covered = 0;
      while (ptr < selt) {
        const int l = myruns[ptr];
        if (l < 8 * grp) break;  // also the end marker -1
        const int q = (l - 8 * grp) & 7;
        const uint32_t off = rowoff0 + (uint32_t)((q ^ (r & 7)) << 4);
        const uint4* src = g.run_rec + ((rbase + ptr) * 4 + c) * PARTS;
        cp_async16(ahi + off, src);
        if (PARTS == 2) cp_async16(alo + off, src + 1);
        covered |= 1u << q;
        ++ptr;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (!((covered >> q) & 1u)) {
          const uint32_t off = rowoff0 + (uint32_t)((q ^ (r & 7)) << 4);
          *reinterpret_cast<uint4*>(ahi + off) = make_uint4(0u, 0u, 0u, 0u);
          if (PARTS == 2) *reinterpret_cast<uint4*>(alo + off) = make_uint4(0u, 0u, 0u, 0u);
        }
      cp_async_commit();
    }
    cp_async_wait0();
    fence_async_smem();
    for (int kb = max(0, nkb - D); kb < nkb; ++kb) mbar_arrive(&full[kb % S]);
  }

  // ---- epilogue: T = acc / Nc, then D = T T_<^T (all six warps once T is staged) ----
  float* smT = reinterpret_cast<float*>(smem);  // [32 atoms][NPAD + 1][4]; the ring is idle now
  if (warp < 4) {
    mbar_wait(accf, 0, g.err);
    __syncwarp();  // tcgen05.ld is warp-collective
    tc_fence_after();
    const uint32_t tb = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < NPAD; c0 += 32) {  // two 16-column loads in flight, one wait
      uint32_t raw[32];
      const bool two = c0 + 16 < NPAD;  // warp-uniform
      tmem_ld16_async(tb + c0, raw);
      if (two) tmem_ld16_async(tb + c0 + 16, raw + 16);
      tmem_wait_ld();
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        if (q >= 16 && !two) break;
        const float x = nkb > 0 ? __uint_as_float(raw[q]) * g.inv_nc : 0.f;
        smT[(ae * (NPAD + 1) + c0 + q) * 4 + c] = x;
      }
    }
    tc_fence_before();
  } else {
    __syncwarp();  // the MMA issuer and the TMA producer are done with their loops: converge
  }
  bar_sync(1, kMomThreads);  // T staged; the MMA and TMA warps join the rest
  const int na = min(kAtoms, row_end - row0);
  {  // T of the tile's atoms (consecutive rows: one contiguous block of Tm), coalesced
    const float4* src = reinterpret_cast<const float4*>(smT);
    float4* dst = reinterpret_cast<float4*>(g.Tm) + (long)row0 * g.M;
    for (int e = r; e < na * g.M; e += kMomThreads) {
      const int a = e / g.M, m = e - a * g.M;
      dst[e] = src[a * (NPAD + 1) + m];
    }
  }
  {  // D: six threads per atom, thread (atom, q) takes m = q, q + 6, ...
    constexpr int kPer = kMomThreads / kAtoms;
    const int ad = r / kPer, q = r - ad * kPer;
    if (ad < na) {
      const long pd = row0 + ad;
      const float4* T4 = reinterpret_cast<const float4*>(smT) + ad * (NPAD + 1);
      float4 tl[16];
#pragma unroll
      for (int l = 0; l < 16; ++l) tl[l] = l < g.A ? T4[l] : make_float4(0.f, 0.f, 0.f, 0.f);
      for (int m = q; m < g.M; m += kPer) {
        const float4 tm = T4[m];
        float d[16];
#pragma unroll
        for (int l = 0; l < 16; ++l) d[l] = tm.x * tl[l].x + tm.y * tl[l].y + tm.z * tl[l].z + tm.w * tl[l].w;
        const long o = (pd * g.M + m) * g.A;
        if (g.d_bf16 == 2) {  // split operands of the FP32 mode's tensor-core fitting net
          __nv_bfloat16* Dh = reinterpret_cast<__nv_bfloat16*>(g.D) + o;
          __nv_bfloat16* Dl = reinterpret_cast<__nv_bfloat16*>(g.D_lo) + o;
          float dl[16];
#pragma unroll
          for (int l = 0; l < 16; ++l) dl[l] = d[l] - __bfloat162float(__float2bfloat16_rn(d[l]));
          if (g.A == 16) {  // the hi parts are d rounded to BF16, the lo parts the remainders rounded
            uint4* h4 = reinterpret_cast<uint4*>(Dh);
            uint4* l4 = reinterpret_cast<uint4*>(Dl);
            h4[0] = make_uint4(pack_b2(d[0], d[1]), pack_b2(d[2], d[3]), pack_b2(d[4], d[5]), pack_b2(d[6], d[7]));
            h4[1] = make_uint4(pack_b2(d[8], d[9]), pack_b2(d[10], d[11]), pack_b2(d[12], d[13]),
                               pack_b2(d[14], d[15]));
            l4[0] = make_uint4(pack_b2(dl[0], dl[1]), pack_b2(dl[2], dl[3]), pack_b2(dl[4], dl[5]),
                               pack_b2(dl[6], dl[7]));
            l4[1] = make_uint4(pack_b2(dl[8], dl[9]), pack_b2(dl[10], dl[11]), pack_b2(dl[12], dl[13]),
                               pack_b2(dl[14], dl[15]));
          } else {
#pragma unroll
            for (int l = 0; l < 16; ++l)
              if (l < g.A) {
                Dh[l] = __float2bfloat16_rn(d[l]);
                Dl[l] = __float2bfloat16_rn(dl[l]);
              }
          }
        } else if (g.d_bf16) {
          __nv_bfloat16* Db = reinterpret_cast<__nv_bfloat16*>(g.D) + o;
          if (g.A == 16) {
            uint4* d4 = reinterpret_cast<uint4*>(Db);
            d4[0] = make_uint4(pack_b2(d[0], d[1]), pack_b2(d[2], d[3]), pack_b2(d[4], d[5]), pack_b2(d[6], d[7]));
            d4[1] = make_uint4(pack_b2(d[8], d[9]), pack_b2(d[10], d[11]), pack_b2(d[12], d[13]),
                               pack_b2(d[14], d[15]));
          } else {
#pragma unroll
            for (int l = 0; l < 16; ++l)
              if (l < g.A) Db[l] = __float2bfloat16_rn(d[l]);
          }
        } else {
          float* Df = reinterpret_cast<float*>(g.D) + o;
          if (g.A == 16) {
            float4* d4 = reinterpret_cast<float4*>(Df);
#pragma unroll
            for (int k4 = 0; k4 < 4; ++k4)
              d4[k4] = make_float4(d[4 * k4], d[4 * k4 + 1], d[4 * k4 + 2], d[4 * k4 + 3]);
          } else {
#pragma unroll
            for (int l = 0; l < 16; ++l)
              if (l < g.A) Df[l] = d[l];
          }
        }
      }
    }
  }
  __syncthreads();
  if (warp == 4) tmem_dealloc(tmem, 128);
}

// =============================================================================================
// dE/dT rows of every tile as the backward's A operand (the shared-memory image, 128-byte
// swizzle, FP16 or BF16 high/low parts, each row scaled by a power of two):
//   gT_m = sum_l gD[m][l] T[l][c] + [m < A] sum_q gD[q][m] T[q][c]
// One CTA per group of four atoms of a tile (blockIdx.y); many CTAs per SM hide the latency of
// the dE/dD rows.
// =============================================================================================
template <int NPASS, int NPAD>
__global__ void __launch_bounds__(kRows)
    k_mom_gT(const MomArgs g) {
  constexpr int A_BYTES = 2 * kABlock;
  constexpr int PARTS = NPASS == 1 ? 1 : 2;
  constexpr int NGRP = kAtoms / kGroupAtoms;
  constexpr int SCRP = NPAD + 4;  // FP32 scratch row pitch
  __shared__ __align__(16) float scr[16 * SCRP];
  static_assert(NGRP == 8, "eight groups of four atoms per tile");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, c = lane & 3;
  int ti = 0;
  while (ti + 1 < g.ntypes && (int)blockIdx.x >= g.tile_start[ti + 1]) ++ti;
  const int row0 = g.row_start[ti] + ((int)blockIdx.x - g.tile_start[ti]) * kAtoms;
  const int row_end = g.row_start[ti + 1];
    // warp w takes atom w of each group of four, lane = (part, c)
    //   gT_m = sum_l gD[m][l] T[l][c] + [m < A] sum_q gD[q][m] T[q][c],  m = part + 8k
    {
      const int part = lane >> 2;
      float* srow = scr + (warp * 4 + c) * SCRP;
      unsigned char* At = g.gta + (long)blockIdx.x * PARTS * A_BYTES;
      {
        const int q = blockIdx.y;
        const int at = q * kGroupAtoms + warp;  // atom of the tile
        const bool va = row0 + at < row_end;   // warp-uniform
        const long gdo = (long)(row0 + at) * g.M * g.A;
        // BF16 dE/dD is tile-blocked: 128-row tiles from the type's first row, 8-column groups
        const int KD = g.M * g.A;
        const int fr0 = g.row_start[ti] + (((row0 + at) - g.row_start[ti]) & ~127);
        const int fnr = min(128, g.row_start[ti + 1] - fr0);
        const __nv_bfloat16* gtile = g.gDh ? g.gDh + (long)fr0 * KD : nullptr;
        const int fr = row0 + at - fr0;
        const float* Ta = g.Tm + (long)(row0 + at) * g.M * 4;
        int ex = 0;
        if (va) {
          float tl[16], ext[16];
#pragma unroll
          for (int l = 0; l < 16; ++l) {
            tl[l] = l < g.A ? Ta[l * 4 + c] : 0.f;
            ext[l] = 0.f;
          }
#pragma unroll 2
          for (int k = 0; k < NPAD / 8; ++k) {
            const int m = part + 8 * k;
            if (m < g.M) {
              float gd[16];
              if (g.gDh && g.A == 16) {
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                  const uint4 x = *reinterpret_cast<const uint4*>(gtile + ((long)(2 * m + e) * fnr + fr) * 8);
                  const uint32_t w4[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                  for (int k = 0; k < 4; ++k) {
                    gd[8 * e + 2 * k] = __uint_as_float(w4[k] << 16);
                    gd[8 * e + 2 * k + 1] = __uint_as_float(w4[k] & 0xFFFF0000u);
                  }
                }
              } else if (g.gDh) {
#pragma unroll
                for (int l = 0; l < 16; ++l) {
                  const int col = m * g.A + l;
                  gd[l] = l < g.A ? __bfloat162float(gtile[((long)(col >> 3) * fnr + fr) * 8 + (col & 7)]) : 0.f;
                }
              } else if (g.A == 16) {
                const float4* g4 = reinterpret_cast<const float4*>(g.gD + gdo + m * 16);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                  const float4 x = g4[e];
                  gd[4 * e] = x.x;
                  gd[4 * e + 1] = x.y;
                  gd[4 * e + 2] = x.z;
                  gd[4 * e + 3] = x.w;
                }
              } else {
#pragma unroll
                for (int l = 0; l < 16; ++l) gd[l] = l < g.A ? g.gD[gdo + m * g.A + l] : 0.f;
              }
              const float tm = Ta[m * 4 + c];
              float v = 0.f;
#pragma unroll
              for (int l = 0; l < 16; ++l) {
                v += gd[l] * tl[l];
                ext[l] += gd[l] * tm;
              }
              srow[m] = v;
            }
          }
#pragma unroll
          for (int l = 0; l < 16; ++l) {
            ext[l] += __shfl_xor_sync(0xffffffffu, ext[l], 4);
            ext[l] += __shfl_xor_sync(0xffffffffu, ext[l], 8);
            ext[l] += __shfl_xor_sync(0xffffffffu, ext[l], 16);
          }
          __syncwarp();
#pragma unroll
          for (int l = 0; l < 16; ++l)
            if (l < g.A && (l & 7) == part) srow[l] += ext[l];
          __syncwarp();
          float mx = 0.f;
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int m = 8 * (part + 8 * h) + e;
              if (m < g.M) mx = fmaxf(mx, fabsf(srow[m]));
            }
          mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 4));
          mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 8));
          mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
          if (mx > 0.f) frexpf(mx, &ex);
        }
        // this lane's two 8-column chunks of A row (atom, c), scaled by 2^-ex (zero without an atom)
        const int rr = at * 4 + c;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int qq = part + 8 * h;
          float v[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int m = 8 * qq + e;
            v[e] = (va && m < g.M) ? ldexpf(srow[m], -ex) : 0.f;
          }
          const uint32_t off = (uint32_t)((qq >> 3) * kABlock) + sw_off(rr, qq & 7);
          store_chunk<NPASS>(At + off, At + A_BYTES + off, v);
        }
        if (part == 0) g.gtx[(long)blockIdx.x * kRows + rr] = ex;
        __syncwarp();  // the scratch row is read before the next atom overwrites it
      }
    }
}

// =============================================================================================
// Backward, tensor-core part: P = C . dE/dT per 8-interval block (TMEM), written out per run.
// Thread r < 128 reads accumulator row r = (atom r / 4, component r % 4) and stores, for each
// run of its atom in the block, the six values of its interval (scaled back by 2^ex / Nc) to the
// run's P record; the per-slot part of the backward is k_force_mom.
// =============================================================================================
template <int NPASS, int NPAD>
__global__ void __launch_bounds__(kMomThreads, 1)
    k_mom_bwd(const __grid_constant__ CUtensorMap bhi, const __grid_constant__ CUtensorMap blo, const MomArgs g) {
  constexpr int PARTS = NPASS == 1 ? 1 : 2;
  constexpr int S = BwdDepth<NPASS>::stages;
  constexpr int kAccBufs = BwdDepth<NPASS>::acc;
  constexpr int A_BYTES = 2 * kABlock;  // K = m in two 64-column blocks
  constexpr int B_KBLK = 64 * 128;      // 64 rows (8 intervals x 8 powers) x 128 B
  constexpr int B_STAGE = PARTS * 2 * B_KBLK;
  constexpr int KSTEPS = NPAD / 16;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char* As = smem;                      // PARTS x A_BYTES, dE/dT rows (A operand)
  unsigned char* ring = smem + PARTS * A_BYTES;  // B stages
  short* runl_s = reinterpret_cast<short*>(ring + S * B_STAGE);  // [32 atoms][nc] run intervals of the tile
  int* ex_s = reinterpret_cast<int*>(runl_s + kAtoms * g.nc);       // [128] power-of-two scale of each row
  uint64_t* bar = reinterpret_cast<uint64_t*>(ex_s + kRows);
  uint64_t* bfull = bar;
  uint64_t* bempty = bar + S;
  uint64_t* afull = bar + 2 * S;
  uint64_t* accfull = afull + 1;     // [kAccBufs]
  uint64_t* accempty = accfull + kAccBufs;  // [kAccBufs]
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(accempty + kAccBufs);
  int* ghi = reinterpret_cast<int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int ti = 0;
  while (ti + 1 < g.ntypes && (int)blockIdx.x >= g.tile_start[ti + 1]) ++ti;
  const int row0 = g.row_start[ti] + ((int)blockIdx.x - g.tile_start[ti]) * kAtoms;
  const int row_end = g.row_start[ti + 1];

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&bfull[s], 1);
      mbar_init(&bempty[s], 1);
    }
    mbar_init(afull, g.gTt ? kRows : 1);
    for (int b = 0; b < kAccBufs; ++b) {
      mbar_init(&accfull[b], 1);
      mbar_init(&accempty[b], kRows);
    }
    for (int t = 0; t < DP_MAX_TYPES; ++t) ghi[t] = -1;
    mbar_fence_init();
  }
  if (warp == 4) tmem_alloc(tmem_holder, 64 * kAccBufs);
  const int r = threadIdx.x;
  const int ae = r >> 2, c = r & 3;
  const int pe = row0 + ae;
  stage_runs(g, row0, row_end, runl_s, threadIdx.x, kMomThreads);
  __syncthreads();
  if (warp == 0) tile_groups(g, runl_s, lane, ghi);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  int nch = 0;
  for (int t = 0; t < g.ntypes; ++t) nch += ghi[t] + 1;

  if (warp == 5) {
    if (lane == 0) {
      // ---- TMA producer: a stage's coefficient blocks as soon as the stage is free ----
      int issued = 0;
      for (int ch = 0; ch < nch; ++ch) {
        const int s = ch % S;
        if (ch >= S && !mbar_wait(&bempty[s], ((ch / S) - 1) & 1, g.err)) break;
        int t, grp;
        block_of(ch, ghi, g.ntypes, t, grp);
        unsigned char* bs = ring + s * B_STAGE;
        mbar_expect_tx(&bfull[s], B_STAGE);
        const int y = ((ti * g.ntypes + t) * g.lcp + 8 * grp) * 8;
        tma_load_2d(bs, &bhi, &bfull[s], 0, y);
        tma_load_2d(bs + B_KBLK, &bhi, &bfull[s], 64, y);
        if (PARTS == 2) {
          tma_load_2d(bs + 2 * B_KBLK, &blo, &bfull[s], 0, y);
          tma_load_2d(bs + 3 * B_KBLK, &blo, &bfull[s], 64, y);
        }
        issued = ch + 1;
      }
      // only the last S loads can still be in flight: they must land before the CTA leaves
      for (int ch = max(0, issued - S); ch < issued; ++ch) mbar_wait(&bfull[ch % S], (ch / S) & 1, g.err);
    }
  } else if (warp == 4) {
    if (lane == 0) {
      // ---- the A operand of this tile and its row scales (copied, or formed by the builder warps) ----
      if (!g.gTt) {
        mbar_expect_tx(afull, PARTS * A_BYTES + kRows * 4);
        bulk_load(As, g.gta + (long)blockIdx.x * PARTS * A_BYTES, PARTS * A_BYTES, afull);
        bulk_load(ex_s, g.gtx + (long)blockIdx.x * kRows, kRows * 4, afull);
      }
      bool ok = mbar_wait(afull, 0, g.err);
      // ---- MMA issuer ----
      const uint32_t idesc = idesc_f16(kRows, 64, NPASS == 1 ? 0 : 1);
      for (int ch = 0; ok && ch < nch; ++ch) {
        const int s = ch % S, buf = ch % kAccBufs;
        if (!mbar_wait(&bfull[s], (ch / S) & 1, g.err)) {
          ok = false;
          break;
        }
        if (ch >= kAccBufs && !mbar_wait(&accempty[buf], ((ch / kAccBufs) - 1) & 1, g.err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t sa = su32(As), sb = su32(ring + s * B_STAGE);
        const uint32_t acc = tmem + (uint32_t)(buf * 64);
#pragma unroll
        for (int ks = 0; ks < KSTEPS; ++ks) {
          const uint32_t kbk = (uint32_t)(ks >> 2), ko = (uint32_t)(ks & 3) * 2;
          const uint64_t ah = sdesc_sw128(sa + kbk * kABlock) + ko;
          const uint64_t bh = sdesc_sw128(sb + kbk * B_KBLK) + ko;
          mma_f16(acc, ah, bh, idesc, ks != 0);
          if (NPASS == 3) {
            const uint64_t al = sdesc_sw128(sa + A_BYTES + kbk * kABlock) + ko;
            const uint64_t bl = sdesc_sw128(sb + 2 * B_KBLK + kbk * B_KBLK) + ko;
            mma_f16(acc, ah, bl, idesc, 1);
            mma_f16(acc, al, bh, idesc, 1);
          }
        }
        mma_commit(&bempty[s]);
        mma_commit(&accfull[buf]);
      }
      if (ok && nch > 0) atomicAdd(&g.mma_blocks[1], (unsigned)nch);
    }
  } else {
    if constexpr (NPASS == 3) if (g.gTt) {
      // row r = (atom ae, component c) of the A operand: dE/dT[m][c] for m < M (zero to NPAD),
      // scaled by a power of two to its largest magnitude, in the swizzled K-major image
      const bool va = pe < row_end;
      const long stride = (long)g.row_start[g.ntypes] * 4;  // one m of every row
      const float* src = g.gTt + (long)pe * 4 + c;
      float v[NPAD];  // every load in flight at once (for one m the warp reads 8 rows x 16 B, contiguous)
#pragma unroll
      for (int m = 0; m < NPAD; ++m) v[m] = (va && m < g.M) ? __ldg(src + m * stride) : 0.f;
      float mx = 0.f;
#pragma unroll
      for (int m = 0; m < NPAD; ++m) mx = fmaxf(mx, fabsf(v[m]));
      int ex = 0;
      if (mx > 0.f) frexpf(mx, &ex);
#pragma unroll
      for (int qq = 0; qq < NPAD / 8; ++qq) {
        float w[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) w[e] = ldexpf(v[8 * qq + e], -ex);
        const uint32_t off = (uint32_t)((qq >> 3) * kABlock) + sw_off(r, qq & 7);
        store_chunk<NPASS>(As + off, As + A_BYTES + off, w);
      }
      ex_s[r] = ex;
      fence_async_smem();
      mbar_arrive(afull);
    }
    mbar_wait(afull, 0, g.err);  // the row scales arrived with the A operand
    const float pscale = ldexpf(g.inv_nc, ex_s[r]);
    int cur_t = -1, ptr = 0, selt = 0;
    long rbase = 0;
    bool dead = false;  // after a timed-out wait: stop waiting, keep taking part in the barriers
    const uint32_t tb = tmem + ((uint32_t)(warp * 32) << 16);
    for (int ch = 0; ch < nch; ++ch) {
      const int buf = ch % kAccBufs;
      if (!dead && !mbar_wait(&accfull[buf], (ch / kAccBufs) & 1, g.err)) dead = true;
      __syncwarp();  // tcgen05.ld is warp-collective
      tc_fence_after();
      float P[64];
#pragma unroll
      {
        uint32_t raw[64];
#pragma unroll
        for (int q = 0; q < 4; ++q) tmem_ld16_async(tb + (uint32_t)(buf * 64 + 16 * q), raw + 16 * q);
        tmem_wait_ld();
#pragma unroll
        for (int e = 0; e < 64; ++e) P[e] = __uint_as_float(raw[e]);
      }
      tc_fence_before();
      mbar_arrive(&accempty[buf]);
      int t, grp;
      block_of(ch, ghi, g.ntypes, t, grp);
      if (t != cur_t) {
        cur_t = t;
        selt = g.sel_off[t + 1] - g.sel_off[t];
        ptr = 0;
        rbase = (long)pe * g.nc + g.sel_off[t];
      }
      const short* myruns = runl_s + ae * g.nc + g.sel_off[t];
      while (ptr < selt) {
        const int l = myruns[ptr];
        if (l < 8 * grp) break;  // also the end marker -1
        float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        switch ((l - 8 * grp) & 7) {
#define DPGB_SEL(Q)                                              \
  case Q:                                                        \
    _Pragma("unroll") for (int e = 0; e < 6; ++e) v[e] = P[8 * Q + e] * pscale; \
    break;
          DPGB_SEL(0)
          DPGB_SEL(1)
          DPGB_SEL(2)
          DPGB_SEL(3)
          DPGB_SEL(4)
          DPGB_SEL(5)
          DPGB_SEL(6)
          DPGB_SEL(7)
#undef DPGB_SEL
        }
        if (NPASS == 1) {  // mixed mode: the six values of the run as BF16 (one 16-byte chunk)
          uint32_t w[4];
#pragma unroll
          for (int h2 = 0; h2 < 3; ++h2) {
            const __nv_bfloat162 pr = __floats2bfloat162_rn(v[2 * h2], v[2 * h2 + 1]);
            w[h2] = *reinterpret_cast<const uint32_t*>(&pr);
          }
          w[3] = 0u;
          reinterpret_cast<uint4*>(g.run_P)[(rbase + ptr) * 4 + c] = make_uint4(w[0], w[1], w[2], w[3]);
        } else {
          float4* dst = g.run_P + ((rbase + ptr) * 4 + c) * 2;
          dst[0] = make_float4(v[0], v[1], v[2], v[3]);
          dst[1] = make_float4(v[4], v[5], 0.f, 0.f);
        }
        ++ptr;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 4) tmem_dealloc(tmem, 64 * kAccBufs);
}

// =============================================================================================
// Backward, per-slot part: dE/dr_ij of every listed pair from its run's P record, the force
// scatter (FP64 atomics on the neighbours, F_i accumulated per atom) and the per-atom virial.
// One warp per atom, lanes over its slots:
//   dE/dR_c = sum_p tau^p P_{p,c},  dE/ds = sum_c R_c sum_p p tau^{p-1} P_{p,c} / Delta_l
//   dE/dr_ij = ds/dr (dE/ds + dE/dR_0 + g.u) u + (s / r) (g - (g.u) u),  g = dE/dR_{1..3}
// =============================================================================================
__global__ void __launch_bounds__(256)
    k_force_mom(PathConst pc, MomArgs g) {
  const int p = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (p >= pc.natoms) return;  // warp-uniform
  const int i = g.perm[p];
  float fi[3] = {0.f, 0.f, 0.f}, vir[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int* nlrow = g.nl_j + (long)i * pc.nc;
  // (type, 32-slot batch) in order; the next batch's list entries are loaded before the current
  // batch is worked on, so one fewer dependent load is exposed per batch
  int t = 0, base = g.sel_off[0];
  int jn = lane < g.sel_off[1] - base ? nlrow[base + lane] : -1;
  while (t < pc.ntypes) {
    const int kb0 = g.sel_off[t], kb1 = g.sel_off[t + 1];
    const int jc = jn;
    const bool any = __any_sync(0xffffffffu, jc >= 0);  // real neighbours fill the front of the block
    int tn = t, bn = base + 32;
    if (!any || bn >= kb1) {
      tn = t + 1;
      bn = tn < pc.ntypes ? g.sel_off[tn] : 0;
    }
    jn = (tn < pc.ntypes && bn + lane < g.sel_off[tn + 1]) ? nlrow[bn + lane] : -1;
    const int k = base + lane;
    const long rbase = (long)p * pc.nc + kb0;
    t = tn;
    base = bn;
    {
      if (!any) continue;
      const int j = jc;
      if (j < 0) continue;
      const long row = (long)p * pc.nc + k;
      const float4 e0 = g.envU[row], e1 = g.envB[row];
      const long run = rbase + g.slot_run[row];
      const float tau = e1.z;
      const int l = __float_as_int(e1.w);
      float gR[4], dg[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float P[6];
        if (g.p_bf16) {
          const uint4 h = reinterpret_cast<const uint4*>(g.run_P)[run * 4 + c];
          P[0] = __uint_as_float(h.x << 16);
          P[1] = __uint_as_float(h.x & 0xFFFF0000u);
          P[2] = __uint_as_float(h.y << 16);
          P[3] = __uint_as_float(h.y & 0xFFFF0000u);
          P[4] = __uint_as_float(h.z << 16);
          P[5] = __uint_as_float(h.z & 0xFFFF0000u);
        } else {
          const float4 x = g.run_P[run * 8 + 2 * c], y = g.run_P[run * 8 + 2 * c + 1];
          P[0] = x.x;
          P[1] = x.y;
          P[2] = x.z;
          P[3] = x.w;
          P[4] = y.x;
          P[5] = y.y;
        }
        gR[c] = P[0] + tau * (P[1] + tau * (P[2] + tau * (P[3] + tau * (P[4] + tau * P[5]))));
        dg[c] = P[1] + tau * (2.f * P[2] + tau * (3.f * P[3] + tau * (4.f * P[4] + tau * (5.f * P[5]))));
      }
      const float s = e0.x, u0 = e0.y, u1 = e0.z, u2 = e0.w, ds = e1.x, rr = e1.y;
      const float invd = l < g.n1 ? g.inv1 : g.inv2;
      const float gs = s * (dg[0] + u0 * dg[1] + u1 * dg[2] + u2 * dg[3]) * invd;
      const float gvu = gR[1] * u0 + gR[2] * u1 + gR[3] * u2;
      const float A_ = ds * (gs + gR[0] + gvu), B_ = s / rr;
      const float gd[3] = {A_ * u0 + B_ * (gR[1] - gvu * u0), A_ * u1 + B_ * (gR[2] - gvu * u1),
                           A_ * u2 + B_ * (gR[3] - gvu * u2)};
      const float dv[3] = {rr * u0, rr * u1, rr * u2};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        atomicAdd(g.force + 3 * j + a, widen(-gd[a]));
        fi[a] += gd[a];
#pragma unroll
        for (int b = 0; b < 3; ++b) vir[a * 3 + b] -= gd[a] * dv[b];
      }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int a = 0; a < 3; ++a) fi[a] += __shfl_xor_sync(0xffffffffu, fi[a], off);
#pragma unroll
    for (int q = 0; q < 9; ++q) vir[q] += __shfl_xor_sync(0xffffffffu, vir[q], off);
  }
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) atomicAdd(g.force + 3 * i + a, widen(fi[a]));
#pragma unroll
    for (int q = 0; q < 9; ++q) g.avir[9L * i + q] = widen(vir[q]);
  }
}

// Tables of the moment contraction from the quintic coefficients (FP64, [net][l][m][8]).
//   fwd [ti * npad + n][(t * lcp + l) * 8 + p]       bwd [((ti * ntypes + t) * lcp + l) * 8 + p][n < 128]
// value a_{l,n,p} Delta_l^p (zero for padding); FP16, or BF16 high and low parts.
__global__ void k_mom_tables(const double* __restrict__ tab, int ntypes, int one_side, int M, int lc, int lcp,
                             int n1, double stride1, double stride2, int npad, int npass, void* fwd_hi, void* fwd_lo,
                             void* bwd_hi, void* bwd_lo) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long total = (long)ntypes * ntypes * lcp * 8 * 128;  // (ti, t, l, p, n < 128)
  if (e >= total) return;
  const int n = (int)(e % 128);
  long rest = e / 128;
  const int pw = (int)(rest % 8);
  rest /= 8;
  const int l = (int)(rest % lcp);
  rest /= lcp;
  const int t = (int)(rest % ntypes);
  const int ti = (int)(rest / ntypes);
  double v = 0.0;
  if (n < M && l < lc && pw < 6) {
    const int net = one_side ? t : ti * ntypes + t;
    const double dl = l < n1 ? stride1 : stride2;
    v = tab[(((size_t)net * lc + l) * M + n) * 8 + (5 - pw)];
    for (int q = 0; q < pw; ++q) v *= dl;
  }
  const long bi = (((long)(ti * ntypes + t) * lcp + l) * 8 + pw) * 128 + n;
  const long fi = (long)(ti * npad + n) * ((long)ntypes * lcp * 8) + (long)(t * lcp + l) * 8 + pw;
  if (npass == 1) {
    const __half h = __double2half(v);
    reinterpret_cast<__half*>(bwd_hi)[bi] = h;
    if (n < npad) reinterpret_cast<__half*>(fwd_hi)[fi] = h;
  } else {
    const __nv_bfloat16 h = __double2bfloat16(v);
    const __nv_bfloat16 lo = __double2bfloat16(v - (double)__bfloat162float(h));
    reinterpret_cast<__nv_bfloat16*>(bwd_hi)[bi] = h;
    reinterpret_cast<__nv_bfloat16*>(bwd_lo)[bi] = lo;
    if (n < npad) {
      reinterpret_cast<__nv_bfloat16*>(fwd_hi)[fi] = h;
      reinterpret_cast<__nv_bfloat16*>(fwd_lo)[fi] = lo;
    }
  }
}

size_t fwd_smem(int npass, int npad, int nc) {
  const int parts = npass == 1 ? 1 : 2, S = npass == 1 ? MomStages<1>::value : MomStages<3>::value;
  return (size_t)S * parts * (kABlock + npad * 128) + (size_t)kAtoms * nc * 2 + (2 * S + 1) * 8 + 4 +
         4 * DP_MAX_TYPES + 1024 + 64;
}
size_t bwd_smem(int npass, int nc) {
  const int parts = npass == 1 ? 1 : 2;
  const int S = npass == 1 ? BwdDepth<1>::stages : BwdDepth<3>::stages;
  const int nacc = npass == 1 ? BwdDepth<1>::acc : BwdDepth<3>::acc;
  return (size_t)parts * 2 * kABlock + S * (size_t)parts * 2 * 64 * 128 + (size_t)kAtoms * nc * 2 +
         kRows * 4 + (2 * S + 1 + 2 * nacc) * 8 + 4 + 4 * DP_MAX_TYPES + 1024 + 64;
}

template <int NPASS, int NPAD>
int launch_mom(const DeviceModel& m, const MomArgs& g, int tiles, int which, cudaStream_t st) {
  const CUtensorMap* maps = reinterpret_cast<const CUtensorMap*>(m.mom_maps.data());
  if (which == 1) {
    k_mom_gT<NPASS, NPAD><<<dim3(tiles, kAtoms / kGroupAtoms), kRows, 0, st>>>(g);
  } else if (which == 0) {
    const size_t sm = fwd_smem(NPASS, NPAD, g.nc);
    DP_CUDA_TRY(allow_max_smem(k_mom_fwd<NPASS, NPAD>));
    k_mom_fwd<NPASS, NPAD><<<tiles, kMomThreads, sm, st>>>(maps[0], maps[1], g);
  } else {
    const size_t sm = bwd_smem(NPASS, g.nc);
    DP_CUDA_TRY(allow_max_smem(k_mom_bwd<NPASS, NPAD>));
    k_mom_bwd<NPASS, NPAD><<<tiles, kMomThreads, sm, st>>>(maps[2], maps[3], g);
  }
  DP_CUDA_TRY(cudaGetLastError());
  return DP_OK;
}

template <int NPASS>
int launch_mom_np(const DeviceModel& m, const MomArgs& g, int tiles, int which, cudaStream_t st) {
  if (m.mom_npad == 16) return launch_mom<NPASS, 16>(m, g, tiles, which, st);
  if (m.mom_npad == 32) return launch_mom<NPASS, 32>(m, g, tiles, which, st);
  if (m.mom_npad == 64) return launch_mom<NPASS, 64>(m, g, tiles, which, st);
  if (m.mom_npad == 112) return launch_mom<NPASS, 112>(m, g, tiles, which, st);
  if (m.mom_npad == 128) return launch_mom<NPASS, 128>(m, g, tiles, which, st);
  set_error("moment path: unsupported padded width");
  return DP_E_UNSUPPORTED;
}

}  // namespace

int mom_npad_of(int M) {
  if (M <= 16) return 16;
  if (M <= 32) return 32;
  if (M <= 64) return 64;
  if (M <= 112) return 112;
  if (M <= 128) return 128;
  return 0;
}

bool mom_supported(const DeviceModel& m) {
  int nc = 0;
  for (int t = 0; t < m.cfg.ntypes; ++t) nc += m.cfg.sel[t];
  // the run lists of a tile's 32 atoms stay in shared memory beside the operand rings
  return m.compressed && (m.precision == DP_PREC_FP32 || m.precision == DP_PREC_BF16) && mom_npad_of(m.M) > 0 &&
         m.A <= 16 && (m.M * m.A) % 4 == 0 && nc <= 512;
}

int build_mom_tables(DeviceModel& m) {
  if (!mom_supported(m) || !m.tab64) return DP_OK;
  const int nt = m.cfg.ntypes, lc = m.tab.n1 + m.tab.n2, lcp = (lc + 7) / 8 * 8;
  const int npad = mom_npad_of(m.M);
  const int npass = m.precision == DP_PREC_BF16 ? 1 : 3;
  const long kcols = (long)nt * lcp * 8;
  const long fwd_elems = (long)nt * npad * kcols;
  const long bwd_elems = (long)nt * nt * lcp * 8 * 128;
  const int parts = npass == 1 ? 1 : 2;
  DP_CUDA_TRY(cudaMalloc(&m.mom_tab, (size_t)parts * (fwd_elems + bwd_elems) * 2));
  unsigned char* base = reinterpret_cast<unsigned char*>(m.mom_tab);
  void* fwd_hi = base;
  void* fwd_lo = base + fwd_elems * 2;
  void* bwd_hi = base + (size_t)parts * fwd_elems * 2;
  void* bwd_lo = reinterpret_cast<unsigned char*>(bwd_hi) + bwd_elems * 2;
  DP_CUDA_TRY(cudaMemset(m.mom_tab, 0, (size_t)parts * (fwd_elems + bwd_elems) * 2));
  const long total = bwd_elems;
  k_mom_tables<<<(unsigned)((total + 255) / 256), 256>>>(m.tab64, nt, m.cfg.type_one_side, m.M, lc, lcp, m.tab.n1,
                                                         m.tab.stride1, m.tab.stride2, npad, npass, fwd_hi, fwd_lo,
                                                         bwd_hi, bwd_lo);
  DP_CUDA_TRY(cudaGetLastError());
  DP_CUDA_TRY(cudaDeviceSynchronize());
  m.mom_maps.assign(4 * sizeof(CUtensorMap), 0);
  CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(m.mom_maps.data());
  int rc = make_tmap_bf16(&maps[0], fwd_hi, (long)nt * npad, kcols, npad);
  if (rc == DP_OK) rc = make_tmap_bf16(&maps[1], parts == 2 ? fwd_lo : fwd_hi, (long)nt * npad, kcols, npad);
  if (rc == DP_OK) rc = make_tmap_bf16(&maps[2], bwd_hi, (long)nt * nt * lcp * 8, 128, 64);
  if (rc == DP_OK) rc = make_tmap_bf16(&maps[3], parts == 2 ? bwd_lo : bwd_hi, (long)nt * nt * lcp * 8, 128, 64);
  if (rc != DP_OK) return rc;
  m.mom_npass = npass;
  m.mom_npad = npad;
  m.mom_lcp = lcp;
  return DP_OK;
}

int run_mom(const DeviceModel& m, const PathConst& pc, const PathIO& io, Arena& ar, cudaStream_t st) {
  const long N = pc.natoms;
  const int M = pc.M, A = pc.A;
  const bool bf16 = m.mom_npass == 1;
  // FP32 mode: the fitting net on split BF16 operands (three tensor-core passes) when the
  // model's low weight halves exist, else on the FP32 CUDA-core kernels
  const bool split_fit = !bf16 && m.fit_wt_bf16_lo != nullptr;
  float* Tm = ar.get<float>(N * M * 4);
  void* D = (bf16 || split_fit) ? (void*)ar.get<__nv_bfloat16>(N * M * A) : (void*)ar.get<float>(N * M * A);
  __nv_bfloat16* D_lo = split_fit ? ar.get<__nv_bfloat16>(N * M * A) : nullptr;
  const long slots = N * pc.nc;
  const int parts = bf16 ? 1 : 2;
  float4* envU = ar.get<float4>(slots);
  float4* envB = ar.get<float4>(slots);
  int* slot_run = ar.get<int>(slots);
  int* run_l = ar.get<int>(slots);
  // run moments (forward) and run P (backward) share one buffer: the moments are dead by then
  void* runs = ar.get<float4>(slots * 8 > slots * 4 * parts ? slots * 8 : slots * 4 * parts);
  const long max_tiles = (N + kAtoms - 1) / kAtoms + pc.ntypes;  // every type's last tile may be short
  unsigned char* gta = ar.get<unsigned char>(max_tiles * (bf16 ? 1 : 2) * 2 * kABlock);
  int* gtx = ar.get<int>(max_tiles * kRows);
  // FP32 mode: dE/dT straight from the split fitting kernel when it runs (M_< = 16)
  float* gTt = split_fit && A == 16 ? ar.get<float>(N * M * 4) : nullptr;
  const float* gD = nullptr;
  const __nv_bfloat16* gDh = nullptr;
  if (ar.measure) {
    if (bf16) return run_fitting_tc(m, pc, reinterpret_cast<const __nv_bfloat16*>(D), io, ar, st, &gD, &gDh);
    if (split_fit)
      return run_fitting_tc(m, pc, reinterpret_cast<const __nv_bfloat16*>(D), io, ar, st, &gD, nullptr, D_lo, Tm,
                            gTt);
    return run_fitting<float>(m, pc, m.p32, reinterpret_cast<const float*>(D), io, ar, st, &gD);
  }
  if (!ar.ok()) {
    set_error("scratch allocation failed");
    return DP_E_OOM;
  }
  MomArgs g;
  std::memset(&g, 0, sizeof(g));
  g.ntypes = pc.ntypes;
  g.nc = pc.nc;
  g.M = M;
  g.A = A;
  g.lc = m.tab.n1 + m.tab.n2;
  if (g.lc > 32767) {  // run intervals are staged as 16-bit values
    set_error("compressed table with more than 32767 intervals");
    return DP_E_ARG;
  }
  g.lcp = m.mom_lcp;
  g.n1 = m.tab.n1;
  g.s0 = (float)m.tab.s0;
  g.stride1 = (float)m.tab.stride1;
  g.stride2 = (float)m.tab.stride2;
  g.inv1 = (float)(1.0 / m.tab.stride1);
  g.inv2 = (float)(1.0 / m.tab.stride2);
  g.split = (float)(m.tab.s0 + m.tab.n1 * m.tab.stride1);
  g.smax = (float)(m.tab.s0 + m.tab.n1 * m.tab.stride1 + m.tab.n2 * m.tab.stride2);
  g.inv_nc = 1.0f / (float)pc.nc;
  for (int t = 0; t <= pc.ntypes; ++t) {
    g.sel_off[t] = pc.sel_off[t];
    g.row_start[t] = io.type_start[t];
  }
  g.tile_start[0] = 0;
  for (int t = 0; t < pc.ntypes; ++t)
    g.tile_start[t + 1] = g.tile_start[t] + (io.type_start[t + 1] - io.type_start[t] + kAtoms - 1) / kAtoms;
  const int tiles = g.tile_start[pc.ntypes];
  g.perm = io.perm;
  g.nl_j = io.nl_j;
  g.envU = envU;
  g.envB = envB;
  g.slot_run = slot_run;
  g.run_l = run_l;
  g.run_rec = reinterpret_cast<uint4*>(runs);
  g.run_P = reinterpret_cast<float4*>(runs);
  g.p_bf16 = bf16 ? 1 : 0;
  g.atom_l = io.atom_l;
  g.atom_m = io.atom_m;
  g.geoms = io.geoms;
  g.disp = io.disp;
  g.Tm = Tm;
  g.D = D;
  g.D_lo = D_lo;
  g.d_bf16 = bf16 ? 1 : (split_fit ? 2 : 0);
  g.force = io.force;
  g.avir = io.atom_virial;
  g.gta = gta;
  g.gtx = gtx;
  char* stw = reinterpret_cast<char*>(io.status);
  g.table_range = reinterpret_cast<int*>(stw + offsetof(DevStatus, table_range));
  g.err = reinterpret_cast<int*>(stw + offsetof(DevStatus, timeout));
  g.mma_blocks = reinterpret_cast<unsigned int*>(stw + offsetof(DevStatus, mma_blocks));
  {
    ProfScope _ps(io.prof, "env", st);
    // one warp per (atom, neighbour type) task; persistent warps, three 8-warp blocks per SM
    const long tasks = N * pc.ntypes;
    const unsigned blocks = (unsigned)std::min<long>((tasks + 7) / 8, 3L * sm_count());
    if (bf16)
      k_env_mom<1><<<blocks, 256, 0, st>>>(pc, g, io.coord, io.nl_code);
    else
      k_env_mom<3><<<blocks, 256, 0, st>>>(pc, g, io.coord, io.nl_code);
    DP_CUDA_TRY(cudaGetLastError());
  }
  if (tiles > 0) {
    ProfScope _ps(io.prof, "mom_fwd", st);
    const int rc = bf16 ? launch_mom_np<1>(m, g, tiles, 0, st) : launch_mom_np<3>(m, g, tiles, 0, st);
    if (rc != DP_OK) return rc;
  }
  int rc;
  if (bf16)
    rc = run_fitting_tc(m, pc, reinterpret_cast<const __nv_bfloat16*>(D), io, ar, st, &gD, &gDh);
  else if (split_fit)
    rc = run_fitting_tc(m, pc, reinterpret_cast<const __nv_bfloat16*>(D), io, ar, st, &gD, nullptr, D_lo, Tm, gTt);
  else
    rc = run_fitting<float>(m, pc, m.p32, reinterpret_cast<const float*>(D), io, ar, st, &gD);
  if (rc != DP_OK) return rc;
  g.gD = gD;
  g.gDh = gDh;
  g.gTt = (split_fit && gD == nullptr) ? gTt : nullptr;  // the split kernel formed dE/dT itself
  if (tiles > 0) {
    if (!g.gTt) {
      ProfScope _ps(io.prof, "mom_gT", st);
      rc = bf16 ? launch_mom_np<1>(m, g, tiles, 1, st) : launch_mom_np<3>(m, g, tiles, 1, st);
      if (rc != DP_OK) return rc;
    }
    {
      ProfScope _ps(io.prof, "mom_bwd", st);
      rc = bf16 ? launch_mom_np<1>(m, g, tiles, 2, st) : launch_mom_np<3>(m, g, tiles, 2, st);
      if (rc != DP_OK) return rc;
    }
    ProfScope _ps(io.prof, "mom_force", st);
    k_force_mom<<<(unsigned)((N * 32 + 255) / 256), 256, 0, st>>>(pc, g);
    DP_CUDA_TRY(cudaGetLastError());
  }
  return DP_OK;
}

}  // namespace dpgb
