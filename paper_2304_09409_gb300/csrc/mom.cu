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
// dE/ds = (1/Nc) sum_c R_c sum_p p tau^{p-1} P_{p,c} / Delta_l.  The epilogue reads P for one
// 8-interval block from TMEM, walks each atom's neighbours in that block and scatters the pair
// forces (FP64 atomics) and the per-atom virial, as the CUDA-core compressed kernel does.
//
// Neighbours of each type block are sorted by distance, so their intervals are non-increasing
// along the list and every (atom, interval) is a contiguous run; the few FP32 rounding
// inversions are folded into the run of the previous neighbour (its polynomial piece evaluated
// a rounding error beyond its end, where the pieces join with C^2 continuity).  Most
// neighbours sit in the first intervals (s < 0.01 reaches from about 0.6 r_c to r_c), so the
// walks are spread evenly: the four warps of a CTA take every fourth slot of each list and the
// 32 lanes of a warp take the 32 atoms of the tile, all in step.
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
constexpr int kThreads = 160;     // 4 builder / epilogue warps + 1 control warp
constexpr int kABlock = kRows * 128;  // one 64-column K block of 128 rows (bytes)
constexpr int kGroupAtoms = 4;        // backward: atoms per staged group of dE/dD rows

struct MomArgs {
  int ntypes, nc, M, A, lc, lcp, n1;
  float s0, stride1, stride2, inv1, inv2, split, smax, inv_nc;
  int sel_off[DP_MAX_TYPES + 1];
  int row_start[DP_MAX_TYPES + 1];
  int tile_start[DP_MAX_TYPES + 1];
  const int* perm;
  const int* nl_j;
  // per-slot records, rows in sorted atom order [N * nc]: (s, s u), (s, u), (ds/dr, r, tau, l)
  const float4* envR;
  const float4* envU;
  const float4* envB;
  float* Tm;          // [N][M][4]
  void* D;            // [N][M * A], BF16 or FP32
  int d_bf16;
  const float* gD;  // [N][M * A]
  double* force;    // [N][3] input order
  double* avir;     // [N][9] input order
  unsigned char* gta;  // backward A operand per tile: the shared-memory image of dE/dT rows
  int* gtx;            // its row scales [tiles][128]
  int* table_range;
  int* err;
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

// Walks of one atom's neighbour list of one type; lane a of a warp takes atom a, so a warp
// advances 32 atoms in step.  Each thread streams its own slots' records through two private
// shared-memory windows with cp.async, one window ahead of the one it reads: no other thread
// touches them, so no synchronisation is needed.  The records carry intervals already made
// non-increasing along the list (k_env_mom).
//
// Forward: warp c walks whole lists for component c, reading R_c and (tau, l) of each slot.
constexpr int kWinF = 8;
struct FWalk {
  int k, kend, wbase, cur;
  bool have;
  int l;
  float tau, R;
};
struct FWindow {  // this thread's two windows
  float* R;       // [2][kWinF]
  float2* tl;     // [2][kWinF]
};
__device__ __forceinline__ void fwin_fill(const MomArgs& g, int p, int c, const FWindow& win, int buf, int k0,
                                          int kend) {
#pragma unroll
  for (int q = 0; q < kWinF; ++q) {
    const int slot = k0 + q;
    if (slot < kend) {
      const long row = (long)p * g.nc + slot;
      cp_async4(win.R + buf * kWinF + q, reinterpret_cast<const float*>(g.envR + row) + c);
      cp_async8(win.tl + buf * kWinF + q, reinterpret_cast<const float*>(g.envB + row) + 2);
    }
  }
  cp_async_commit();
}
__device__ __forceinline__ void fwalk_start(const MomArgs& g, int p, int c, const FWindow& win, FWalk& w, int kbeg,
                                            int kend) {
  w.k = kbeg;
  w.kend = kend;
  w.wbase = kbeg;
  w.cur = 0;
  w.have = false;
  for (int slot = kbeg + 2 * kWinF + c * 8; slot < kend; slot += 32) {  // the four warps split the lines
    const long row = (long)p * g.nc + slot;
    prefetch_l2(g.envR + row);
    prefetch_l2(g.envB + row);
  }
  cp_async_wait0();  // no copy of an earlier walk is still in flight into the windows
  fwin_fill(g, p, c, win, 0, kbeg, kend);
  fwin_fill(g, p, c, win, 1, kbeg + kWinF, kend);
  cp_async_wait1();
}
__device__ __forceinline__ void fwalk_next(const MomArgs& g, int p, int c, const FWindow& win, FWalk& w) {
  w.have = false;
  if (w.k >= w.kend) return;
  if (w.k >= w.wbase + kWinF) {  // current window used up: refill it two windows ahead, switch
    fwin_fill(g, p, c, win, w.cur, w.wbase + 2 * kWinF, w.kend);
    w.cur ^= 1;
    w.wbase += kWinF;
    cp_async_wait1();
  }
  const int q = w.cur * kWinF + (w.k - w.wbase);
  const float2 tl = win.tl[q];
  const int l = __float_as_int(tl.y);
  if (l < 0) {  // padding: real neighbours fill the front of the type block
    w.kend = w.k;
    return;
  }
  w.R = win.R[q];
  w.l = l;
  w.tau = tl.x;
  w.have = true;
  ++w.k;
}

// Backward: the four warps take every fourth slot (phase = warp) and read (s, u), (ds, r, tau, l)
// and the neighbour index; the phase's slots are also prefetched into L2 when its walk starts.
constexpr int kWin = 4;
constexpr int kStep = 4;
struct Walk {
  int k, kend, wbase, cur;  // next slot, end of the block, first slot of the current window, its buffer
  bool have;
  int l, j;
  float tau;
  float4 e0, e1;  // (s, u), (ds, r, tau, l)
};
struct Window {  // this thread's two windows
  float4* e0;    // [2][kWin]
  float4* e1;    // [2][kWin]
  int* j;        // [2][kWin]
};

__device__ __forceinline__ void win_fill(const MomArgs& g, int p, int i, const Window& win, int buf, int k0,
                                         int kend) {
#pragma unroll
  for (int q = 0; q < kWin; ++q) {
    const int slot = k0 + kStep * q;
    if (slot < kend) {
      const long row = (long)p * g.nc + slot;
      cp_async16(win.e0 + buf * kWin + q, g.envU + row);
      cp_async16(win.e1 + buf * kWin + q, g.envB + row);
      cp_async4(win.j + buf * kWin + q, g.nl_j + (long)i * g.nc + slot);
    }
  }
  cp_async_commit();
}

__device__ __forceinline__ void walk_start(const MomArgs& g, int p, int i, const Window& win, Walk& w, int kbeg,
                                           int kend) {
  w.k = kbeg;
  w.kend = kend;
  w.wbase = kbeg;
  w.cur = 0;
  w.have = false;
  for (int slot = kbeg + 2 * kStep * kWin; slot < kend; slot += kStep) {
    const long row = (long)p * g.nc + slot;
    prefetch_l2(g.envU + row);
    prefetch_l2(g.envB + row);
  }
  cp_async_wait0();  // no copy of an earlier walk is still in flight into the windows
  win_fill(g, p, i, win, 0, kbeg, kend);
  win_fill(g, p, i, win, 1, kbeg + kStep * kWin, kend);
  cp_async_wait1();
}

__device__ __forceinline__ void walk_next(const MomArgs& g, int p, int i, const Window& win, Walk& w) {
  w.have = false;
  if (w.k >= w.kend) return;
  if (w.k >= w.wbase + kStep * kWin) {  // current window used up: refill it two windows ahead, switch
    win_fill(g, p, i, win, w.cur, w.wbase + 2 * kStep * kWin, w.kend);
    w.cur ^= 1;
    w.wbase += kStep * kWin;
    cp_async_wait1();
  }
  const int q = w.cur * kWin + (w.k - w.wbase) / kStep;
  w.e1 = win.e1[q];
  const int l = __float_as_int(w.e1.w);
  if (l < 0) {  // padding: real neighbours fill the front of the type block
    w.kend = w.k;
    return;
  }
  w.e0 = win.e0[q];
  w.j = win.j[q];
  w.l = l;
  w.tau = w.e1.z;
  w.have = true;
  w.k += kStep;
}

// Largest 8-interval group holding a neighbour of each type, over the tile's atoms.
__device__ __forceinline__ void tile_groups(const MomArgs& g, int p, int i, bool valid, int* ghi) {
  if (!valid) return;
  for (int t = 0; t < g.ntypes; ++t) {
    const int k = g.sel_off[t];
    if (k < g.sel_off[t + 1]) {
      const int l = __float_as_int(g.envB[(long)p * g.nc + k].w);
      if (l >= 0) atomicMax(&ghi[t], l >> 3);
    }
  }
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

// Ring depth of the operand stages.
template <int NPASS>
struct MomStages {
  static constexpr int value = 2;
};

// FP32 rows of one atom in the staging / P buffers: 4 rows of 68 floats (8 chunks of 8 and a
// pad), atoms 276 floats apart, which spreads a warp's 32 atoms over the banks.
constexpr int kRowPitch = 68;
constexpr int kAtomPitch = 276;
constexpr uint32_t kRowBufBytes = kAtoms * kAtomPitch * 4;
constexpr uint32_t kFwdWinBytes = kRows * 2 * kWinF * 12;  // per thread: two windows of R_c, (tau, l)
constexpr uint32_t kBwdWinBytes = kRows * 2 * kWin * 36;  // per thread: two windows of (e0, e1, j)

__host__ __device__ inline uint32_t fwd_ring_bytes(int npass, int npad) {
  const uint32_t parts = npass == 1 ? 1 : 2, stages = 2;
  return stages * parts * (uint32_t)(kABlock + npad * 128);
}
// Backward shared memory after the A operand: the B ring, the P buffer, the neighbour windows
// and the row scales.
__host__ __device__ inline uint32_t bwd_ring_bytes(int npass) {
  const uint32_t parts = npass == 1 ? 1 : 2, stages = 2;
  return stages * parts * 2u * 64u * 128u;
}
__host__ __device__ inline uint32_t bwd_region(int npass) {
  return bwd_ring_bytes(npass) + kRowBufBytes + kBwdWinBytes + kRows * 4;
}

// Per-slot records of the listed pairs (sorted atom order): (s, u) and (ds/dr, r, tau, l), with
// l = -1 marking padding; exact FP64 displacement, FP32 switch (Eq. (switch)).  One warp takes
// one (atom, neighbour type) block: the interval is lowered to the running minimum along the
// list (a prefix-minimum scan), so intervals never increase from slot to slot even where FP32
// rounding of s inverts two nearly equal distances.
__global__ void __launch_bounds__(256)
    k_env_mom(PathConst pc, MomArgs g, const double* __restrict__ coord, const int* __restrict__ nl_code,
              float4* __restrict__ envR, float4* __restrict__ envU, float4* __restrict__ envB) {
  const long task = (long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (task >= (long)pc.natoms * pc.ntypes) return;  // warp-uniform
  const int p = (int)(task / pc.ntypes), t = (int)(task % pc.ntypes);
  const int i = g.perm[p];
  int carry = INT_MAX;
  bool oor = false;
  for (int base = g.sel_off[t]; base < g.sel_off[t + 1]; base += 32) {
    const int k = base + lane;
    const bool in = k < g.sel_off[t + 1];
    const long row = (long)p * pc.nc + k;
    const int j = in ? g.nl_j[(long)i * pc.nc + k] : -1;
    int l = INT_MAX;
    float r = 0.f, s = 0.f, ds = 0.f, u[3] = {0.f, 0.f, 0.f}, tau = 0.f;
    if (j >= 0) {
      double d0, d1, d2;
      listed_disp(coord + 3 * i, coord + 3 * j, nl_code[(long)i * pc.nc + k], pc, frame_of(pc, i), d0, d1, d2);
      pair_env<float>(d0, d1, d2, norm2_exact(d0, d1, d2), pc.rs, pc.rc, pc.near2, r, s, ds, u);
      float invd;
      l = mom_interval(g, s, INT_MAX, tau, invd, oor);
    }
    int m = l;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int o = __shfl_up_sync(0xffffffffu, m, off);
      if (lane >= off) m = min(m, o);
    }
    m = min(m, carry);
    if (j >= 0 && m < l) {
      l = m;
      tau = tau_at(g, s, l);
    }
    if (in) {
      if (j >= 0) {
        envR[row] = make_float4(s, s * u[0], s * u[1], s * u[2]);
        envU[row] = make_float4(s, u[0], u[1], u[2]);
        envB[row] = make_float4(ds, r, tau, __int_as_float(l));
      } else {
        envB[row] = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
      }
    }
    carry = __shfl_sync(0xffffffffu, m, 31);
  }
  if (__any_sync(0xffffffffu, oor) && lane == 0) atomicOr(g.table_range, 1);
}

// =============================================================================================
// Forward: T and D
// =============================================================================================
template <int NPASS, int NPAD>
__global__ void __launch_bounds__(kThreads, 1)
    k_mom_fwd(const __grid_constant__ CUtensorMap bhi, const __grid_constant__ CUtensorMap blo, const MomArgs g) {
  constexpr int PARTS = NPASS == 1 ? 1 : 2;
  constexpr int S = MomStages<NPASS>::value;
  constexpr int B_BYTES = NPAD * 128;
  constexpr int STAGE = PARTS * (kABlock + B_BYTES);
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char* wins = smem + S * STAGE;
  uint64_t* full = reinterpret_cast<uint64_t*>(wins + kFwdWinBytes);
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
  // thread r < 128 owns accumulator row r = (atom r / 4, component r % 4) in the epilogue and
  // the conversion of staging row r; as a builder it walks phase `warp` of atom `lane`
  const int r = threadIdx.x;
  const int ae = r >> 2, c = r & 3;
  const int pe = row0 + ae;
  const bool valid_e = warp < 4 && pe < row_end;
  const int pb = row0 + lane;
  const bool valid_b = warp < 4 && pb < row_end;
  const int ib = valid_b ? g.perm[pb] : 0;
  if (warp == 0) tile_groups(g, pb, ib, valid_b, ghi);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  int nkb = 0;
  for (int t = 0; t < g.ntypes; ++t) nkb += ghi[t] + 1;

  if (warp == 4) {
    if (lane == 0) {
      // ---- TMA producer and MMA issuer ----
      const uint32_t idesc = idesc_f16(kRows, NPAD, NPASS == 1 ? 0 : 1);
      auto issue = [&](int kb) {
        int t, grp;
        block_of(kb, ghi, g.ntypes, t, grp);
        const int s = kb % S;
        unsigned char* bs = smem + s * STAGE + PARTS * kABlock;
        mbar_expect_tx(&full[s], PARTS * B_BYTES);
        const int x = (t * g.lcp + 8 * grp) * 8;
        tma_load_2d(bs, &bhi, &full[s], x, ti * NPAD);
        if (PARTS == 2) tma_load_2d(bs + B_BYTES, &blo, &full[s], x, ti * NPAD);
      };
      int issued = 0;
      for (; issued < S - 1 && issued < nkb; ++issued) issue(issued);
      bool ok = true;
      int done = 0;  // blocks whose loads were consumed
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % S;
        if (!mbar_wait(&full[s], (kb / S) & 1, g.err)) {
          ok = false;
          break;
        }
        done = kb + 1;
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
        const int kn = kb + S - 1;
        if (kn < nkb) {
          if (kn >= S && !mbar_wait(&empty[kn % S], ((kn / S) - 1) & 1, g.err)) {
            ok = false;
            break;
          }
          issue(kn);
          issued = kn + 1;
        }
      }
      if (ok && nkb > 0)
        mma_commit(accf);
      else
        mbar_arrive(accf);
      // loads still in flight after an error must land before the CTA leaves
      for (int kb = done; kb < issued; ++kb) mbar_wait(&full[kb % S], (kb / S) & 1, g.err);
    }
  } else {
    // ---- moment builders: warp c builds component c of the 32 atoms (lane = atom), i.e. A
    //      row (lane, c); each thread walks its atom's whole list and owns its row outright ----
    const int crow = warp;            // component built by this warp
    const int arow = lane * 4 + crow;  // A row written by this thread
    FWindow win;
    win.R = reinterpret_cast<float*>(wins) + r * 2 * kWinF;
    win.tl = reinterpret_cast<float2*>(wins + kRows * 2 * kWinF * 4) + r * 2 * kWinF;
    FWalk w;
    w.have = false;
    int cur_t = -1;
    bool dead = false;  // after a timed-out wait: stop waiting, keep going through the blocks
    const uint32_t rowoff0 = (uint32_t)((arow >> 3) * 1024 + (arow & 7) * 128);
    for (int kb = 0; kb < nkb; ++kb) {
      int t, grp;
      block_of(kb, ghi, g.ntypes, t, grp);
      const int s = kb % S;
      if (kb >= S && !dead && !mbar_wait(&empty[s], ((kb / S) - 1) & 1, g.err)) dead = true;
      if (t != cur_t) {
        cur_t = t;
        w.have = false;
        if (valid_b) {
          fwalk_start(g, pb, crow, win, w, g.sel_off[t], g.sel_off[t + 1]);
          fwalk_next(g, pb, crow, win, w);
        }
      }
      unsigned char* ahi = smem + s * STAGE;
      unsigned char* alo = ahi + kABlock;
      // runs of equal interval, accumulated in registers; intervals without neighbours get zeros
      float mu[8];
      int cur_q = -1;
      unsigned written = 0;
      for (;;) {
        const bool act = w.have && w.l >= 8 * grp;
        if (!__any_sync(0xffffffffu, act)) break;
        if (act) {
          const int q = (w.l - 8 * grp) & 7;
          if (q != cur_q) {
            if (cur_q >= 0) {
              const uint32_t off = rowoff0 + (uint32_t)((cur_q ^ (arow & 7)) << 4);
              store_chunk<NPASS>(ahi + off, alo + off, mu);
              written |= 1u << cur_q;
            }
#pragma unroll
            for (int pp = 0; pp < 8; ++pp) mu[pp] = 0.f;
            cur_q = q;
          }
          float pw = w.R;
#pragma unroll
          for (int pp = 0; pp < 6; ++pp) {
            mu[pp] += pw;
            pw *= w.tau;
          }
          fwalk_next(g, pb, crow, win, w);
        }
      }
      if (cur_q >= 0) {
        const uint32_t off = rowoff0 + (uint32_t)((cur_q ^ (arow & 7)) << 4);
        store_chunk<NPASS>(ahi + off, alo + off, mu);
        written |= 1u << cur_q;
      }
      const float zero8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (!((written >> q) & 1u)) {
          const uint32_t off = rowoff0 + (uint32_t)((q ^ (arow & 7)) << 4);
          store_chunk<NPASS>(ahi + off, alo + off, zero8);
        }
      fence_async_smem();
      mbar_arrive(&full[s]);
    }
    cp_async_wait0();  // window copies still in flight land before the CTA leaves
  }

  // ---- epilogue: T = acc / Nc, then D = T T_<^T ----
  if (warp < 4) {
    mbar_wait(accf, 0, g.err);
    __syncwarp();  // tcgen05.ld is warp-collective
    tc_fence_after();
    float* smT = reinterpret_cast<float*>(smem);  // [32 atoms][NPAD + 1][4]; the ring is idle now
    const uint32_t tb = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < NPAD; c0 += 16) {
      float v[16];
      tmem_ld16(tb + c0, v);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const float x = nkb > 0 ? v[q] * g.inv_nc : 0.f;
        smT[(ae * (NPAD + 1) + c0 + q) * 4 + c] = x;
        if (valid_e && c0 + q < g.M) g.Tm[((long)pe * g.M + c0 + q) * 4 + c] = x;
      }
    }
    tc_fence_before();
    bar_sync(1, kRows);
    if (valid_e) {
      const float4* T4 = reinterpret_cast<const float4*>(smT) + ae * (NPAD + 1);
      float4 tl[16];
#pragma unroll
      for (int l = 0; l < 16; ++l) tl[l] = l < g.A ? T4[l] : make_float4(0.f, 0.f, 0.f, 0.f);
      for (int m = c; m < g.M; m += 4) {
        const float4 tm = T4[m];
        float d[16];
#pragma unroll
        for (int l = 0; l < 16; ++l) d[l] = tm.x * tl[l].x + tm.y * tl[l].y + tm.z * tl[l].z + tm.w * tl[l].w;
        const long o = ((long)pe * g.M + m) * g.A;
        if (g.d_bf16) {
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
            for (int q = 0; q < 4; ++q) d4[q] = make_float4(d[4 * q], d[4 * q + 1], d[4 * q + 2], d[4 * q + 3]);
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
        const float* gDa = g.gD + (long)(row0 + at) * g.M * g.A;
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
              if (g.A == 16) {
                const float4* g4 = reinterpret_cast<const float4*>(gDa + m * 16);
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
                for (int l = 0; l < 16; ++l) gd[l] = l < g.A ? gDa[m * g.A + l] : 0.f;
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
// Backward: dE/dT -> P -> per-neighbour dE/dr_ij -> forces and per-atom virial
// =============================================================================================
template <int NPASS, int NPAD>
__global__ void __launch_bounds__(kThreads, 1)
    k_mom_bwd(const __grid_constant__ CUtensorMap bhi, const __grid_constant__ CUtensorMap blo, const MomArgs g) {
  constexpr int PARTS = NPASS == 1 ? 1 : 2;
  constexpr int S = MomStages<NPASS>::value;
  constexpr int A_BYTES = 2 * kABlock;  // K = m in two 64-column blocks
  constexpr int B_KBLK = 64 * 128;      // 64 rows (8 intervals x 8 powers) x 128 B
  constexpr int B_STAGE = PARTS * 2 * B_KBLK;
  constexpr int KSTEPS = NPAD / 16;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char* As = smem;                      // PARTS x A_BYTES, dE/dT rows (A operand)
  unsigned char* ring = smem + PARTS * A_BYTES;  // B stages
  float* Ps = reinterpret_cast<float*>(ring + bwd_ring_bytes(NPASS));  // P of one block [atom][c][chunk][8]
  unsigned char* wins = ring + bwd_ring_bytes(NPASS) + kRowBufBytes;
  int* ex_s = reinterpret_cast<int*>(wins + kBwdWinBytes);  // [128] power-of-two scale of each dE/dT row
  uint64_t* bar = reinterpret_cast<uint64_t*>(ex_s + kRows);
  uint64_t* bfull = bar;
  uint64_t* bempty = bar + S;
  uint64_t* afull = bar + 2 * S;
  uint64_t* accfull = afull + 1;     // [2]
  uint64_t* accempty = accfull + 2;  // [2]
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(accempty + 2);
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
    mbar_init(afull, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accfull[b], 1);
      mbar_init(&accempty[b], kRows);
    }
    for (int t = 0; t < DP_MAX_TYPES; ++t) ghi[t] = -1;
    mbar_fence_init();
  }
  if (warp == 4) tmem_alloc(tmem_holder, 128);
  const int r = threadIdx.x;  // accumulator row (atom r / 4, component r % 4)
  const int c = r & 3;
  const int pb = row0 + lane;  // phase-2 walker: atom `lane`, phase `warp`
  const bool valid_b = warp < 4 && pb < row_end;
  const int ib = valid_b ? g.perm[pb] : 0;
  if (warp == 0) tile_groups(g, pb, ib, valid_b, ghi);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  int nch = 0;
  for (int t = 0; t < g.ntypes; ++t) nch += ghi[t] + 1;

  if (warp == 4) {
    if (lane == 0) {
      // ---- the A operand of this tile and its row scales ----
      mbar_expect_tx(afull, PARTS * A_BYTES + kRows * 4);
      bulk_load(As, g.gta + (long)blockIdx.x * PARTS * A_BYTES, PARTS * A_BYTES, afull);
      bulk_load(ex_s, g.gtx + (long)blockIdx.x * kRows, kRows * 4, afull);
      bool ok = true;
      // ---- phase 2: TMA producer and MMA issuer ----
      ok = mbar_wait(afull, 0, g.err);
      const uint32_t idesc = idesc_f16(kRows, 64, NPASS == 1 ? 0 : 1);
      auto issue = [&](int ch) {
        int t, grp;
        block_of(ch, ghi, g.ntypes, t, grp);
        const int s = ch % S;
        unsigned char* bs = ring + s * B_STAGE;
        mbar_expect_tx(&bfull[s], B_STAGE);
        const int y = ((ti * g.ntypes + t) * g.lcp + 8 * grp) * 8;
        tma_load_2d(bs, &bhi, &bfull[s], 0, y);
        tma_load_2d(bs + B_KBLK, &bhi, &bfull[s], 64, y);
        if (PARTS == 2) {
          tma_load_2d(bs + 2 * B_KBLK, &blo, &bfull[s], 0, y);
          tma_load_2d(bs + 3 * B_KBLK, &blo, &bfull[s], 64, y);
        }
      };
      int issued = 0, done = 0;
      if (ok)
        for (; issued < S - 1 && issued < nch; ++issued) issue(issued);
      for (int ch = 0; ok && ch < nch; ++ch) {
        const int s = ch % S, buf = ch & 1;
        if (!mbar_wait(&bfull[s], (ch / S) & 1, g.err)) {
          ok = false;
          break;
        }
        done = ch + 1;
        if (ch >= 2 && !mbar_wait(&accempty[buf], ((ch >> 1) - 1) & 1, g.err)) {
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
        const int kn = ch + S - 1;
        if (kn < nch) {
          if (kn >= S && !mbar_wait(&bempty[kn % S], ((kn / S) - 1) & 1, g.err)) {
            ok = false;
            break;
          }
          issue(kn);
          issued = kn + 1;
        }
      }
      for (int ch = done; ch < issued; ++ch) mbar_wait(&bfull[ch % S], (ch / S) & 1, g.err);
    }
  } else {
    // ---- the A operand (dE/dT rows, k_mom_gT) and the row scales arrive by bulk copy ----
    mbar_wait(afull, 0, g.err);

    // ---- phase 2, per 8-interval block: P from TMEM to shared memory, then every warp walks
    //      its phase of the 32 atoms' neighbours in the block ----
    const float pscale = ldexpf(g.inv_nc, ex_s[r]);
    float* prow = Ps + (r >> 2) * kAtomPitch + c * kRowPitch;  // this thread's P row
    const float* patom = Ps + lane * kAtomPitch;                // the walked atom's four rows
    Window win;
    win.e0 = reinterpret_cast<float4*>(wins) + r * 2 * kWin;
    win.e1 = reinterpret_cast<float4*>(wins) + (kRows + r) * 2 * kWin;
    win.j = reinterpret_cast<int*>(wins + 2 * kRows * 2 * kWin * 16) + r * 2 * kWin;
    Walk w;
    w.have = false;
    int cur_t = -1;
    bool dead = false;  // after a timed-out wait: stop waiting, keep taking part in the barriers
    float fi[3] = {0.f, 0.f, 0.f}, vir[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const uint32_t tb = tmem + ((uint32_t)(warp * 32) << 16);
    for (int ch = 0; ch < nch; ++ch) {
      const int buf = ch & 1;
      if (!dead && !mbar_wait(&accfull[buf], (ch >> 1) & 1, g.err)) dead = true;
      __syncwarp();  // tcgen05.ld is warp-collective
      tc_fence_after();
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float v[16];
        tmem_ld16(tb + (uint32_t)(buf * 64 + 16 * q), v);
#pragma unroll
        for (int e = 0; e < 16; e += 4)
          *reinterpret_cast<float4*>(prow + 16 * q + e) =
              make_float4(v[e] * pscale, v[e + 1] * pscale, v[e + 2] * pscale, v[e + 3] * pscale);
      }
      tc_fence_before();
      mbar_arrive(&accempty[buf]);
      bar_sync(1, kRows);  // the whole P block is in shared memory
      int t, grp;
      block_of(ch, ghi, g.ntypes, t, grp);
      if (t != cur_t) {
        cur_t = t;
        w.have = false;
        if (valid_b) {
          walk_start(g, pb, ib, win, w, g.sel_off[t] + warp, g.sel_off[t + 1]);
          walk_next(g, pb, ib, win, w);
        }
      }
      for (;;) {
        const bool act = w.have && w.l >= 8 * grp;
        if (!__any_sync(0xffffffffu, act)) break;
        if (act) {
          const int q = w.l - 8 * grp;
          const float tau = w.tau;
          float gR[4], dg[4];
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            const float4* p4 = reinterpret_cast<const float4*>(patom + cc * kRowPitch + (q & 7) * 8);
            const float4 x = p4[0], y = p4[1];
            gR[cc] = x.x + tau * (x.y + tau * (x.z + tau * (x.w + tau * (y.x + tau * y.y))));
            dg[cc] = x.y + tau * (2.f * x.z + tau * (3.f * x.w + tau * (4.f * y.x + tau * (5.f * y.y))));
          }
          const float s = w.e0.x, u0 = w.e0.y, u1 = w.e0.z, u2 = w.e0.w, ds = w.e1.x, rr = w.e1.y;
          const float invd = w.l < g.n1 ? g.inv1 : g.inv2;
          const float gs = s * (dg[0] + u0 * dg[1] + u1 * dg[2] + u2 * dg[3]) * invd;
          const float gvu = gR[1] * u0 + gR[2] * u1 + gR[3] * u2;
          const float A_ = ds * (gs + gR[0] + gvu), B_ = s / rr;
          const float gd[3] = {A_ * u0 + B_ * (gR[1] - gvu * u0), A_ * u1 + B_ * (gR[2] - gvu * u1),
                               A_ * u2 + B_ * (gR[3] - gvu * u2)};
          const float dv[3] = {rr * u0, rr * u1, rr * u2};
#pragma unroll
          for (int aa = 0; aa < 3; ++aa) {
            atomicAdd(g.force + 3 * w.j + aa, widen(-gd[aa]));
            fi[aa] += gd[aa];
#pragma unroll
            for (int bb = 0; bb < 3; ++bb) vir[aa * 3 + bb] -= gd[aa] * dv[bb];
          }
          walk_next(g, pb, ib, win, w);
        }
      }
      bar_sync(1, kRows);  // every walker is done with this P block
    }
    cp_async_wait0();
    // force on i and the atom's virial: the four phases' partial sums meet in shared memory
    float* red = Ps;  // [4 phases][32 atoms][12]
#pragma unroll
    for (int e = 0; e < 3; ++e) red[(warp * kAtoms + lane) * 12 + e] = fi[e];
#pragma unroll
    for (int e = 0; e < 9; ++e) red[(warp * kAtoms + lane) * 12 + 3 + e] = vir[e];
    bar_sync(1, kRows);
    if (warp == 0 && valid_b) {
      float tot[12];
#pragma unroll
      for (int e = 0; e < 12; ++e)
        tot[e] = red[lane * 12 + e] + red[(kAtoms + lane) * 12 + e] + red[(2 * kAtoms + lane) * 12 + e] +
                 red[(3 * kAtoms + lane) * 12 + e];
#pragma unroll
      for (int e = 0; e < 3; ++e) atomicAdd(g.force + 3 * ib + e, widen(tot[e]));
#pragma unroll
      for (int e = 0; e < 9; ++e) g.avir[9L * ib + e] = widen(tot[3 + e]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 4) tmem_dealloc(tmem, 128);
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

size_t fwd_smem(int npass, int npad) {
  const int S = 2;
  return (size_t)fwd_ring_bytes(npass, npad) + kFwdWinBytes + (2 * S + 1) * 8 + 4 +
         4 * DP_MAX_TYPES + 1024 + 64;
}
size_t bwd_smem(int npass, int npad, int M, int A) {
  const int parts = npass == 1 ? 1 : 2, S = 2;
  return (size_t)parts * 2 * kABlock + bwd_region(npass) + (2 * S + 5) * 8 + 4 + 4 * DP_MAX_TYPES + 1024 + 64;
}

template <int NPASS, int NPAD>
int launch_mom(const DeviceModel& m, const MomArgs& g, int tiles, int which, cudaStream_t st) {
  const CUtensorMap* maps = reinterpret_cast<const CUtensorMap*>(m.mom_maps.data());
  if (which == 1) {
    k_mom_gT<NPASS, NPAD><<<dim3(tiles, kAtoms / kGroupAtoms), kRows, 0, st>>>(g);
  } else if (which == 0) {
    const size_t sm = fwd_smem(NPASS, NPAD);
    DP_CUDA_TRY(cudaFuncSetAttribute(k_mom_fwd<NPASS, NPAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_mom_fwd<NPASS, NPAD><<<tiles, kThreads, sm, st>>>(maps[0], maps[1], g);
  } else {
    const size_t sm = bwd_smem(NPASS, NPAD, g.M, g.A);
    DP_CUDA_TRY(cudaFuncSetAttribute(k_mom_bwd<NPASS, NPAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_mom_bwd<NPASS, NPAD><<<tiles, kThreads, sm, st>>>(maps[2], maps[3], g);
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
  return m.compressed && (m.precision == DP_PREC_FP32 || m.precision == DP_PREC_BF16) && mom_npad_of(m.M) > 0 &&
         m.A <= 16 && (m.M * m.A) % 4 == 0;
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
  float* Tm = ar.get<float>(N * M * 4);
  void* D = bf16 ? (void*)ar.get<__nv_bfloat16>(N * M * A) : (void*)ar.get<float>(N * M * A);
  float4* envR = ar.get<float4>(N * pc.nc);
  float4* envU = ar.get<float4>(N * pc.nc);
  float4* envB = ar.get<float4>(N * pc.nc);
  const long max_tiles = (N + kAtoms - 1) / kAtoms + pc.ntypes;  // every type's last tile may be short
  unsigned char* gta = ar.get<unsigned char>(max_tiles * (bf16 ? 1 : 2) * 2 * kABlock);
  int* gtx = ar.get<int>(max_tiles * kRows);
  const float* gD = nullptr;
  if (ar.measure) {
    if (bf16) return run_fitting_tc(m, pc, reinterpret_cast<const __nv_bfloat16*>(D), io, ar, st, &gD);
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
  g.envR = envR;
  g.envU = envU;
  g.envB = envB;
  g.Tm = Tm;
  g.D = D;
  g.d_bf16 = bf16 ? 1 : 0;
  g.force = io.force;
  g.avir = io.atom_virial;
  g.gta = gta;
  g.gtx = gtx;
  char* stw = reinterpret_cast<char*>(io.status);
  g.table_range = reinterpret_cast<int*>(stw + offsetof(DevStatus, table_range));
  g.err = reinterpret_cast<int*>(stw + offsetof(DevStatus, timeout));
  {
    ProfScope _ps(io.prof, "env", st);
    const long tasks = N * pc.ntypes;  // one warp per (atom, neighbour type)
    k_env_mom<<<(unsigned)((tasks + 7) / 8), 256, 0, st>>>(pc, g, io.coord, io.nl_code, envR, envU, envB);
    DP_CUDA_TRY(cudaGetLastError());
  }
  if (tiles > 0) {
    ProfScope _ps(io.prof, "mom_fwd", st);
    const int rc = bf16 ? launch_mom_np<1>(m, g, tiles, 0, st) : launch_mom_np<3>(m, g, tiles, 0, st);
    if (rc != DP_OK) return rc;
  }
  int rc;
  if (bf16)
    rc = run_fitting_tc(m, pc, reinterpret_cast<const __nv_bfloat16*>(D), io, ar, st, &gD);
  else
    rc = run_fitting<float>(m, pc, m.p32, reinterpret_cast<const float*>(D), io, ar, st, &gD);
  if (rc != DP_OK) return rc;
  g.gD = gD;
  if (tiles > 0) {
    {
      ProfScope _ps(io.prof, "mom_gT", st);
      rc = bf16 ? launch_mom_np<1>(m, g, tiles, 1, st) : launch_mom_np<3>(m, g, tiles, 1, st);
      if (rc != DP_OK) return rc;
    }
    ProfScope _ps(io.prof, "mom_bwd", st);
    rc = bf16 ? launch_mom_np<1>(m, g, tiles, 2, st) : launch_mom_np<3>(m, g, tiles, 2, st);
    if (rc != DP_OK) return rc;
  }
  return DP_OK;
}

}  // namespace dpgb
