// Fitting net F_0^{a_i} (Eq. (fitting_energy), layers of Eq. (NN)) and its input gradient on
// tensor cores: BF16 operands, FP32 accumulation, one tcgen05 GEMM launch per layer and
// direction covering all atom types.
//
//   forward  hidden layer l   y_l = tanh(y_{l-1} W_l + b_l) (+ skip)      TC_EPI_FWD
//            last hidden      ... and E_i = y . w_out + b_out, gz = w_out (1 - t^2)
//                                                                            TC_EPI_FWD_LAST
//   backward layer l >= 1     gy_{l-1} = gz_l W_l^T + skip^T(gy_l),
//                             gz_{l-1} = gy_{l-1} (1 - t_{l-1}^2)           TC_EPI_BWD
//   backward layer 0          dE/dD = gz_0 W_0^T                           TC_EPI_PLAIN
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "fit_tc.cuh"
#include "tc_gemm.cuh"

namespace dpgb {

namespace {

uint16_t bf16_bits_rne(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7F800000u) == 0x7F800000u) return (uint16_t)(u >> 16);  // inf / nan
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

int skip_kind(int n_in, int n_out) { return n_out == n_in ? 1 : (n_out == 2 * n_in ? 2 : 0); }

}  // namespace

// Tensor map of fitting layer l of type t: dir 0 the forward B operand W^T [n_out][n_in], dir 1
// the backward one W [n_in][n_out]; box of 64 columns x box_rows rows; cached on the model.
const CUtensorMap* fit_weight_map(const DeviceModel& m, int t, int l, int dir, int box_rows, bool lo) {
  const long key = ((((long)t * 64 + l) * 2 + dir) * 1024 + box_rows) * 2 + (lo ? 1 : 0);
  for (auto& kv : m.tmap_cache)
    if (kv.first == key) return reinterpret_cast<const CUtensorMap*>(kv.second.data());
  const int nfl = m.n_fit_layers;
  const LayerDesc& L = m.fit[(size_t)t * nfl + l];
  const long off = m.fit_bf16_off[(size_t)t * (nfl - 1) + l];
  std::vector<unsigned char> buf(sizeof(CUtensorMap));
  CUtensorMap* map = reinterpret_cast<CUtensorMap*>(buf.data());
  int rc;
  const void* wt = lo ? m.fit_wt_bf16_lo : m.fit_wt_bf16;
  const void* w = lo ? m.fit_w_bf16_lo : m.fit_w_bf16;
  if (!wt || !w) {
    set_error("fitting weights: low halves were not prepared for this model");
    return nullptr;
  }
  if (dir == 0)  // forward B^T = W^T [n_out][n_in]
    rc = make_tmap_bf16(map, static_cast<const __nv_bfloat16*>(wt) + off, L.n_out, L.n_in, box_rows);
  else  // backward B^T = W [n_in][n_out]
    rc = make_tmap_bf16(map, static_cast<const __nv_bfloat16*>(w) + off, L.n_in, L.n_out, box_rows);
  if (rc != DP_OK) return nullptr;
  m.tmap_cache.emplace_back(key, std::move(buf));
  return reinterpret_cast<const CUtensorMap*>(m.tmap_cache.back().second.data());
}

bool fit_tc_supported(const DeviceModel& m) {
  const int nfl = m.n_fit_layers, nh = nfl - 1;
  if (nh < 1) return false;
  for (int t = 0; t < m.cfg.ntypes; ++t)
    for (int l = 0; l < nh; ++l) {
      const LayerDesc& L = m.fit[(size_t)t * nfl + l];
      if (L.n_in % 8 || L.n_out % 16 || L.n_out > 256 || (l == 0 && L.skip) || L.skip == 2) return false;
    }
  return true;
}

int prepare_fit_bf16(DeviceModel& m, const double* params_host, bool split) {
  const int nfl = m.n_fit_layers, nh = nfl - 1;
  if (!fit_tc_supported(m)) {
    set_error("tensor-core fitting needs at least one hidden layer, hidden widths that are multiples of 16 and "
              "<= 256, inputs multiple of 8, skips of kind 0 or 1");
    return DP_E_UNSUPPORTED;
  }
  long total = 0;
  m.fit_bf16_off.assign((size_t)m.cfg.ntypes * nh, 0);
  for (int t = 0; t < m.cfg.ntypes; ++t)
    for (int l = 0; l < nh; ++l) {
      const LayerDesc& L = m.fit[(size_t)t * nfl + l];
      m.fit_bf16_off[(size_t)t * nh + l] = total;
      total += ((long)L.n_in * L.n_out + 7) / 8 * 8;
    }
  std::vector<uint16_t> wt((size_t)total), w((size_t)total), wtl, wl;
  if (split) {
    wtl.assign((size_t)total, 0);
    wl.assign((size_t)total, 0);
  }
  for (int t = 0; t < m.cfg.ntypes; ++t)
    for (int l = 0; l < nh; ++l) {
      const LayerDesc& L = m.fit[(size_t)t * nfl + l];
      const long off = m.fit_bf16_off[(size_t)t * nh + l];
      const double* W = params_host + L.w_off;
      for (int i = 0; i < L.n_in; ++i)
        for (int o = 0; o < L.n_out; ++o) {
          const float x = (float)W[(long)i * L.n_out + o];
          const uint16_t b = bf16_bits_rne(x);
          w[off + (long)i * L.n_out + o] = b;
          wt[off + (long)o * L.n_in + i] = b;
          if (split) {  // low half: the remainder x - hi, rounded to BF16
            const uint32_t hb = (uint32_t)b << 16;
            float hi;
            std::memcpy(&hi, &hb, 4);
            const uint16_t bl = bf16_bits_rne(x - hi);
            wl[off + (long)i * L.n_out + o] = bl;
            wtl[off + (long)o * L.n_in + i] = bl;
          }
        }
    }
  DP_CUDA_TRY(cudaMalloc(&m.fit_wt_bf16, sizeof(uint16_t) * total));
  DP_CUDA_TRY(cudaMalloc(&m.fit_w_bf16, sizeof(uint16_t) * total));
  DP_CUDA_TRY(cudaMemcpy(m.fit_wt_bf16, wt.data(), sizeof(uint16_t) * total, cudaMemcpyHostToDevice));
  DP_CUDA_TRY(cudaMemcpy(m.fit_w_bf16, w.data(), sizeof(uint16_t) * total, cudaMemcpyHostToDevice));
  if (split) {
    DP_CUDA_TRY(cudaMalloc(&m.fit_wt_bf16_lo, sizeof(uint16_t) * total));
    DP_CUDA_TRY(cudaMalloc(&m.fit_w_bf16_lo, sizeof(uint16_t) * total));
    DP_CUDA_TRY(cudaMemcpy(m.fit_wt_bf16_lo, wtl.data(), sizeof(uint16_t) * total, cudaMemcpyHostToDevice));
    DP_CUDA_TRY(cudaMemcpy(m.fit_w_bf16_lo, wl.data(), sizeof(uint16_t) * total, cudaMemcpyHostToDevice));
  }
  return DP_OK;
}

int run_fitting_tc(const DeviceModel& m, const PathConst& pc, const __nv_bfloat16* Dbf, const PathIO& io, Arena& ar,
                   cudaStream_t st, const float** gD_out, const __nv_bfloat16** gDh_out, const __nv_bfloat16* Dlo,
                   const float* Tm, float* gT) {
  const bool split = Dlo != nullptr;
  if (!split && gDh_out && fit_fused_supported(m)) {  // the whole net in one kernel per tile
    *gD_out = nullptr;
    return run_fitting_fused(m, pc, Dbf, io, ar, st, gDh_out);
  }
  // the fused kernel runs one CTA per 128-atom tile through the whole chain: it pays off once the
  // tiles fill half the SMs; smaller batches spread each layer over more CTAs with per-layer launches
  if (split && fit_split_supported(m)) {
    long tiles = 0;
    for (int t = 0; t < pc.ntypes; ++t) tiles += (io.type_start[t + 1] - io.type_start[t] + 127) / 128;
    if (2 * tiles >= sm_count()) return run_fitting_split(m, pc, Dbf, Dlo, io, ar, st, gD_out, Tm, gT);
  }
  if (split) gDh_out = nullptr;  // split operands: dE/dD in FP32
  const long N = pc.natoms;
  const int nfl = m.n_fit_layers, nh = nfl - 1;
  const int D = pc.M * pc.A;
  const int nt = pc.ntypes;
  // ---- scratch ----
  std::vector<float*> Yf(nh), T(nh), gY(nh);
  std::vector<__nv_bfloat16*> Yb(nh), gZ(nh), Ybl(nh, nullptr), gZl(nh, nullptr);
  for (int l = 0; l < nh; ++l) {
    const int w = m.fit[l].n_out;
    Yf[l] = ar.get<float>(N * w);
    Yb[l] = ar.get<__nv_bfloat16>(N * w);
    T[l] = ar.get<float>(N * w);
    gY[l] = ar.get<float>(N * w);
    gZ[l] = ar.get<__nv_bfloat16>(N * w);
    if (split) {
      Ybl[l] = ar.get<__nv_bfloat16>(N * w);
      gZl[l] = ar.get<__nv_bfloat16>(N * w);
    }
  }
  // per-atom energy partials, one per output-column block of the last hidden layer (blocks are at
  // least 64 columns wide)
  float* E = ar.get<float>(N * ((m.fit[nh - 1].n_out + 63) / 64));
  float* gD = gDh_out ? nullptr : ar.get<float>(N * D);
  __nv_bfloat16* gDh = gDh_out ? ar.get<__nv_bfloat16>(N * D) : nullptr;
  if (ar.measure) return DP_OK;
  if (!ar.ok()) {
    set_error("scratch allocation failed");
    return DP_E_OOM;
  }
  TcArgs base;
  std::memset(&base, 0, sizeof(base));
  base.ntypes = nt;
  int tiles = 0;
  for (int t = 0; t <= nt; ++t) {
    base.row_start[t] = io.type_start[t];
    base.tile_start[t] = tiles;
    if (t < nt) tiles += (io.type_start[t + 1] - io.type_start[t] + 127) / 128;
  }
  base.err = &io.status->timeout;  // bounded waits that give up are reported by the call
  const float* p32 = m.p32;
  // the staged epilogues hold at most 128 output columns per CTA; split operands take 64 (two
  // CTAs of 97 KB share an SM)
  auto pick_bn = [&](int n, bool staged) {
    const int bn = tc_pick_bn(n, tiles);
    return split ? std::min(bn, 64) : (staged ? std::min(bn, 128) : bn);
  };
  // A operand (high part, and the low part when split) and the type's weight maps
  auto maps = [&](const void* A_hi, const void* A_lo, int K, int l, int dir, int BN, CUtensorMap& ta, TcMaps& tb,
                  TcLo& lo) -> int {
    int rc = make_tmap_bf16(&ta, A_hi, N, K, 128);
    if (rc == DP_OK && split) rc = make_tmap_bf16(&lo.a, A_lo, N, K, 128);
    if (rc != DP_OK) return rc;
    for (int t = 0; t < nt; ++t) {
      const CUtensorMap* wm = fit_weight_map(m, t, l, dir, BN);
      if (!wm) return DP_E_CUDA;
      tb.m[t] = *wm;
      if (split) {
        const CUtensorMap* wl = fit_weight_map(m, t, l, dir, BN, true);
        if (!wl) return DP_E_CUDA;
        lo.b.m[t] = *wl;
      }
    }
    return DP_OK;
  };
  // ---- forward ----
  for (int l = 0; l < nh; ++l) {
    const LayerDesc& L0 = m.fit[l];
    const bool last = (l == nh - 1);
    TcArgs a = base;
    a.K = L0.n_in;
    a.N = L0.n_out;
    a.BN = pick_bn(a.N, true);
    CUtensorMap ta;
    TcMaps tb;
    TcLo lo;
    std::memset(&lo, 0, sizeof(lo));
    int rc = maps(l == 0 ? (const void*)Dbf : (const void*)Yb[l - 1], l == 0 ? (const void*)Dlo : (const void*)Ybl[l - 1],
                  a.K, l, 0, a.BN, ta, tb, lo);
    if (rc != DP_OK) return rc;
    for (int t = 0; t < nt; ++t) {
      const LayerDesc& L = m.fit[(size_t)t * nfl + l];
      a.bias[t] = p32 + L.w_off + (long)L.n_in * L.n_out;
      if (last) {
        const LayerDesc& Lo = m.fit[(size_t)t * nfl + nh];
        a.w_last[t] = p32 + Lo.w_off;
        a.b_last[t] = m.fit_out_bias[t];
      }
    }
    a.skip_kind = L0.skip;
    a.skip_mat = l > 0 ? Yf[l - 1] : nullptr;
    a.skip_ld = a.K;
    if (!last) {
      a.out_f32 = Yf[l];
      a.out_bf16 = Yb[l];
      a.out_bf16_lo = Ybl[l];
      a.out_t = T[l];
    } else {
      a.out_bf16 = gZ[l];
      a.out_bf16_lo = gZl[l];
      a.e_out = E;
      a.e_ld = N;
    }
    ProfScope _ps(io.prof, last ? "fit_fwd_last_tc" : "fit_fwd_tc", st);
    DP_CUDA_TRY(launch_tc_gemm(last ? TC_EPI_FWD_LAST : TC_EPI_FWD, ta, tb, a, st, split ? &lo : nullptr));
  }
  {
    ProfScope _ps(io.prof, "energy_sum", st);
    const int bn = pick_bn(m.fit[nh - 1].n_out, true);
    DP_CUDA_TRY(launch_energy_f32(E, (m.fit[nh - 1].n_out + bn - 1) / bn, io.perm, (int)N, io.atom_energy, st));
  }
  // ---- backward ----
  for (int l = nh - 1; l >= 0; --l) {
    const LayerDesc& L0 = m.fit[l];
    TcArgs a = base;
    a.K = L0.n_out;
    a.N = L0.n_in;
    a.BN = pick_bn(a.N, l > 0);
    CUtensorMap ta;
    TcMaps tb;
    TcLo lo;
    std::memset(&lo, 0, sizeof(lo));
    int rc = maps(gZ[l], gZl[l], a.K, l, 1, a.BN, ta, tb, lo);
    if (rc != DP_OK) return rc;
    for (int t = 0; t < nt; ++t) {
      const LayerDesc& Lo = m.fit[(size_t)t * nfl + nh];
      a.w_last[t] = p32 + Lo.w_off;
    }
    if (l == 0) {
      a.out_f32 = gD;
      a.out_bf16 = gDh;
      ProfScope _ps(io.prof, "fit_bwd_tc", st);
      DP_CUDA_TRY(launch_tc_gemm(TC_EPI_PLAIN, ta, tb, a, st, split ? &lo : nullptr));
    } else {
      a.skip_kind = L0.skip;
      a.skip_vec = (l == nh - 1) ? 1 : 0;
      a.skip_mat = (l == nh - 1) ? nullptr : gY[l];
      a.skip_ld = a.K;
      a.tact = T[l - 1];
      a.out_f32 = m.fit[l - 1].skip ? gY[l - 1] : nullptr;
      a.out_bf16 = gZ[l - 1];
      a.out_bf16_lo = gZl[l - 1];
      ProfScope _ps(io.prof, "fit_bwd_tc", st);
      DP_CUDA_TRY(launch_tc_gemm(TC_EPI_BWD, ta, tb, a, st, split ? &lo : nullptr));
    }
  }
  *gD_out = gD;
  if (gDh_out) *gDh_out = gDh;
  (void)skip_kind;
  return DP_OK;
}

}  // namespace dpgb
