// Plain FP64 CPU oracle for the Deep Potential energy / force / virial path (descriptors
// se_e2_a, se_e2_r, se_e3 and the hybrids of se_e2_a with either), and the derivative of the
// training loss along a parameter direction.
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
// cpu_baseline leg (and its --impl reference arm) load this library.  The product path
// (the CUDA library behind include/dpgb.h) never links, calls or reads anything here,
// and nothing here is shared with it.
//
// Everything is written straight from the DeePMD-kit v2 paper (arXiv 2304.09409):
//   Eq. (model)      y_i = F(D(x_i, {x_j})),  E = sum_i E_i                 Sec. II.A
//   Eq. (rij)        R_j = (s, s x/r, s y/r, s z/r),  r_ij = r_j - r_i     Sec. II.A.1
//   Eq. (switch)     s(r)                                                  Sec. II.A.1
//   Eq. (G2)         G_j = N_{e,2}^{a_i,a_j}(s(r_ij))                      Sec. II.A.1
//   se_e2_a          D = (1/Nc^2) G^T R R^T G_<                            Sec. II.A.1
//   se_e2_r          D = (1/Nc) G^T s  (R reduced to its radial column)    Sec. II.A.1
//   se_e3            D = (1/Nc^2) sum_jk theta_jk G(theta_jk), theta = R_j . R_k   Sec. II.A.1
//   hybrid           D = the two descriptors concatenated                  Sec. II.A.1
//   Eq. (fitting)    E_i = F_0^{a_i}(D^i)                                  Sec. II.A.2
//   force / virial   F = -dE/dr,  Xi = -sum_g dE/dh_{g a} h_{g b}           Sec. II.A.2
//   Eq. (NN)         layer y = phi(x w + b) (+ x | + {x,x})                Sec. II.A.6
//   Eq. (compress)   quintic tabulation of the embedding net               Sec. II.A.6
//   neighbour order  by (type, distance, index)                            Sec. III.B.1
//   Eq. (loss)       pE dE^2/N + pF |dF|^2/(3N) + pXi |dXi|^2/(9N)         Sec. II.B
//
// Readings of the paper used here (where it is silent or ambiguous):
//   * Nc in 1/Nc^2 is the padded sum of sel; padded rows of R are zero.
//   * The virial is dE/dh at fixed fractional coordinates, which equals
//     Xi_ab = -sum_{pairs} (dE/d r_ij)_a (r_ij)_b.
//   * Neighbour order is the exact total order (type, r^2 as IEEE bits, j, image shift);
//     a pair displacement is (x_j + t) - x_i with t = n0 h0 + n1 h1 + n2 h2 evaluated
//     left to right without fused multiply-add (build flag -ffp-contract=off).
//   * ResNet timestep w_hat = 1; the last fitting layer (width 1) is linear.
//   * Quintic pieces are evaluated at t = x - x_l (the offset inside the interval).
//   * se_e2_r keeps s(r) as the weight of each row (the radial column of R), so a neighbour's
//     term vanishes smoothly at r_c and padded rows contribute nothing; its 1/Nc is that of the
//     contraction G^T R with one column.
//   * se_e3: theta_jk over all four columns of R, j = k included; nets indexed a_j * ntypes + a_k
//     (ntypes^2 nets whatever type_one_side says).
//   * A hybrid descriptor's parts each have their own r_c, r_s, sel and embedding nets and share the
//     net index rule (type_one_side); they read one neighbour list built with the larger cutoff and,
//     per type, the larger sel, of which each part takes the entries inside its own r_c and sel;
//     the se_e2_a block comes first.
//
// Forces come from a hand-written reverse pass in plain loops.  A second, independent
// mechanism -- forward-mode dual numbers through a templated energy -- exists only to
// pin that reverse pass (orc_energy_dual).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

struct OrcConfig {
  int ntypes;
  int sel[8];
  double rcut;
  double rcut_smth;
  int n_embed;
  int embed[8];
  int axis;
  int n_fit;
  int fit[8];
  int type_one_side;
  // 0 se_e2_a; 1 se_e2_r; 2 hybrid se_e2_a + se_e2_r; 3 se_e3; 4 hybrid se_e2_a + se_e3
  int descriptor;
  // hybrids: the second part's cutoffs, sel and embedding widths
  double rcut_2, rcut_smth_2;
  int sel_2[8];
  int n_embed_2;
  int embed_2[8];
};

}  // extern "C"

namespace {

// ------------------------------------------------------------------------------------------
// Scalar types: double, first-order dual, and second-order jet (value, d1, d2) used for the
// table nodes (y, y', y'') and for pins.
// ------------------------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual(double a = 0.0, double b = 0.0) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) { return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
inline bool operator<(Dual a, Dual b) { return a.v < b.v; }
inline bool operator>=(Dual a, Dual b) { return a.v >= b.v; }
inline Dual dsqrt(Dual a) { double s = std::sqrt(a.v); return Dual(s, a.d / (2.0 * s)); }
inline Dual dtanh(Dual a) { double t = std::tanh(a.v); return Dual(t, (1.0 - t * t) * a.d); }
inline double val(Dual a) { return a.v; }

inline double dsqrt(double a) { return std::sqrt(a); }
inline double dtanh(double a) { return std::tanh(a); }
inline double val(double a) { return a; }

struct Jet {  // f, f', f'' along one input direction
  double v, d1, d2;
  Jet(double a = 0.0, double b = 0.0, double c = 0.0) : v(a), d1(b), d2(c) {}
};
inline Jet operator+(Jet a, Jet b) { return Jet(a.v + b.v, a.d1 + b.d1, a.d2 + b.d2); }
inline Jet operator*(Jet a, double w) { return Jet(a.v * w, a.d1 * w, a.d2 * w); }
inline Jet jtanh(Jet a) {
  double t = std::tanh(a.v), g = 1.0 - t * t;
  return Jet(t, g * a.d1, g * a.d2 - 2.0 * t * g * a.d1 * a.d1);
}

// Hyper-dual number v + a e1 + b e2 + ab e1 e2 (e1^2 = e2^2 = 0): the e1 e2 part of f(x) is an
// exact mixed second derivative.  Used with e1 along a coordinate direction and e2 along a
// parameter direction to differentiate the force term of the loss with respect to parameters.
struct HD {
  double v, a, b, ab;
  HD(double x = 0.0, double p = 0.0, double q = 0.0, double r = 0.0) : v(x), a(p), b(q), ab(r) {}
};
inline HD operator+(HD x, HD y) { return HD(x.v + y.v, x.a + y.a, x.b + y.b, x.ab + y.ab); }
inline HD operator-(HD x, HD y) { return HD(x.v - y.v, x.a - y.a, x.b - y.b, x.ab - y.ab); }
inline HD operator*(HD x, HD y) {
  return HD(x.v * y.v, x.a * y.v + x.v * y.a, x.b * y.v + x.v * y.b, x.ab * y.v + x.a * y.b + x.b * y.a + x.v * y.ab);
}
// f applied to x given f(v), f'(v), f''(v)
inline HD hd_apply(HD x, double f, double f1, double f2) {
  return HD(f, f1 * x.a, f1 * x.b, f1 * x.ab + f2 * x.a * x.b);
}
inline HD operator/(HD x, HD y) {
  const double iv = 1.0 / y.v;
  return x * hd_apply(y, iv, -iv * iv, 2.0 * iv * iv * iv);
}
inline bool operator<(HD x, HD y) { return x.v < y.v; }
inline double val(HD x) { return x.v; }
inline HD dsqrt(HD x) {
  const double s = std::sqrt(x.v);
  return hd_apply(x, s, 0.5 / s, -0.25 / (s * x.v));
}
inline HD dtanh(HD x) {
  const double t = std::tanh(x.v), g = 1.0 - t * t;
  return hd_apply(x, t, g, -2.0 * t * g);
}

// ------------------------------------------------------------------------------------------
// Parameter layout helpers (flat FP64 array, see the inputs module)
// ------------------------------------------------------------------------------------------
// One family of embedding nets: per net (in net-index order), layer by layer.
struct NetSet {
  int nl = 0, m = 0;          // layers, output width
  std::vector<int> in, out;   // layer shapes
  std::vector<long> off;      // per net, per layer: offset of W (b follows W)
};

// One descriptor part (Sec. II.A.1): se_e2_a (A), se_e2_r (R) or se_e3 (E3), with its own
// cutoffs, sel and embedding nets, writing the block [doff, doff + dwid) of D.
enum { PART_A = 0, PART_R = 1, PART_E3 = 2 };
struct Part {
  int kind;
  double rc, rs;
  int sel[8], sel_off[9], nc;
  NetSet nets;
  int axis;        // A: M_<
  int doff, dwid;
};

struct Layout {
  int ntypes;
  // the neighbour list every part reads: cutoff and per-type sizes of the widest part
  double lrc;
  int lsel[8];
  int nc, sel_off[9];
  std::vector<Part> parts;
  int dw;                      // width of D
  // first part's nets (tables and jets are built for these)
  NetSet e1;
  int m, axis, n_embed_nets;
  std::vector<int> fin, fout;  // fitting layer shapes (last has fout = 1)
  std::vector<long> foff;      // per fitting net, per layer
  long n_params;
};

void add_nets(NetSet& S, int nl, const int* widths, int nnets, long& off) {
  S.nl = nl;
  S.m = widths[nl - 1];
  int prev = 1;
  for (int l = 0; l < nl; ++l) { S.in.push_back(prev); S.out.push_back(widths[l]); prev = widths[l]; }
  for (int n = 0; n < nnets; ++n)
    for (int l = 0; l < nl; ++l) { S.off.push_back(off); off += (long)S.in[l] * S.out[l] + S.out[l]; }
}

Part make_part(const OrcConfig& c, int kind, double rc, double rs, const int* sel, int nl, const int* widths,
               long& off) {
  Part P;
  P.kind = kind;
  P.rc = rc;
  P.rs = rs;
  P.nc = 0;
  for (int t = 0; t < c.ntypes; ++t) { P.sel[t] = sel[t]; P.sel_off[t] = P.nc; P.nc += sel[t]; }
  P.sel_off[c.ntypes] = P.nc;
  // se_e3 nets are indexed by the two neighbours' types; the two-body nets by (a_i, a_j) or a_j
  const int nnets = (kind == PART_E3 || !c.type_one_side) ? c.ntypes * c.ntypes : c.ntypes;
  add_nets(P.nets, nl, widths, nnets, off);
  P.axis = kind == PART_A ? c.axis : 0;
  P.dwid = kind == PART_A ? P.nets.m * c.axis : P.nets.m;
  return P;
}

// Sec. II.A.1: se_e2_a gives D = T T_<^T (M x M_<); se_e2_r, with only the radial column s of R,
// gives D = G^T s / N_c (M values); se_e3 gives D = (R R^T) : G / N_c^2 (M values); a hybrid
// descriptor is the concatenation of its parts.
Layout make_layout(const OrcConfig& c) {
  Layout L;
  L.ntypes = c.ntypes;
  long off = 0;
  const int d = c.descriptor;
  const int k1 = (d == 1) ? PART_R : (d == 3 ? PART_E3 : PART_A);
  L.parts.push_back(make_part(c, k1, c.rcut, c.rcut_smth, c.sel, c.n_embed, c.embed, off));
  if (d == 2 || d == 4)
    L.parts.push_back(make_part(c, d == 2 ? PART_R : PART_E3, c.rcut_2, c.rcut_smth_2, c.sel_2, c.n_embed_2,
                                c.embed_2, off));
  L.lrc = 0.0;
  for (int t = 0; t < c.ntypes; ++t) L.lsel[t] = 0;
  L.dw = 0;
  for (Part& P : L.parts) {
    L.lrc = std::max(L.lrc, P.rc);
    for (int t = 0; t < c.ntypes; ++t) L.lsel[t] = std::max(L.lsel[t], P.sel[t]);
    P.doff = L.dw;
    L.dw += P.dwid;
  }
  L.nc = 0;
  for (int t = 0; t < c.ntypes; ++t) { L.sel_off[t] = L.nc; L.nc += L.lsel[t]; }
  L.sel_off[c.ntypes] = L.nc;
  L.e1 = L.parts[0].nets;
  L.m = L.e1.m;
  L.axis = c.axis;
  L.n_embed_nets = (int)(L.e1.off.size() / std::max(1, L.e1.nl));
  int prev = L.dw;
  for (int l = 0; l < c.n_fit; ++l) { L.fin.push_back(prev); L.fout.push_back(c.fit[l]); prev = c.fit[l]; }
  L.fin.push_back(prev); L.fout.push_back(1);
  for (int n = 0; n < c.ntypes; ++n)
    for (size_t l = 0; l < L.fin.size(); ++l) { L.foff.push_back(off); off += (long)L.fin[l] * L.fout[l] + L.fout[l]; }
  L.n_params = off;
  return L;
}

// The list geometry widened to n entries per type (every atom within the list cutoff).
Layout widened(Layout L, int n) {
  L.nc = 0;
  for (int t = 0; t < L.ntypes; ++t) { L.lsel[t] = n; L.sel_off[t] = L.nc; L.nc += n; }
  L.sel_off[L.ntypes] = L.nc;
  return L;
}

inline int embed_net_index(const OrcConfig& c, int ai, int aj) {
  return c.type_one_side ? aj : ai * c.ntypes + aj;
}

// Eq. (NN): the skip term of a layer with n_in inputs and n_out outputs (ResNet on).
//   n_out == n_in   : + x
//   n_out == 2 n_in : + {x, x}
//   otherwise       : none
inline int skip_kind(int n_in, int n_out) { return n_out == n_in ? 1 : (n_out == 2 * n_in ? 2 : 0); }

// ------------------------------------------------------------------------------------------
// Eq. (switch) and its derivative ds/dr
// ------------------------------------------------------------------------------------------
template <class T>
T switch_fn(T r, double rs, double rc) {
  if (val(r) < rs) return T(1.0) / r;
  if (val(r) >= rc) return T(0.0);
  T x = (r - T(rs)) / T(rc - rs);
  T poly = x * x * x * (T(-6.0) * x * x + T(15.0) * x - T(10.0)) + T(1.0);
  return poly / r;
}

double switch_deriv(double r, double rs, double rc) {
  if (r < rs) return -1.0 / (r * r);
  if (r >= rc) return 0.0;
  double x = (r - rs) / (rc - rs);
  double u = x * x * x * (-6.0 * x * x + 15.0 * x - 10.0) + 1.0;
  double du = -30.0 * x * x * (x - 1.0) * (x - 1.0) / (rc - rs);
  return -u / (r * r) + du / r;
}

// ------------------------------------------------------------------------------------------
// Dense layer, Eq. (NN), generic scalar
// ------------------------------------------------------------------------------------------
template <class T, class P>
void layer_forward(const P* W, const P* b, int n_in, int n_out, const T* x, T* y, bool tanh_act, bool resnet) {
  int sk = resnet ? skip_kind(n_in, n_out) : 0;
  for (int o = 0; o < n_out; ++o) {
    T z = T(b[o]);
    for (int i = 0; i < n_in; ++i) z = z + x[i] * T(W[(long)i * n_out + o]);
    T a = tanh_act ? dtanh(z) : z;
    if (sk == 1) a = a + x[o];
    if (sk == 2) a = a + x[o % n_in];
    y[o] = a;
  }
}

// ------------------------------------------------------------------------------------------
// Neighbour list: brute force over all atoms and all periodic images (Sec. III.B.1 order)
// ------------------------------------------------------------------------------------------
struct Cand {
  int type;
  uint64_t r2bits;
  int j;
  int code;
};
inline bool cand_less(const Cand& a, const Cand& b) {
  if (a.type != b.type) return a.type < b.type;
  if (a.r2bits != b.r2bits) return a.r2bits < b.r2bits;
  if (a.j != b.j) return a.j < b.j;
  return (unsigned)a.code < (unsigned)b.code;
}
inline int pack_shift(int n0, int n1, int n2) { return ((n0 + 512) << 20) | ((n1 + 512) << 10) | (n2 + 512); }
inline void unpack_shift(int code, int* n) {
  n[0] = ((code >> 20) & 1023) - 512;
  n[1] = ((code >> 10) & 1023) - 512;
  n[2] = (code & 1023) - 512;
}

// Pair displacement (x_j + t) - x_i, t = n0 h0 + n1 h1 + n2 h2, left to right.
inline void pair_disp(const double* xi, const double* xj, const int* n, const double* box, double* d) {
  for (int a = 0; a < 3; ++a) {
    double t = 0.0;
    if (box) t = ((double)n[0] * box[0 * 3 + a] + (double)n[1] * box[1 * 3 + a]) + (double)n[2] * box[2 * 3 + a];
    double p = xj[a] + t;
    d[a] = p - xi[a];
  }
}
inline double norm2(const double* d) { return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]; }

void inverse3(const double* h, double* inv) {
  double c00 = h[4] * h[8] - h[5] * h[7], c01 = h[5] * h[6] - h[3] * h[8], c02 = h[3] * h[7] - h[4] * h[6];
  double det = h[0] * c00 + h[1] * c01 + h[2] * c02;
  inv[0] = c00 / det; inv[1] = (h[2] * h[7] - h[1] * h[8]) / det; inv[2] = (h[1] * h[5] - h[2] * h[4]) / det;
  inv[3] = c01 / det; inv[4] = (h[0] * h[8] - h[2] * h[6]) / det; inv[5] = (h[2] * h[3] - h[0] * h[5]) / det;
  inv[6] = c02 / det; inv[7] = (h[1] * h[6] - h[0] * h[7]) / det; inv[8] = (h[0] * h[4] - h[1] * h[3]) / det;
}

// Returns the number of (atom, type) blocks whose candidate count exceeded sel.
int build_nlist(const OrcConfig& c, const Layout& L, int N, const double* coord, const int* type, const double* box,
                int* nl_j, int* nl_code, int* counts /*[N*ntypes] or null*/) {
  const double rc2 = L.lrc * L.lrc;
  std::vector<int> lo(3 * N, 0), hi(3 * N, 0);
  int K[3] = {0, 0, 0};
  std::vector<long> m(3 * (size_t)N, 0);
  if (box) {
    double inv[9];
    inverse3(box, inv);
    double vol = std::fabs(box[0] * (box[4] * box[8] - box[5] * box[7]) - box[1] * (box[3] * box[8] - box[5] * box[6]) +
                           box[2] * (box[3] * box[7] - box[4] * box[6]));
    for (int d = 0; d < 3; ++d) {
      const double* u = box + 3 * ((d + 1) % 3);
      const double* v = box + 3 * ((d + 2) % 3);
      double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
      double width = vol / std::sqrt(cx * cx + cy * cy + cz * cz);
      K[d] = (int)std::ceil(L.lrc / width) + 1;
    }
    for (int i = 0; i < N; ++i)
      for (int d = 0; d < 3; ++d) {
        double f = coord[3 * i + 0] * inv[0 * 3 + d] + coord[3 * i + 1] * inv[1 * 3 + d] + coord[3 * i + 2] * inv[2 * 3 + d];
        m[3 * i + d] = (long)std::floor(f);
      }
  }
  int overflow = 0;
  std::vector<Cand> cand;
  for (int i = 0; i < N; ++i) {
    cand.clear();
    for (int j = 0; j < N; ++j) {
      int base[3] = {0, 0, 0};
      if (box)
        for (int d = 0; d < 3; ++d) base[d] = (int)(m[3 * i + d] - m[3 * j + d]);
      int n[3];
      for (n[0] = base[0] - K[0]; n[0] <= base[0] + K[0]; ++n[0])
        for (n[1] = base[1] - K[1]; n[1] <= base[1] + K[1]; ++n[1])
          for (n[2] = base[2] - K[2]; n[2] <= base[2] + K[2]; ++n[2]) {
            if (j == i && n[0] == 0 && n[1] == 0 && n[2] == 0) continue;
            double d[3];
            pair_disp(coord + 3 * i, coord + 3 * j, n, box, d);
            double r2 = norm2(d);
            if (r2 < rc2) {
              Cand e;
              e.type = type[j];
              std::memcpy(&e.r2bits, &r2, 8);
              e.j = j;
              e.code = pack_shift(n[0], n[1], n[2]);
              cand.push_back(e);
            }
          }
    }
    std::sort(cand.begin(), cand.end(), cand_less);
    for (int k = 0; k < L.nc; ++k) { nl_j[(long)i * L.nc + k] = -1; nl_code[(long)i * L.nc + k] = pack_shift(0, 0, 0); }
    std::vector<int> cnt(c.ntypes, 0);
    for (const Cand& e : cand) {
      int t = e.type;
      if (cnt[t] < L.lsel[t]) {
        long slot = (long)i * L.nc + L.sel_off[t] + cnt[t];
        nl_j[slot] = e.j;
        nl_code[slot] = e.code;
      }
      cnt[t]++;
    }
    for (int t = 0; t < c.ntypes; ++t) {
      if (cnt[t] > L.lsel[t]) overflow++;
      if (counts) counts[(long)i * c.ntypes + t] = cnt[t];
    }
  }
  return overflow;
}

// ------------------------------------------------------------------------------------------
// Per-atom forward + reverse pass (FP64).  Embedding either by the network (Eq. G2) or by
// the quintic table (Eq. compress).
// ------------------------------------------------------------------------------------------
struct Table {
  const double* coef;  // [nets][L_c][M][6] : a b c d e f
  double s0, stride1, stride2;
  int n1, n2;
  int lc() const { return n1 + n2; }
  double node(int l) const { return l <= n1 ? s0 + l * stride1 : s0 + n1 * stride1 + (l - n1) * stride2; }
  int interval(double s, int* out_of_range) const {
    double split = s0 + n1 * stride1;
    int l;
    if (s < s0) { l = 0; *out_of_range = 1; }
    else if (s < split) { l = (int)std::floor((s - s0) / stride1); if (l > n1 - 1) l = n1 - 1; }
    else {
      l = n1 + (int)std::floor((s - split) / stride2);
      if (l > n1 + n2 - 1) { l = n1 + n2 - 1; }
      if (s > node(n1 + n2)) *out_of_range = 1;
    }
    return l;
  }
};

struct AtomOut {
  double e;
  int range_err;
};

// Embedding forward of net `net` of family S for one scalar input; keeps the tanh outputs
// and the layer outputs (the last is G, M values).
void embed_forward(const NetSet& S, const double* params, int net, double s, std::vector<std::vector<double>>& act,
                   std::vector<std::vector<double>>& outs) {
  act.assign(S.nl, {});
  outs.assign(S.nl, {});
  std::vector<double> x(1, s);
  for (int l = 0; l < S.nl; ++l) {
    const double* W = params + S.off[(size_t)net * S.nl + l];
    const double* b = W + (long)S.in[l] * S.out[l];
    int ni = S.in[l], no = S.out[l];
    act[l].assign(no, 0.0);
    outs[l].assign(no, 0.0);
    int sk = skip_kind(ni, no);
    for (int o = 0; o < no; ++o) {
      double z = b[o];
      for (int i = 0; i < ni; ++i) z += x[i] * W[(long)i * no + o];
      double t = std::tanh(z);
      act[l][o] = t;
      outs[l][o] = t + (sk == 1 ? x[o] : (sk == 2 ? x[o % ni] : 0.0));
    }
    x = outs[l];
  }
}

// Reverse pass of the embedding net: given dE/dG (M), returns dE/ds.
double embed_backward(const NetSet& S, const double* params, int net, const std::vector<std::vector<double>>& act,
                      std::vector<double> gy) {
  for (int l = S.nl - 1; l >= 0; --l) {
    const double* W = params + S.off[(size_t)net * S.nl + l];
    int ni = S.in[l], no = S.out[l];
    int sk = skip_kind(ni, no);
    std::vector<double> gx(ni, 0.0);
    for (int o = 0; o < no; ++o) {
      double gz = gy[o] * (1.0 - act[l][o] * act[l][o]);
      for (int i = 0; i < ni; ++i) gx[i] += gz * W[(long)i * no + o];
      if (sk == 1) gx[o] += gy[o];
      if (sk == 2) gx[o % ni] += gy[o];
    }
    gy = gx;
  }
  return gy[0];
}

// Embedding outputs of one neighbour for a family: by the nets (Eq. (G2)), or, when `tab` is
// given, by the quintic pieces (Eq. (compress)) with their derivatives dG/ds.
struct EmbedRow {
  std::vector<double> G, dG;
  std::vector<std::vector<double>> act, outs;
};

void embed_row(const NetSet& S, const double* params, const Table* tab, int net, double s, EmbedRow& e, int* oor) {
  const int M = S.m;
  e.G.assign(M, 0.0);
  e.dG.assign(M, 0.0);
  if (!tab) {
    embed_forward(S, params, net, s, e.act, e.outs);
    for (int mm = 0; mm < M; ++mm) e.G[mm] = e.outs[S.nl - 1][mm];
    return;
  }
  // g(t) with t = s - x_l inside interval l
  int l = tab->interval(s, oor);
  double t = s - tab->node(l);
  const double* co = tab->coef + (((size_t)net * tab->lc() + l) * M) * 6;
  for (int mm = 0; mm < M; ++mm) {
    const double* p = co + (size_t)mm * 6;
    e.G[mm] = ((((p[0] * t + p[1]) * t + p[2]) * t + p[3]) * t + p[4]) * t + p[5];
    e.dG[mm] = (((5.0 * p[0] * t + 4.0 * p[1]) * t + 3.0 * p[2]) * t + 2.0 * p[3]) * t + p[4];
  }
}

// dE/ds through the embedding of one neighbour, given dE/dG.
double embed_row_backward(const NetSet& S, const double* params, const Table* tab, int net, const EmbedRow& e,
                          const std::vector<double>& gG) {
  if (!tab) return embed_backward(S, params, net, e.act, gG);
  double acc = 0.0;
  for (int mm = 0; mm < S.m; ++mm) acc += gG[mm] * e.dG[mm];
  return acc;
}

// Environment of atom i for one part: its slots (type block t, position q < sel_P[t]) read the
// same positions of the list's type blocks; a listed neighbour at or beyond the part's cutoff is
// padding for that part.  The list holds, per type, the nearest neighbours within the widest
// cutoff sorted by distance, so a part's own list is exactly this prefix.
struct PartEnv {
  std::vector<double> R, dvec, rr, ss;  // [nc*4] rows (s, s u), [nc*3] r_ij, [nc] r, [nc] s
  std::vector<int> valid, tk, ls;       // per part slot: real neighbour, its type, list slot
};

void part_env(const Layout& L, const Part& P, int i, const double* coord, const double* box, const int* nl_j,
              const int* nl_code, PartEnv& E) {
  const int nc = P.nc;
  E.R.assign((size_t)nc * 4, 0.0);
  E.dvec.assign((size_t)nc * 3, 0.0);
  E.rr.assign(nc, 0.0);
  E.ss.assign(nc, 0.0);
  E.valid.assign(nc, 0);
  E.tk.assign(nc, 0);
  E.ls.assign(nc, 0);
  for (int t = 0; t < L.ntypes; ++t)
    for (int q = 0; q < P.sel[t]; ++q) {
      const int k = P.sel_off[t] + q, ls = L.sel_off[t] + q;
      E.tk[k] = t;
      E.ls[k] = ls;
      const int j = nl_j[(long)i * L.nc + ls];
      if (j < 0) continue;
      int n[3];
      unpack_shift(nl_code[(long)i * L.nc + ls], n);
      double d[3];
      pair_disp(coord + 3 * i, coord + 3 * j, n, box, d);
      const double r2 = norm2(d);
      if (!(r2 < P.rc * P.rc)) continue;
      const double r = std::sqrt(r2), sv = switch_fn(r, P.rs, P.rc);
      E.valid[k] = 1;
      E.rr[k] = r;
      E.ss[k] = sv;
      for (int a = 0; a < 3; ++a) E.dvec[(size_t)k * 3 + a] = d[a];
      E.R[(size_t)k * 4 + 0] = sv;
      for (int a = 0; a < 3; ++a) E.R[(size_t)k * 4 + 1 + a] = sv * d[a] / r;
    }
}

inline double dot4(const double* a, const double* b) { return ((a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]) + a[3] * b[3]; }

// Forward state of one part of one atom, kept for its reverse pass.
struct PartState {
  PartEnv E;
  std::vector<int> netk;      // two-body parts: net of each slot
  std::vector<EmbedRow> emb;  // two-body parts: embedding rows
  std::vector<double> T;      // se_e2_a: T (M x 4)
};

void part_forward(const OrcConfig& c, const Layout& L, const Part& P, const double* params, const Table* tab, int i,
                  int ai, const double* coord, const double* box, const int* nl_j, const int* nl_code, PartState& S,
                  double* D, int* range_err) {
  part_env(L, P, i, coord, box, nl_j, nl_code, S.E);
  const PartEnv& E = S.E;
  const int nc = P.nc, M = P.nets.m;
  if (P.kind == PART_E3) {
    // D_m = (1/Nc^2) sum_{j,k} theta_jk G_jkm, theta_jk = R_j . R_k, G_jk = N^{a_j,a_k}(theta_jk)
    // (by the nets, or by the quintic pieces in theta when a table is given)
    std::vector<double> acc(M, 0.0);
    EmbedRow row;
    for (int j = 0; j < nc; ++j) {
      if (!E.valid[j]) continue;
      for (int k = 0; k < nc; ++k) {
        if (!E.valid[k]) continue;
        const double th = dot4(&E.R[(size_t)j * 4], &E.R[(size_t)k * 4]);
        int oor = 0;
        embed_row(P.nets, params, tab, E.tk[j] * L.ntypes + E.tk[k], th, row, &oor);
        if (oor) *range_err = 1;
        for (int m = 0; m < M; ++m) acc[m] += th * row.G[m];
      }
    }
    for (int m = 0; m < M; ++m) D[P.doff + m] = acc[m] / ((double)nc * nc);
    return;
  }
  // two-body parts: Eq. (G2) / Eq. (compress) rows of real neighbours
  S.netk.assign(nc, 0);
  S.emb.assign(nc, EmbedRow());
  for (int k = 0; k < nc; ++k) {
    S.netk[k] = embed_net_index(c, ai, E.tk[k]);
    if (!E.valid[k]) continue;
    int oor = 0;
    embed_row(P.nets, params, tab, S.netk[k], E.ss[k], S.emb[k], &oor);
    if (oor) *range_err = 1;
  }
  if (P.kind == PART_R) {
    // D_m = (1/Nc) sum_k G_km s_k
    for (int m = 0; m < M; ++m) {
      double acc = 0.0;
      for (int k = 0; k < nc; ++k)
        if (E.valid[k]) acc += S.emb[k].G[m] * E.ss[k];
      D[P.doff + m] = acc / nc;
    }
    return;
  }
  // se_e2_a: T = (1/Nc) G^T R (M x 4), D = T T_<^T (M x M_<), flattened row-major
  const int A = P.axis;
  S.T.assign((size_t)M * 4, 0.0);
  for (int m = 0; m < M; ++m)
    for (int q = 0; q < 4; ++q) {
      double acc = 0.0;
      for (int k = 0; k < nc; ++k)
        if (E.valid[k]) acc += S.emb[k].G[m] * E.R[(size_t)k * 4 + q];
      S.T[(size_t)m * 4 + q] = acc / nc;
    }
  for (int m = 0; m < M; ++m)
    for (int l = 0; l < A; ++l) {
      double acc = 0.0;
      for (int q = 0; q < 4; ++q) acc += S.T[(size_t)m * 4 + q] * S.T[(size_t)l * 4 + q];
      D[P.doff + (size_t)m * A + l] = acc;
    }
}

// Reverse pass of one part: adds dE/dr_ij of each of its slots to gd at the slot's list position.
void part_backward(const Layout& L, const Part& P, const double* params, const Table* tab, const PartState& S,
                   const double* gD, double* gd) {
  const PartEnv& E = S.E;
  const int nc = P.nc, M = P.nets.m;
  std::vector<double> gR((size_t)nc * 4, 0.0), gs(nc, 0.0);  // dE/dR rows; dE/ds through the nets
  if (P.kind == PART_E3) {
    // dE/dtheta_jk = (1/Nc^2) [ sum_m gD_m G_jkm + dE/dtheta through the net with dE/dG_jkm = gD_m theta ];
    // dtheta_jk/dR_j = R_k, dtheta_jk/dR_k = R_j
    const double inv = 1.0 / ((double)nc * nc);
    EmbedRow row;
    std::vector<double> gG(M);
    for (int j = 0; j < nc; ++j) {
      if (!E.valid[j]) continue;
      for (int k = 0; k < nc; ++k) {
        if (!E.valid[k]) continue;
        const double* Rj = &E.R[(size_t)j * 4];
        const double* Rk = &E.R[(size_t)k * 4];
        const double th = dot4(Rj, Rk);
        const int net = E.tk[j] * L.ntypes + E.tk[k];
        int oor = 0;
        embed_row(P.nets, params, tab, net, th, row, &oor);
        double direct = 0.0;
        for (int m = 0; m < M; ++m) {
          direct += gD[P.doff + m] * row.G[m];
          gG[m] = gD[P.doff + m] * th * inv;
        }
        const double gth = direct * inv + embed_row_backward(P.nets, params, tab, net, row, gG);
        for (int q = 0; q < 4; ++q) {
          gR[(size_t)j * 4 + q] += gth * Rk[q];
          gR[(size_t)k * 4 + q] += gth * Rj[q];
        }
      }
    }
  } else {
    std::vector<double> gT;
    if (P.kind == PART_A) {
      // dE/dT[p][q] = sum_l gD[p][l] T[l][q] + [p < M_<] sum_m gD[m][p] T[m][q]
      const int A = P.axis;
      const double* g = gD + P.doff;
      gT.assign((size_t)M * 4, 0.0);
      for (int p = 0; p < M; ++p)
        for (int q = 0; q < 4; ++q) {
          double acc = 0.0;
          for (int l = 0; l < A; ++l) acc += g[(size_t)p * A + l] * S.T[(size_t)l * 4 + q];
          if (p < A)
            for (int m = 0; m < M; ++m) acc += g[(size_t)m * A + p] * S.T[(size_t)m * 4 + q];
          gT[(size_t)p * 4 + q] = acc;
        }
    }
    std::vector<double> gG(M);
    for (int k = 0; k < nc; ++k) {
      if (!E.valid[k]) continue;
      const std::vector<double>& G = S.emb[k].G;
      if (P.kind == PART_A) {
        // dE/dR_k[q] = (1/Nc) sum_m gT[m][q] G_k[m];  dE/dG_k[m] = (1/Nc) sum_q gT[m][q] R_k[q]
        for (int q = 0; q < 4; ++q) {
          double acc = 0.0;
          for (int m = 0; m < M; ++m) acc += gT[(size_t)m * 4 + q] * G[m];
          gR[(size_t)k * 4 + q] = acc / nc;
        }
        for (int m = 0; m < M; ++m) {
          double acc = 0.0;
          for (int q = 0; q < 4; ++q) acc += gT[(size_t)m * 4 + q] * E.R[(size_t)k * 4 + q];
          gG[m] = acc / nc;
        }
      } else {
        // dE/dG_k[m] = gD_m s_k / Nc and the direct dE/ds_k = sum_m gD_m G_k[m] / Nc
        double direct = 0.0;
        for (int m = 0; m < M; ++m) {
          gG[m] = gD[P.doff + m] * E.ss[k] / nc;
          direct += gD[P.doff + m] * G[m] / nc;
        }
        gR[(size_t)k * 4 + 0] = direct;
      }
      gs[k] = embed_row_backward(P.nets, params, tab, S.netk[k], S.emb[k], gG);
    }
  }
  // chain through R_k = (s, s u) with u = d / r, s = s(r), r = |d|
  for (int k = 0; k < nc; ++k) {
    if (!E.valid[k]) continue;
    const double r = E.rr[k], sv = E.ss[k];
    const double sp = switch_deriv(r, P.rs, P.rc);
    const double* d = &E.dvec[(size_t)k * 3];
    const double* g = &gR[(size_t)k * 4];
    const double u[3] = {d[0] / r, d[1] / r, d[2] / r};
    const double gvu = g[1] * u[0] + g[2] * u[1] + g[3] * u[2];
    const double gsum = gs[k] + g[0] + gvu;  // total dE/ds at fixed u
    for (int a = 0; a < 3; ++a) gd[(size_t)E.ls[k] * 3 + a] += sp * gsum * u[a] + (sv / r) * (g[1 + a] - gvu * u[a]);
  }
}

// One atom: descriptor (all parts), fitting net, and the reverse pass down to dE/dr_ij per list
// slot (gd [L.nc * 3]).  The table, when given, replaces the nets of the first part: pieces in s for
// a two-body part, in theta for se_e3.
void atom_pass(const OrcConfig& c, const Layout& L, const double* params, const Table* tab, int i, const double* coord,
               const int* type, const double* box, const int* nl_j, const int* nl_code, double* gd, AtomOut* out) {
  const int ai = type[i];
  out->range_err = 0;
  const size_t np = L.parts.size();
  std::vector<PartState> S(np);
  std::vector<double> D(L.dw, 0.0);
  for (size_t q = 0; q < np; ++q)
    part_forward(c, L, L.parts[q], params, q == 0 ? tab : nullptr, i, ai, coord, box, nl_j, nl_code, S[q], D.data(),
                 &out->range_err);
  // Eq. (fitting): E_i = F_0^{a_i}(D)
  const int nfl = (int)L.fin.size();
  std::vector<std::vector<double>> fx(nfl + 1), fa(nfl);
  fx[0] = D;
  for (int l = 0; l < nfl; ++l) {
    const double* W = params + L.foff[(size_t)ai * nfl + l];
    const double* b = W + (long)L.fin[l] * L.fout[l];
    int ni = L.fin[l], no = L.fout[l];
    bool last = (l == nfl - 1);
    int sk = last ? 0 : skip_kind(ni, no);
    fx[l + 1].assign(no, 0.0);
    fa[l].assign(no, 0.0);
    for (int o = 0; o < no; ++o) {
      double z = b[o];
      for (int q = 0; q < ni; ++q) z += fx[l][q] * W[(long)q * no + o];
      double t = last ? z : std::tanh(z);
      fa[l][o] = t;
      fx[l + 1][o] = t + (sk == 1 ? fx[l][o] : (sk == 2 ? fx[l][o % ni] : 0.0));
    }
  }
  out->e = fx[nfl][0];
  // ---------------- reverse pass ----------------
  std::vector<double> gy(1, 1.0);
  for (int l = nfl - 1; l >= 0; --l) {
    const double* W = params + L.foff[(size_t)ai * nfl + l];
    int ni = L.fin[l], no = L.fout[l];
    bool last = (l == nfl - 1);
    int sk = last ? 0 : skip_kind(ni, no);
    std::vector<double> gx(ni, 0.0);
    for (int o = 0; o < no; ++o) {
      double gz = last ? gy[o] : gy[o] * (1.0 - fa[l][o] * fa[l][o]);
      for (int q = 0; q < ni; ++q) gx[q] += gz * W[(long)q * no + o];
      if (sk == 1) gx[o] += gy[o];
      if (sk == 2) gx[o % ni] += gy[o];
    }
    gy = gx;
  }
  for (int k = 0; k < L.nc * 3; ++k) gd[k] = 0.0;
  for (size_t q = 0; q < np; ++q) part_backward(L, L.parts[q], params, q == 0 ? tab : nullptr, S[q], gy.data(), gd);
}

// ------------------------------------------------------------------------------------------
// Templated energy (for the dual-number pins only): same definitions, generic scalar.
// ------------------------------------------------------------------------------------------
template <class T, class P>
std::vector<T> embed_generic(const NetSet& S, const P* params, int net, T s) {
  std::vector<T> x(1, s), y;
  for (int l = 0; l < S.nl; ++l) {
    const P* W = params + S.off[(size_t)net * S.nl + l];
    y.assign(S.out[l], T(0.0));
    layer_forward(W, W + (long)S.in[l] * S.out[l], S.in[l], S.out[l], x.data(), y.data(), true, true);
    x = y;
  }
  return x;
}

template <class T, class P>
T energy_generic(const OrcConfig& c, const Layout& L, const P* params, int N, const T* coord, const int* type,
                 const T* box, const int* nl_j, const int* nl_code, T* atom_e) {
  T E(0.0);
  for (int i = 0; i < N; ++i) {
    const int ai = type[i];
    std::vector<T> x(L.dw, T(0.0));
    for (const Part& Pt : L.parts) {
      const int nc = Pt.nc, M = Pt.nets.m;
      std::vector<std::vector<T>> R(nc);
      std::vector<T> sv(nc, T(0.0));
      std::vector<int> tk(nc, 0), valid(nc, 0);
      for (int t = 0; t < c.ntypes; ++t)
        for (int q = 0; q < Pt.sel[t]; ++q) {
          const int k = Pt.sel_off[t] + q, ls = L.sel_off[t] + q;
          tk[k] = t;
          const int j = nl_j[(long)i * L.nc + ls];
          if (j < 0) continue;
          int n[3];
          unpack_shift(nl_code[(long)i * L.nc + ls], n);
          T d[3];
          for (int a = 0; a < 3; ++a) {
            T tt(0.0);
            if (box) tt = T((double)n[0]) * box[a] + T((double)n[1]) * box[3 + a] + T((double)n[2]) * box[6 + a];
            d[a] = (coord[3 * j + a] + tt) - coord[3 * i + a];
          }
          T r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
          if (!(val(r2) < Pt.rc * Pt.rc)) continue;
          T r = dsqrt(r2);
          T s = switch_fn(r, Pt.rs, Pt.rc);
          valid[k] = 1;
          sv[k] = s;
          R[k] = {s, s * d[0] / r, s * d[1] / r, s * d[2] / r};
        }
      if (Pt.kind == PART_E3) {
        std::vector<T> acc(M, T(0.0));
        for (int j = 0; j < nc; ++j)
          for (int k = 0; k < nc; ++k) {
            if (!valid[j] || !valid[k]) continue;
            T th = ((R[j][0] * R[k][0] + R[j][1] * R[k][1]) + R[j][2] * R[k][2]) + R[j][3] * R[k][3];
            std::vector<T> g = embed_generic<T, P>(Pt.nets, params, tk[j] * c.ntypes + tk[k], th);
            for (int m = 0; m < M; ++m) acc[m] = acc[m] + th * g[m];
          }
        for (int m = 0; m < M; ++m) x[Pt.doff + m] = acc[m] / T((double)nc * nc);
        continue;
      }
      std::vector<T> Tm((size_t)M * 4, T(0.0)), Dr(M, T(0.0));
      for (int k = 0; k < nc; ++k) {
        if (!valid[k]) continue;
        std::vector<T> g = embed_generic<T, P>(Pt.nets, params, embed_net_index(c, ai, tk[k]), sv[k]);
        for (int m = 0; m < M; ++m) {
          if (Pt.kind == PART_R) Dr[m] = Dr[m] + g[m] * sv[k];
          else
            for (int q = 0; q < 4; ++q) Tm[(size_t)m * 4 + q] = Tm[(size_t)m * 4 + q] + g[m] * R[k][q];
        }
      }
      if (Pt.kind == PART_R) {
        for (int m = 0; m < M; ++m) x[Pt.doff + m] = Dr[m] / T((double)nc);
        continue;
      }
      const int A = Pt.axis;
      for (auto& v : Tm) v = v / T((double)nc);
      for (int m = 0; m < M; ++m)
        for (int l = 0; l < A; ++l) {
          T acc(0.0);
          for (int q = 0; q < 4; ++q) acc = acc + Tm[(size_t)m * 4 + q] * Tm[(size_t)l * 4 + q];
          x[Pt.doff + (size_t)m * A + l] = acc;
        }
    }
    const int nfl = (int)L.fin.size();
    for (int l = 0; l < nfl; ++l) {
      const P* W = params + L.foff[(size_t)ai * nfl + l];
      std::vector<T> y(L.fout[l]);
      bool last = l == nfl - 1;
      layer_forward(W, W + (long)L.fin[l] * L.fout[l], L.fin[l], L.fout[l], x.data(), y.data(), !last, !last);
      x = y;
    }
    if (atom_e) atom_e[i] = x[0];
    E = E + x[0];
  }
  return E;
}

// Node values y, y', y'' of every output of embedding net `net` at input s (second-order jets).
void embed_jets(const Layout& L, const double* params, int net, double s, double* y, double* y1,
                double* y2) {
  const NetSet& S = L.e1;
  std::vector<Jet> x(1, Jet(s, 1.0, 0.0));
  for (int l = 0; l < S.nl; ++l) {
    const double* W = params + S.off[(size_t)net * S.nl + l];
    const double* b = W + (long)S.in[l] * S.out[l];
    int ni = S.in[l], no = S.out[l];
    int sk = skip_kind(ni, no);
    std::vector<Jet> yv(no);
    for (int o = 0; o < no; ++o) {
      Jet z(b[o], 0.0, 0.0);
      for (int i = 0; i < ni; ++i) z = z + x[i] * W[(long)i * no + o];
      Jet a = jtanh(z);
      if (sk == 1) a = a + x[o];
      if (sk == 2) a = a + x[o % ni];
      yv[o] = a;
    }
    x = yv;
  }
  for (int mm = 0; mm < L.m; ++mm) { y[mm] = x[mm].v; y1[mm] = x[mm].d1; y2[mm] = x[mm].d2; }
}

// Eq. (compress): quintic coefficients (a..f) on an interval of width dx from the values,
// first and second derivatives at its two ends.
void quintic(double y0, double y1, double d0, double d1, double dd0, double dd1, double dx, double* out) {
  double h = y1 - y0;
  double dx2 = dx * dx, dx3 = dx2 * dx, dx4 = dx3 * dx, dx5 = dx4 * dx;
  out[0] = (12.0 * h - 6.0 * (d1 + d0) * dx + (dd1 - dd0) * dx2) / (2.0 * dx5);
  out[1] = (-30.0 * h + (14.0 * d1 + 16.0 * d0) * dx + (-2.0 * dd1 + 3.0 * dd0) * dx2) / (2.0 * dx4);
  out[2] = (20.0 * h - (8.0 * d1 + 12.0 * d0) * dx + (dd1 - 3.0 * dd0) * dx2) / (2.0 * dx3);
  out[3] = 0.5 * dd0;
  out[4] = d0;
  out[5] = y0;
}

}  // namespace

// ==========================================================================================
// C entry points (ctypes)
// ==========================================================================================
extern "C" {

long orc_n_params(const OrcConfig* c) { return make_layout(*c).n_params; }

void orc_switch(double r, double rs, double rc, double* s, double* ds) {
  *s = switch_fn(r, rs, rc);
  *ds = switch_deriv(r, rs, rc);
}

void orc_quintic(double y0, double y1, double d0, double d1, double dd0, double dd1, double dx, double* out) {
  quintic(y0, y1, d0, d1, dd0, dd1, dx, out);
}

// Brute-force neighbour list.  nl_shift is [N*Nc*3] image integers (0 for padding).
int orc_nlist(const OrcConfig* c, int N, const double* coord, const int* type, const double* box, int* nl_j,
              int* nl_shift, int* counts) {
  Layout L = make_layout(*c);
  std::vector<int> code((size_t)N * L.nc);
  int ov = build_nlist(*c, L, N, coord, type, box, nl_j, code.data(), counts);
  for (size_t k = 0; k < code.size(); ++k) unpack_shift(code[k], nl_shift + 3 * k);
  return ov;
}

// Embedding-net outputs and their first/second derivatives at inputs xs[n] for net `net`.
void orc_embed_jets(const OrcConfig* c, const double* params, int net, int n, const double* xs, double* y,
                    double* y1, double* y2) {
  Layout L = make_layout(*c);
  for (int q = 0; q < n; ++q)
    embed_jets(L, params, net, xs[q], y + (size_t)q * L.m, y1 + (size_t)q * L.m, y2 + (size_t)q * L.m);
}

// Quintic table over nodes x_0 .. x_{n1+n2}: first n1 intervals of width stride1 from s0,
// then n2 intervals of width stride2.  table: [nets][n1+n2][M][6].
void orc_table_build(const OrcConfig* c, const double* params, double s0, double stride1, int n1, double stride2,
                     int n2, double* table) {
  Layout L = make_layout(*c);
  Table tb{nullptr, s0, stride1, stride2, n1, n2};
  int lc = n1 + n2, M = L.m;
  std::vector<double> y((size_t)(lc + 1) * M), y1(y.size()), y2(y.size());
  for (int net = 0; net < L.n_embed_nets; ++net) {
    for (int l = 0; l <= lc; ++l)
      embed_jets(L, params, net, tb.node(l), &y[(size_t)l * M], &y1[(size_t)l * M], &y2[(size_t)l * M]);
    for (int l = 0; l < lc; ++l) {
      double dx = tb.node(l + 1) - tb.node(l);
      for (int mm = 0; mm < M; ++mm) {
        size_t a = (size_t)l * M + mm, b = (size_t)(l + 1) * M + mm;
        quintic(y[a], y[b], y1[a], y1[b], y2[a], y2[b], dx, table + (((size_t)net * lc + l) * M + mm) * 6);
      }
    }
  }
}

// Energy, forces, virial (and per-atom energies).  If nl_j is null the brute-force
// neighbour list is built here.  table null => embedding network; else quintic table.
// Returns (number of overflowing neighbour blocks) + 1000000 * (any table range error).
int orc_compute(const OrcConfig* cfg, const double* params, int N, const double* coord, const int* type,
                const double* box, const int* nl_j_in, const int* nl_shift_in, const double* table, double s0,
                double stride1, int n1, double stride2, int n2, double* energy, double* force, double* virial,
                double* atom_energy, int nthreads) {
  const OrcConfig& c = *cfg;
  Layout L = make_layout(c);
  const int nc = L.nc;
  std::vector<int> nl_j((size_t)N * nc), code((size_t)N * nc);
  int ov = 0;
  if (!nl_j_in) {
    ov = build_nlist(c, L, N, coord, type, box, nl_j.data(), code.data(), nullptr);
  } else {
    for (size_t k = 0; k < nl_j.size(); ++k) {
      nl_j[k] = nl_j_in[k];
      code[k] = pack_shift(nl_shift_in[3 * k], nl_shift_in[3 * k + 1], nl_shift_in[3 * k + 2]);
    }
  }
  Table tb{table, s0, stride1, stride2, n1, n2};
  const Table* tp = table ? &tb : nullptr;
  std::vector<double> gd((size_t)N * nc * 3, 0.0);
  std::vector<AtomOut> ao(N);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int i = 0; i < N; ++i)
    atom_pass(c, L, params, tp, i, coord, type, box, nl_j.data(), code.data(), &gd[(size_t)i * nc * 3], &ao[i]);
  (void)nthreads;
  // E = sum_i E_i ; F_i += dE/dr_ij, F_j -= dE/dr_ij ; Xi_ab = -sum (dE/dr_ij)_a (r_ij)_b
  double E = 0.0;
  int rerr = 0;
  for (int i = 0; i < N; ++i) {
    E += ao[i].e;
    rerr |= ao[i].range_err;
    if (atom_energy) atom_energy[i] = ao[i].e;
  }
  *energy = E;
  for (int k = 0; k < 3 * N; ++k) force[k] = 0.0;
  for (int k = 0; k < 9; ++k) virial[k] = 0.0;
  for (int i = 0; i < N; ++i)
    for (int k = 0; k < nc; ++k) {
      int j = nl_j[(size_t)i * nc + k];
      if (j < 0) continue;
      int n[3];
      unpack_shift(code[(size_t)i * nc + k], n);
      double d[3];
      pair_disp(coord + 3 * i, coord + 3 * j, n, box, d);
      const double* g = &gd[((size_t)i * nc + k) * 3];
      for (int a = 0; a < 3; ++a) {
        force[3 * i + a] += g[a];
        force[3 * j + a] -= g[a];
      }
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) virial[3 * a + b] -= g[a] * d[b];
    }
  return ov + (rerr ? 1000000 : 0);
}

// Dual-number directional derivative of E along a coordinate direction dcoord [N*3] and a
// box direction dbox [9] (the neighbour list is given and held fixed).  Returns E; writes
// the derivative into *dE.  Per-atom energies (values) are written to atom_energy if given.
double orc_energy_dual(const OrcConfig* c, const double* params, int N, const double* coord, const double* dcoord,
                       const int* type, const double* box, const double* dbox, const int* nl_j, const int* nl_shift,
                       double* dE, double* atom_energy) {
  Layout L = make_layout(*c);
  std::vector<int> code((size_t)N * L.nc);
  for (size_t k = 0; k < code.size(); ++k)
    code[k] = pack_shift(nl_shift[3 * k], nl_shift[3 * k + 1], nl_shift[3 * k + 2]);
  std::vector<Dual> x((size_t)N * 3), h(9), ae(N);
  for (int k = 0; k < 3 * N; ++k) x[k] = Dual(coord[k], dcoord ? dcoord[k] : 0.0);
  if (box)
    for (int k = 0; k < 9; ++k) h[k] = Dual(box[k], dbox ? dbox[k] : 0.0);
  Dual E = energy_generic<Dual>(*c, L, params, N, x.data(), type, box ? h.data() : nullptr, nl_j, code.data(),
                                ae.data());
  if (atom_energy)
    for (int i = 0; i < N; ++i) atom_energy[i] = ae[i].v;
  *dE = E.d;
  return E.v;
}

// Brute-force neighbour rows of single atoms (Sec. III.B.1 order), for frames too large for the
// full list: every j and every image within K cells of the nearest one, sorted by the exact key.
struct RowBuilder {
  const OrcConfig& c;
  const Layout& L;
  int N;
  const double* coord;
  const int* type;
  const double* box;
  double rc2;
  double inv[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  int K[3] = {0, 0, 0};
  RowBuilder(const OrcConfig& c_, const Layout& L_, int N_, const double* coord_, const int* type_,
             const double* box_)
      : c(c_), L(L_), N(N_), coord(coord_), type(type_), box(box_), rc2(L_.lrc * L_.lrc) {
    if (box) {
      inverse3(box, inv);
      double vol = std::fabs(box[0] * (box[4] * box[8] - box[5] * box[7]) -
                             box[1] * (box[3] * box[8] - box[5] * box[6]) + box[2] * (box[3] * box[7] - box[4] * box[6]));
      for (int d = 0; d < 3; ++d) {
        const double* u = box + 3 * ((d + 1) % 3);
        const double* v = box + 3 * ((d + 2) % 3);
        double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
        K[d] = (int)std::ceil(L.lrc / (vol / std::sqrt(cx * cx + cy * cy + cz * cz))) + 1;
      }
    }
  }
  long mfloor(int a, int d) const {
    if (!box) return 0;
    double f = coord[3 * a] * inv[d] + coord[3 * a + 1] * inv[3 + d] + coord[3 * a + 2] * inv[6 + d];
    return (long)std::floor(f);
  }
  // Row of atom i into nl_j / nl_code (Nc entries each); returns the number of overflowing blocks.
  int row(int i, int* nl_j, int* nl_code) const {
    std::vector<Cand> cand;
    for (int j = 0; j < N; ++j) {
      int base[3];
      for (int d = 0; d < 3; ++d) base[d] = (int)(mfloor(i, d) - mfloor(j, d));
      int n[3];
      for (n[0] = base[0] - K[0]; n[0] <= base[0] + K[0]; ++n[0])
        for (n[1] = base[1] - K[1]; n[1] <= base[1] + K[1]; ++n[1])
          for (n[2] = base[2] - K[2]; n[2] <= base[2] + K[2]; ++n[2]) {
            if (j == i && n[0] == 0 && n[1] == 0 && n[2] == 0) continue;
            double d[3];
            pair_disp(coord + 3 * i, coord + 3 * j, n, box, d);
            double r2 = norm2(d);
            if (r2 < rc2) {
              Cand e;
              e.type = type[j];
              std::memcpy(&e.r2bits, &r2, 8);
              e.j = j;
              e.code = pack_shift(n[0], n[1], n[2]);
              cand.push_back(e);
            }
          }
    }
    std::sort(cand.begin(), cand.end(), cand_less);
    for (int k = 0; k < L.nc; ++k) {
      nl_j[k] = -1;
      nl_code[k] = pack_shift(0, 0, 0);
    }
    std::vector<int> cnt(c.ntypes, 0);
    for (const Cand& e : cand) {
      if (cnt[e.type] < L.lsel[e.type]) {
        nl_j[L.sel_off[e.type] + cnt[e.type]] = e.j;
        nl_code[L.sel_off[e.type] + cnt[e.type]] = e.code;
      }
      cnt[e.type]++;
    }
    int ov = 0;
    for (int t = 0; t < c.ntypes; ++t) ov += cnt[t] > L.lsel[t];
    return ov;
  }
};

// Neighbour rows and atomic energies of a subset of atoms only (brute force over all j and
// images for each selected atom), for sampled checks of frames too large for the full oracle.
int orc_atom_subset(const OrcConfig* cfg, const double* params, int N, const double* coord, const int* type,
                    const double* box, int nsel, const int* idx, int* nl_j_out, int* nl_shift_out, double* e_out) {
  const OrcConfig& c = *cfg;
  Layout L = make_layout(c);
  const int nc = L.nc;
  RowBuilder rb(c, L, N, coord, type, box);
  std::vector<int> nl_j((size_t)N * nc, -1), nl_code((size_t)N * nc, pack_shift(0, 0, 0));
  int ov = 0;
  for (int s = 0; s < nsel; ++s) {
    const int i = idx[s];
    ov += rb.row(i, &nl_j[(size_t)i * nc], &nl_code[(size_t)i * nc]);
  }
  std::vector<double> gd((size_t)nc * 3);
  for (int s = 0; s < nsel; ++s) {
    const int i = idx[s];
    AtomOut ao;
    atom_pass(c, L, params, nullptr, i, coord, type, box, nl_j.data(), nl_code.data(), gd.data(), &ao);
    if (e_out) e_out[s] = ao.e;
    for (int k = 0; k < nc; ++k) {
      if (nl_j_out) nl_j_out[(size_t)s * nc + k] = nl_j[(size_t)i * nc + k];
      if (nl_shift_out) unpack_shift(nl_code[(size_t)i * nc + k], nl_shift_out + 3 * ((size_t)s * nc + k));
    }
  }
  return ov;
}

// Forces on a subset of atoms only.  F_k = -dE/dr_k collects, from every atom i whose list holds
// k, the pair term of each slot (F_i += dE/dr_ij, F_j -= dE/dr_ij, Sec. II.A.2); those atoms lie
// within r_c of k, so only the rows and atom passes of k's neighbourhood are formed (by brute
// force, as orc_atom_subset).  Network embedding only.  force_out [nsel][3]; e_out [nsel] or null.
int orc_force_subset(const OrcConfig* cfg, const double* params, int N, const double* coord, const int* type,
                     const double* box, int nsel, const int* idx, double* force_out, double* e_out, int nthreads) {
  const OrcConfig& c = *cfg;
  Layout L = make_layout(c);
  const int nc = L.nc;
  RowBuilder rb(c, L, N, coord, type, box);
  // the sampled atoms' rows name their neighbourhoods
  std::vector<int> need(N, 0);
  std::vector<int> rj(nc), rcode(nc);
  int ov = 0;
  for (int s = 0; s < nsel; ++s) {
    need[idx[s]] = 1;
    // every atom within r_c of k, listed or beyond sel: a wider row with sel = the atom count
    Layout Lw = widened(L, N * 27);
    RowBuilder rw(c, Lw, N, coord, type, box);
    std::vector<int> wj(Lw.nc), wc(Lw.nc);
    rw.row(idx[s], wj.data(), wc.data());
    for (int k = 0; k < Lw.nc; ++k)
      if (wj[k] >= 0) need[wj[k]] = 1;
  }
  std::vector<int> rows;
  for (int i = 0; i < N; ++i)
    if (need[i]) rows.push_back(i);
  std::vector<int> nl_j((size_t)N * nc, -1), nl_code((size_t)N * nc, pack_shift(0, 0, 0));
  std::vector<double> gd(rows.size() * (size_t)nc * 3, 0.0);
  std::vector<AtomOut> ao(rows.size());
  std::vector<int> ovr(rows.size(), 0);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (long q = 0; q < (long)rows.size(); ++q) {
    const int i = rows[q];
    ovr[q] = rb.row(i, &nl_j[(size_t)i * nc], &nl_code[(size_t)i * nc]);
    atom_pass(c, L, params, nullptr, i, coord, type, box, nl_j.data(), nl_code.data(), &gd[(size_t)q * nc * 3], &ao[q]);
  }
  (void)nthreads;
  for (size_t q = 0; q < rows.size(); ++q) ov += ovr[q];
  for (int s = 0; s < nsel; ++s) {
    const int k = idx[s];
    double f[3] = {0.0, 0.0, 0.0};
    for (size_t q = 0; q < rows.size(); ++q) {
      const int i = rows[q];
      for (int sl = 0; sl < nc; ++sl) {
        const int j = nl_j[(size_t)i * nc + sl];
        if (j < 0) continue;
        const double* g = &gd[((size_t)q * nc + sl) * 3];
        for (int a = 0; a < 3; ++a) {
          if (i == k) f[a] += g[a];
          if (j == k) f[a] -= g[a];
        }
      }
      if (e_out && i == k) e_out[s] = ao[q].e;
    }
    for (int a = 0; a < 3; ++a) force_out[3 * s + a] = f[a];
  }
  return ov;
}

// Loss of a batch of frames, Sec. II.B, Eq. (loss) with the energy, force and virial terms:
//   L = (1/B) sum_f [ pE (E_f - E*_f)^2 / N_f + pF sum_i |F_i - F*_i|^2 / (3 N_f)
//                     + pXi sum_ab (Xi_f,ab - Xi*_f,ab)^2 / (9 N_f) ]
// and its derivative along the parameter direction v.  Forces and virials come from the reverse
// pass.  With Delta F = F - F*, sum_i Delta F_i . dF_i/dtheta . v = -d2E/(de1 de2) for the
// perturbation r + e1 Delta F, theta + e2 v; with G = Xi - Xi*, sum_ab G_ab dXi_ab/dtheta . v is
// -d2E/(de1 de2) for the homogeneous deformation r -> r + e1 r G^T, h -> h + e1 h G^T (the
// virial being minus the derivative of E under r -> r (I + eps), h -> h (I + eps) with respect
// to eps transposed).  Both deformations go into the one e1 direction, weighted by their loss
// coefficients, so one hyper-dual evaluation per frame gives the derivative exactly.
// Frames are concatenated (natoms[f] atoms each); boxes [B][9]; lists [sum natoms][Nc] (+shift);
// v_ref [B][9] may be null (no virial term).
double orc_loss_dir(const OrcConfig* cfg, const double* params, const double* vdir, int B, const int* natoms,
                    const double* coord, const int* type, const double* boxes, const int* nl_j, const int* nl_shift,
                    const double* e_ref, const double* f_ref, double pE, double pF, double* dL, const double* v_ref,
                    double pXi) {
  Layout L = make_layout(*cfg);
  const int nc = L.nc;
  const long np = L.n_params;
  std::vector<HD> hp(np);
  for (long k = 0; k < np; ++k) hp[k] = HD(params[k], 0.0, vdir ? vdir[k] : 0.0, 0.0);
  double loss = 0.0, dloss = 0.0;
  long off = 0;
  for (int f = 0; f < B; ++f) {
    const int n = natoms[f];
    const double* x = coord + 3 * off;
    const int* ty = type + off;
    const double* box = boxes + 9 * f;
    std::vector<int> nj(nl_j + off * nc, nl_j + (off + n) * nc);
    std::vector<int> ns(nl_shift + off * nc * 3, nl_shift + (off + n) * nc * 3);
    // shift the frame's neighbour indices to frame-local numbering
    for (auto& j : nj)
      if (j >= 0) j -= (int)off;
    std::vector<double> force((size_t)3 * n), vir(9), ae(n);
    double e = 0.0;
    orc_compute(cfg, params, n, x, ty, box, nj.data(), ns.data(), nullptr, 0, 0, 0, 0, 0, &e, force.data(), vir.data(),
                ae.data(), 0);
    const double dE = e - e_ref[f];
    const double cF = 2.0 * pF / (3.0 * n), cX = v_ref ? 2.0 * pXi / (9.0 * n) : 0.0;
    double G[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, x2 = 0.0;
    if (v_ref)
      for (int k = 0; k < 9; ++k) {
        G[k] = vir[k] - v_ref[9 * f + k];
        x2 += G[k] * G[k];
      }
    double f2 = 0.0;
    std::vector<HD> hx((size_t)3 * n), hb(9);
    for (int i = 0; i < n; ++i)
      for (int b = 0; b < 3; ++b) {
        const double dF = force[3 * i + b] - f_ref[3 * (off + i) + b];
        f2 += dF * dF;
        double t = cF * dF;  // e1 direction: force term ...
        for (int a = 0; a < 3; ++a) t += cX * x[3 * i + a] * G[3 * b + a];  // ... and deformation (r G^T)_b
        hx[3 * i + b] = HD(x[3 * i + b], t, 0.0, 0.0);
      }
    for (int g = 0; g < 3; ++g)
      for (int b = 0; b < 3; ++b) {
        double t = 0.0;
        for (int a = 0; a < 3; ++a) t += cX * box[3 * g + a] * G[3 * b + a];  // (h G^T)_gb
        hb[3 * g + b] = HD(box[3 * g + b], t, 0.0, 0.0);
      }
    std::vector<int> code((size_t)n * nc);
    for (size_t k = 0; k < code.size(); ++k) code[k] = pack_shift(ns[3 * k], ns[3 * k + 1], ns[3 * k + 2]);
    const HD E = energy_generic<HD, HD>(*cfg, L, hp.data(), n, hx.data(), ty, hb.data(), nj.data(), code.data(),
                                        nullptr);
    loss += pE * dE * dE / n + pF * f2 / (3.0 * n) + (v_ref ? pXi * x2 / (9.0 * n) : 0.0);
    dloss += 2.0 * pE * dE / n * E.b - E.ab;
    off += n;
  }
  if (dL) *dL = dloss / B;
  return loss / B;
}

// Plain-double energy through the generic template (pins the reverse-pass forward).
double orc_energy_plain(const OrcConfig* c, const double* params, int N, const double* coord, const int* type,
                        const double* box, const int* nl_j, const int* nl_shift) {
  Layout L = make_layout(*c);
  std::vector<int> code((size_t)N * L.nc);
  for (size_t k = 0; k < code.size(); ++k)
    code[k] = pack_shift(nl_shift[3 * k], nl_shift[3 * k + 1], nl_shift[3 * k + 2]);
  return energy_generic<double>(*c, L, params, N, coord, type, box, nl_j, code.data(), nullptr);
}

}  // extern "C"
