// qp_oracle.cpp -- plain FP64 CPU oracle for the QPINN hot path.
//
// TEST INFRASTRUCTURE ONLY. Only tests/, the package smoke check and the
// benchmark's CPU-baseline leg may load this library. It shares no code,
// header or constant table with the CUDA path; the only interface contract is
// the numeric meaning of the integer/double config arrays documented below.
//
// What it computes (arxiv 2506.23246):
//   * premap: direct angle map, or random Fourier features (Sec. 2.2, RFF bullet)
//     followed by a tanh MLP and one of the five angle scalings of Eq. 27a-e;
//   * the PQC of Sec. 2.3: RX (or RY) angle embedding on |0...0>, L ansatz layers
//     (Basic / Strongly entangling with Rot gates of Eq. 28, a RY,RZ variant,
//     or no entanglement), Pauli-Z readout per qubit (noiseless statevector,
//     Sec. 2.4), then a classical linear head to (Ez, Hx, Hy);
//   * the Maxwell residuals Eqs. 8-10, L_phys Eqs. 11-13, L_IC Eqs. 14-17,
//     Poynting energy residual Eq. 23, total loss Eq. 24 and the energy slice sums
//     U(t) of Eq. 31.
//
// Every derivative -- d/dx, d/dy, d/dt of the fields and d/dp of the loss for a
// selected parameter p -- is taken by forward-mode truncated Taylor arithmetic
// ("hyper-dual" numbers): each scalar carries 8 components
//   [0] value, [1..3] d/dx,d/dy,d/dt, [4] d/dp, [5..7] d^2/(dx dp), d^2/(dy dp), d^2/(dt dp).
// No adjoint, no fusion, no reordering: the gradient for parameter p is one
// full forward evaluation with component [4] seeded at p.
//
// Conventions (readings of the paper, fixed here and in the CUDA path):
//   * gates use the half-angle convention: RX(t)=exp(-i t X/2) etc., so that a
//     single qubit after RX(t) has <Z> = cos t (Fig. 3 caption).
//   * Rot(a,b,g) = RZ(g) RY(b) RZ(a) (Eq. 28).
//   * qubit q <-> bit (n-1-q) of the basis index (big-endian).
//   * CNOT ring of layer l: CNOT(i, (i+r) mod n) for i = 0..n-1 in this order,
//     r = 1 (Basic) or r = 1 + (l mod (n-1)) (Strongly entangling, Sec. 2.3 item 2).
//
// Config arrays (ctypes-friendly):
//   ci[ 0..11] = n_qubits, n_layers, n_readout, ansatz, enc, scale, premap,
//                n_direct, rff_freqs, mlp_width, mlp_depth, periodic
//     periodic (RFF premap): 1 = the periodic input map of Eqs. 25-26 before the RFF layer:
//       (x, y, t) -> (sin(2 pi x / 2), cos(2 pi x / 2), sin(2 pi y / 2), cos(2 pi y / 2),
//       sin(2 pi t / T), cos(2 pi t / T)) with the domain lengths L_x = L_y = 2 of [-1, 1]^2 and
//       a learned time period T
//     ansatz: 0 Basic RY,RZ   1 Basic Rot   2 Strongly Rot   3 No-entanglement Rot
//             4 Cross-Mesh (RX per qubit, CRZ(i,j) for every ordered pair i != j)
//             5 Cross-Mesh-2-Rotations (RX then RZ per qubit, the same CRZ mesh)
//             6 Cross-Mesh-CNOT (Rot per qubit, CNOT(i,j) for every ordered pair i != j)
//     (Sec. 2.3 items 3-5, Eq. 29; the mesh gates run i = 0..n-1 outer, j = 0..n-1 inner)
//     enc:    0 RX  1 RY;  scale: 0 none 1 pi 2 bias 3 asin 4 acos (Eq. 27a-e)
//     premap: 0 direct (theta_j = scale(v_j), j < n_direct; 0 otherwise)
//             1 RFF + tanh MLP (a = tanh(h_out), theta = scale(a))
//   pi[0..2]  = medium (0 vacuum, 1 dielectric), energy_slice_size, energy_nt
//   pi[3..7]  = sharding: whole-loss counts of the collocation, IC and BC sets (0 = this
//               call's), whole-set points inside the disk, global index of the first
//               collocation point (see Prob)
//   pi[8]     = physics loss of the dielectric case: 0 Eq. 13 (separate MSEs of res1 over the
//               vacuum and dielectric sets, 1/eps(x,y) pointwise), 1 Eqs. 34-35 (one MSE of
//               res1 over all collocation points, eps = 1 or eps_r by set)
//   pd[0..11] = eps_r, disk_r, disk_x0, disk_y0, sigmoid_w, ic_sigma, ic_x0, ic_y0,
//               w_ic, w_bc, w_energy, w_sym (weight of L_sym, Eq. 18; 0 = off)
// Parameter layout (flat):
//   premap RFF+MLP: Omega[F][3] (Omega[F][6] with the periodic map; fixed, zero gradient), the
//     learned period T (periodic map only), then per hidden layer W[H][in] (in = 2F first, H
//     after), b[H]; then W_out[n][H], b_out[n]
//   circuit: per layer [n][k] single-qubit angles, k = 2 (RY, RZ) for ansatz 0, 1 (RX) for
//     ansatz 4, 2 (RX, RZ) for ansatz 5, else 3 (Rot a,b,g); then, for ansatz 4 and 5, the
//     n (n-1) CRZ angles [i][j != i] (control i, targets j in increasing order)
//   head: W[3][m], b[3]
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

typedef std::complex<double> cd;

// ---------------------------------------------------------------- HD numbers
template <class T>
struct HD {
  T c[8];
  HD() { for (auto& x : c) x = T(0); }
  explicit HD(T v) { for (auto& x : c) x = T(0); c[0] = v; }
};
typedef HD<double> R;
typedef HD<cd> C;

template <class T>
HD<T> operator+(const HD<T>& a, const HD<T>& b) {
  HD<T> r;
  for (int i = 0; i < 8; ++i) r.c[i] = a.c[i] + b.c[i];
  return r;
}
template <class T>
HD<T> operator-(const HD<T>& a, const HD<T>& b) {
  HD<T> r;
  for (int i = 0; i < 8; ++i) r.c[i] = a.c[i] - b.c[i];
  return r;
}
template <class T, class S>
HD<T> scal(const HD<T>& a, S s) {
  HD<T> r;
  for (int i = 0; i < 8; ++i) r.c[i] = a.c[i] * s;
  return r;
}
// Product rule truncated at first order in each of {x,y,t} and in p, keeping
// the mixed (d, p) terms; products of two different input directions are dropped.
template <class T>
HD<T> operator*(const HD<T>& a, const HD<T>& b) {
  HD<T> r;
  r.c[0] = a.c[0] * b.c[0];
  for (int d = 1; d <= 3; ++d) r.c[d] = a.c[0] * b.c[d] + a.c[d] * b.c[0];
  r.c[4] = a.c[0] * b.c[4] + a.c[4] * b.c[0];
  for (int d = 1; d <= 3; ++d)
    r.c[4 + d] = a.c[0] * b.c[4 + d] + a.c[d] * b.c[4] + a.c[4] * b.c[d] + a.c[4 + d] * b.c[0];
  return r;
}
C to_c(const R& a) {
  C r;
  for (int i = 0; i < 8; ++i) r.c[i] = cd(a.c[i], 0.0);
  return r;
}
C conj(const C& a) {
  C r;
  for (int i = 0; i < 8; ++i) r.c[i] = std::conj(a.c[i]);
  return r;
}
R re(const C& a) {
  R r;
  for (int i = 0; i < 8; ++i) r.c[i] = a.c[i].real();
  return r;
}
C times_i(const C& a, double sgn) {  // a * (sgn i)
  C r;
  for (int i = 0; i < 8; ++i) r.c[i] = a.c[i] * cd(0.0, sgn);
  return r;
}
// Chain rule for a scalar function g with g(a0), g'(a0), g''(a0) given.
R fun(const R& a, double g0, double g1, double g2) {
  R r;
  r.c[0] = g0;
  for (int i = 1; i <= 4; ++i) r.c[i] = g1 * a.c[i];
  for (int d = 1; d <= 3; ++d) r.c[4 + d] = g1 * a.c[4 + d] + g2 * a.c[d] * a.c[4];
  return r;
}
R hcos(const R& a) { return fun(a, std::cos(a.c[0]), -std::sin(a.c[0]), -std::cos(a.c[0])); }
R hsin(const R& a) { return fun(a, std::sin(a.c[0]), std::cos(a.c[0]), -std::sin(a.c[0])); }
R htanh(const R& a) {
  double t = std::tanh(a.c[0]);
  double s2 = 1.0 - t * t;
  return fun(a, t, s2, -2.0 * t * s2);
}
R hexp(const R& a) { double e = std::exp(a.c[0]); return fun(a, e, e, e); }

// ---------------------------------------------------------------- configs
struct Circ {
  int n, L, m, ansatz, enc, scale, premap, n_direct, F, H, depth, periodic;
  int in_dim() const { return periodic ? 6 : 3; }   // RFF input width
  int k() const { return ansatz == 0 || ansatz == 5 ? 2 : (ansatz == 4 ? 1 : 3); }
  bool crz() const { return ansatz == 4 || ansatz == 5; }
  int64_t layer_count() const { return (int64_t)n * k() + (crz() ? (int64_t)n * (n - 1) : 0); }
  int64_t premap_count() const {
    if (premap == 0) return 0;
    int64_t c = (int64_t)in_dim() * F + (periodic ? 1 : 0);
    int in = 2 * F;
    for (int l = 0; l < depth; ++l) { c += (int64_t)H * in + H; in = H; }
    c += (int64_t)n * in + n;
    return c;
  }
  int64_t circuit_offset() const { return premap_count(); }
  int64_t circuit_count() const { return (int64_t)L * layer_count(); }
  int64_t head_offset() const { return circuit_offset() + circuit_count(); }
  int64_t total() const { return head_offset() + 3LL * m + 3; }
};
Circ read_circ(const int* ci) {
  Circ c;
  c.n = ci[0]; c.L = ci[1]; c.m = ci[2]; c.ansatz = ci[3]; c.enc = ci[4]; c.scale = ci[5];
  c.premap = ci[6]; c.n_direct = ci[7]; c.F = ci[8]; c.H = ci[9]; c.depth = ci[10];
  c.periodic = ci[11];
  return c;
}
bool circ_ok(const Circ& c) {
  if (c.n < 1 || c.n > 12 || c.L < 0 || c.m < 1 || c.m > c.n) return false;
  if (c.ansatz < 0 || c.ansatz > 6 || c.enc < 0 || c.enc > 1 || c.scale < 0 || c.scale > 4) return false;
  if (c.premap == 0) return c.n_direct >= 0 && c.n_direct <= 3 && c.n_direct <= c.n;
  if (c.premap == 1) return c.F >= 1 && c.H >= 1 && c.depth >= 0 && (c.periodic == 0 || c.periodic == 1);
  return false;
}

struct Prob {
  int medium, slice, nt;
  // Sharding of one loss over several calls: the means of Eqs. 11-17 and 23 run over the
  // whole point sets, so a call holding part of them divides its sums by the whole counts
  // (norm_*; 0 = this call's own sets), uses the whole set's number of points inside the
  // disk (norm_diel, read when norm_c > 0) and places its collocation points in the energy
  // slices of Eq. 31 from global index colloc_off on.
  int64_t norm_c, norm_i, norm_b, norm_diel, colloc_off;
  int phys_loss;
  double eps_r, disk_r, x0, y0, sw, ic_sigma, ic_x0, ic_y0, w_ic, w_bc, w_energy, w_sym;
};
Prob read_prob(const int* pi, const double* pd) {
  Prob p;
  p.medium = pi[0]; p.slice = pi[1]; p.nt = pi[2];
  p.norm_c = pi[3]; p.norm_i = pi[4]; p.norm_b = pi[5]; p.norm_diel = pi[6]; p.colloc_off = pi[7];
  p.phys_loss = pi[8];
  p.eps_r = pd[0]; p.disk_r = pd[1]; p.x0 = pd[2]; p.y0 = pd[3]; p.sw = pd[4];
  p.ic_sigma = pd[5]; p.ic_x0 = pd[6]; p.ic_y0 = pd[7];
  p.w_ic = pd[8]; p.w_bc = pd[9]; p.w_energy = pd[10]; p.w_sym = pd[11];
  return p;
}

// ---------------------------------------------------------------- scalings, Eq. 27
// Angle as a function of the raw input a (direct premap).
R scale_direct(int s, const R& a) {
  switch (s) {
    case 0: return a;
    case 1: return scal(a, M_PI);
    case 2: { R r = scal(a, M_PI / 2); r.c[0] += M_PI / 2; return r; }
    case 3: { double x = a.c[0], q = 1.0 / std::sqrt(1 - x * x);
              return fun(a, std::asin(x) + M_PI / 2, q, x * q * q * q); }
    default: { double x = a.c[0], q = 1.0 / std::sqrt(1 - x * x);
               return fun(a, std::acos(x), -q, -x * q * q * q); }
  }
}
// Angle as a function of the pre-activation h, a = tanh(h) (MLP premap). The
// composite derivatives avoid the 1/sqrt(1-a^2) factor of asin/acos at |a| -> 1:
// d acos(tanh h)/dh = -sech h, d asin(tanh h)/dh = sech h.
R scale_tanh(int s, const R& h) {
  double t = std::tanh(h.c[0]);
  double s2 = 1.0 - t * t;          // sech^2
  double sh = 1.0 / std::cosh(h.c[0]);  // sech
  switch (s) {
    case 0: return fun(h, t, s2, -2 * t * s2);
    case 1: return fun(h, M_PI * t, M_PI * s2, -2 * M_PI * t * s2);
    case 2: return fun(h, (t + 1) * M_PI / 2, M_PI / 2 * s2, -M_PI * t * s2);
    case 3: return fun(h, std::asin(t) + M_PI / 2, sh, -sh * t);
    default: return fun(h, std::acos(t), -sh, sh * t);
  }
}

// ---------------------------------------------------------------- gates
struct G2 { C a, b, c, d; };  // [[a, b], [c, d]]
G2 mul(const G2& x, const G2& y) {
  return {x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c, x.c * y.b + x.d * y.d};
}
G2 g_rx(const R& t) {
  R h = scal(t, 0.5);
  C c = to_c(hcos(h)), s = to_c(hsin(h));
  return {c, times_i(s, -1), times_i(s, -1), c};
}
G2 g_ry(const R& t) {
  R h = scal(t, 0.5);
  C c = to_c(hcos(h)), s = to_c(hsin(h));
  return {c, scal(s, -1.0), s, c};
}
G2 g_rz(const R& t) {
  R h = scal(t, 0.5);
  C c = to_c(hcos(h)), s = to_c(hsin(h));
  return {c - times_i(s, 1), C(), C(), c + times_i(s, 1)};
}
G2 g_rot(const R& al, const R& be, const R& ga) { return mul(g_rz(ga), mul(g_ry(be), g_rz(al))); }

int bitpos(int n, int q) { return n - 1 - q; }

// Textbook pair loop: amplitude pairs differing only in qubit q.
void apply1(std::vector<C>& s, int n, int q, const G2& g) {
  const int64_t bit = 1LL << bitpos(n, q);
  const int64_t dim = 1LL << n;
  for (int64_t k0 = 0; k0 < dim; ++k0) {
    if (k0 & bit) continue;
    const int64_t k1 = k0 | bit;
    C x = s[k0], y = s[k1];
    s[k0] = g.a * x + g.b * y;
    s[k1] = g.c * x + g.d * y;
  }
}
void apply_cnot(std::vector<C>& s, int n, int ctl, int tgt) {
  const int64_t bc = 1LL << bitpos(n, ctl), bt = 1LL << bitpos(n, tgt);
  const int64_t dim = 1LL << n;
  for (int64_t k = 0; k < dim; ++k)
    if ((k & bc) && !(k & bt)) std::swap(s[k], s[k | bt]);
}
int ring_stride(const Circ& c, int l) {
  if (c.ansatz == 2) return c.n > 1 ? 1 + (l % (c.n - 1)) : 1;
  return 1;
}
// Controlled RZ (Sec. 2.3 item 3): RZ(t) on the target where the control qubit is 1.
void apply_crz(std::vector<C>& s, int n, int ctl, int tgt, const R& t) {
  const int64_t bc = 1LL << bitpos(n, ctl), bt = 1LL << bitpos(n, tgt);
  const G2 g = g_rz(t);
  const int64_t dim = 1LL << n;
  for (int64_t k = 0; k < dim; ++k)
    if (k & bc) s[k] = ((k & bt) ? g.d : g.a) * s[k];
}
// One ansatz layer l: single-qubit rotations on every qubit, then the entangling part (CNOT
// ring, CRZ mesh or CNOT mesh).
void apply_layer(std::vector<C>& s, const Circ& c, const R* cp, int l) {
  const int k = c.k();
  const R* lp = cp + (int64_t)l * c.layer_count();
  for (int q = 0; q < c.n; ++q) {
    const R* p = lp + (int64_t)q * k;
    G2 g;
    switch (c.ansatz) {
      case 0: g = mul(g_rz(p[1]), g_ry(p[0])); break;   // RY(a) then RZ(b)
      case 4: g = g_rx(p[0]); break;                     // RX(a)
      case 5: g = mul(g_rz(p[1]), g_rx(p[0])); break;   // RX(a) then RZ(b)
      default: g = g_rot(p[0], p[1], p[2]); break;
    }
    apply1(s, c.n, q, g);
  }
  if (c.ansatz == 3 || c.n < 2) return;
  if (c.crz()) {
    const R* t = lp + (int64_t)c.n * k;
    for (int i = 0; i < c.n; ++i)
      for (int j = 0; j < c.n; ++j)
        if (j != i) apply_crz(s, c.n, i, j, t[i * (c.n - 1) + (j < i ? j : j - 1)]);
    return;
  }
  if (c.ansatz == 6) {
    for (int i = 0; i < c.n; ++i)
      for (int j = 0; j < c.n; ++j)
        if (j != i) apply_cnot(s, c.n, i, j);
    return;
  }
  const int r = ring_stride(c, l);
  for (int i = 0; i < c.n; ++i) apply_cnot(s, c.n, i, (i + r) % c.n);
}

// ---------------------------------------------------------------- premap
void premap(const Circ& c, const R* P, const R v[3], std::vector<R>& theta) {
  theta.assign(c.n, R());
  if (c.premap == 0) {
    for (int j = 0; j < c.n_direct; ++j) theta[j] = scale_direct(c.scale, v[j]);
    return;
  }
  const R* om = P;  // Omega[F][in_dim]
  const int di = c.in_dim();
  // periodic map (Eqs. 25-26): space over the domain lengths 2, time over the learned period
  std::vector<R> u(di);
  if (c.periodic) {
    const R T = P[(int64_t)di * c.F];
    const R ax = scal(v[0], M_PI), ay = scal(v[1], M_PI);
    const R invT = fun(T, 1.0 / T.c[0], -1.0 / (T.c[0] * T.c[0]), 2.0 / (T.c[0] * T.c[0] * T.c[0]));
    const R at = scal(v[2] * invT, 2.0 * M_PI);
    u[0] = hsin(ax); u[1] = hcos(ax); u[2] = hsin(ay); u[3] = hcos(ay); u[4] = hsin(at); u[5] = hcos(at);
  } else {
    u[0] = v[0]; u[1] = v[1]; u[2] = v[2];
  }
  std::vector<R> x(2 * c.F);
  for (int f = 0; f < c.F; ++f) {
    R arg = om[(int64_t)di * f] * u[0];
    for (int j = 1; j < di; ++j) arg = arg + om[(int64_t)di * f + j] * u[j];
    x[f] = hcos(arg);
    x[c.F + f] = hsin(arg);
  }
  const R* w = P + (int64_t)di * c.F + (c.periodic ? 1 : 0);
  int in = 2 * c.F;
  for (int l = 0; l < c.depth; ++l) {
    std::vector<R> y(c.H);
    const R* b = w + (int64_t)c.H * in;
    for (int o = 0; o < c.H; ++o) {
      R acc = b[o];
      for (int i = 0; i < in; ++i) acc = acc + w[(int64_t)o * in + i] * x[i];
      y[o] = htanh(acc);
    }
    w = b + c.H;
    x.swap(y);
    in = c.H;
  }
  const R* b = w + (int64_t)c.n * in;
  for (int o = 0; o < c.n; ++o) {
    R acc = b[o];
    for (int i = 0; i < in; ++i) acc = acc + w[(int64_t)o * in + i] * x[i];
    theta[o] = scale_tanh(c.scale, acc);
  }
}

// ---------------------------------------------------------------- circuit
// Embedding G(theta_j)|0> per qubit, product state, layers. Returns final state.
void run_circuit(const Circ& c, const R* cp, const std::vector<R>& theta, std::vector<C>& s) {
  const int64_t dim = 1LL << c.n;
  std::vector<C> g0(c.n), g1(c.n);
  for (int j = 0; j < c.n; ++j) {
    G2 g = c.enc == 0 ? g_rx(theta[j]) : g_ry(theta[j]);
    g0[j] = g.a;  // first column = G|0>
    g1[j] = g.c;
  }
  s.assign(dim, C());
  for (int64_t k = 0; k < dim; ++k) {
    C a(cd(1.0, 0.0));
    for (int j = 0; j < c.n; ++j) a = a * (((k >> bitpos(c.n, j)) & 1) ? g1[j] : g0[j]);
    s[k] = a;
  }
  for (int l = 0; l < c.L; ++l) apply_layer(s, c, cp, l);
}
void readout(const Circ& c, const std::vector<C>& s, std::vector<R>& z) {
  z.assign(c.m, R());
  const int64_t dim = 1LL << c.n;
  for (int64_t k = 0; k < dim; ++k) {
    R pr = re(conj(s[k]) * s[k]);
    for (int i = 0; i < c.m; ++i) {
      if ((k >> bitpos(c.n, i)) & 1) z[i] = z[i] - pr;
      else z[i] = z[i] + pr;
    }
  }
}
// Full point evaluation: v (x,y,t) -> fields f[3] as HD numbers.
void eval_point(const Circ& c, const R* P, const double* pt, R f[3]) {
  R v[3];
  for (int d = 0; d < 3; ++d) { v[d] = R(pt[d]); v[d].c[1 + d] = 1.0; }
  std::vector<R> theta;
  premap(c, P, v, theta);
  std::vector<C> s;
  run_circuit(c, P + c.circuit_offset(), theta, s);
  std::vector<R> z;
  readout(c, s, z);
  const R* W = P + c.head_offset();
  const R* b = W + 3 * c.m;
  for (int o = 0; o < 3; ++o) {
    R acc = b[o];
    for (int i = 0; i < c.m; ++i) acc = acc + W[o * c.m + i] * z[i];
    f[o] = acc;
  }
}

// ---------------------------------------------------------------- losses
// Dual number in the selected parameter p only (value, d/dp).
struct D {
  double v, p;
};
D operator+(D a, D b) { return {a.v + b.v, a.p + b.p}; }
D operator-(D a, D b) { return {a.v - b.v, a.p - b.p}; }
D operator*(D a, D b) { return {a.v * b.v, a.v * b.p + a.p * b.v}; }
D operator*(double s, D a) { return {s * a.v, s * a.p}; }

// eps(x, y) of the dielectric case: 1 + (eps_r - 1) sigmoid((R - r)/w) around the
// disk centre; 1 in vacuum.
double eps_at(const Prob& pb, double x, double y) {
  if (pb.medium == 0) return 1.0;
  double dx = x - pb.x0, dy = y - pb.y0, r = std::sqrt(dx * dx + dy * dy);
  return 1.0 + (pb.eps_r - 1.0) / (1.0 + std::exp(-(pb.disk_r - r) / pb.sw));
}
// Dielectric-set membership, decided in float32 arithmetic exactly like the kernel.
bool in_diel(const Prob& pb, double x, double y) {
  if (pb.medium == 0) return false;
  float dx = (float)x - (float)pb.x0, dy = (float)y - (float)pb.y0;
  float r2 = __builtin_fmaf(dx, dx, dy * dy);
  float R2 = (float)pb.disk_r * (float)pb.disk_r;
  return r2 < R2;
}

// Loss terms from fields. Fc: per collocation point [3] values (Ez,Hx,Hy) and
// DFc [3][3] (c, d) input derivatives, as duals in p. Layout of out (values) and
// outp (d/dp): see header comment of qpo_loss.
// Symmetry penalty of Eq. 18 summed over the collocation points (before the 1/N of the mean):
// Fmx = f(-x, y, t), Fmy = f(x, -y, t) per point; in the dielectric case the terms mirrored
// along x are left out (the disk breaks that symmetry).
D sym_sum(const Prob& pb, int64_t Bc, const std::vector<D>& Fc, const std::vector<D>& Fmx,
          const std::vector<D>& Fmy) {
  D s{0, 0};
  for (int64_t b = 0; b < Bc; ++b) {
    const D* f = &Fc[3 * b];
    if (pb.medium == 0) {
      const D* m = &Fmx[3 * b];   // (i) Ez even, (ii) Hx even, (iii) Hy odd in x
      const D a = f[0] - m[0], c = f[1] - m[1], e = f[2] + m[2];
      s = s + a * a + c * c + e * e;
    }
    const D* m = &Fmy[3 * b];     // (i) Ez even, (ii) Hx odd, (iii) Hy even in y
    const D a = f[0] - m[0], c = f[1] + m[1], e = f[2] - m[2];
    s = s + a * a + c * c + e * e;
  }
  return s;
}

void loss_terms(const Prob& pb, const double* pc, int64_t Bc, const std::vector<D>& Fc,
                const std::vector<D>& DFc, const double* pi_, int64_t Bi, const std::vector<D>& Fi,
                const double* pbnd, int64_t Bb, const std::vector<D>& Fb, double* out, double* outp,
                const std::vector<D>& Fmx, const std::vector<D>& Fmy) {
  D s1v{0, 0}, s1d{0, 0}, s2{0, 0}, s3{0, 0}, se{0, 0};
  int64_t nd = 0;
  for (int64_t b = 0; b < Bc; ++b) nd += in_diel(pb, pc[3 * b], pc[3 * b + 1]) ? 1 : 0;
  const int64_t Nc = pb.norm_c > 0 ? pb.norm_c : Bc;   // collocation mean denominator
  if (pb.norm_c > 0) nd = pb.norm_diel;
  const int64_t nv = Nc - nd;
  const int64_t Ni = pb.norm_i > 0 ? pb.norm_i : Bi, Nb = pb.norm_b > 0 ? pb.norm_b : Bb;
  std::vector<double> U(pb.nt > 0 ? pb.nt : 0, 0.0);
  for (int64_t b = 0; b < Bc; ++b) {
    const double x = pc[3 * b], y = pc[3 * b + 1];
    const double eps = eps_at(pb, x, y);
    const D* f = &Fc[3 * b];
    const D* Df = &DFc[9 * b];  // Df[c*3+d]
    auto dd = [&](int cc, int d) { return Df[cc * 3 + d]; };
    // Eq. 8 / 9 (1/eps pointwise in the dielectric case), Eq. 10a-b; the intuitive form
    // (Eq. 34) takes eps = eps_r on the dielectric set and 1 elsewhere, in one MSE
    D curl = dd(2, 0) - dd(1, 1);
    const bool intuitive = pb.medium == 1 && pb.phys_loss == 1;
    const double e1 = intuitive ? (in_diel(pb, x, y) ? pb.eps_r : 1.0) : eps;
    D r1 = dd(0, 2) - (1.0 / e1) * curl;
    D r2 = dd(1, 2) + dd(0, 1);
    D r3 = dd(2, 2) - dd(0, 0);
    if (pb.medium == 1 && !intuitive && in_diel(pb, x, y)) s1d = s1d + r1 * r1;
    else s1v = s1v + r1 * r1;
    s2 = s2 + r2 * r2;
    s3 = s3 + r3 * r3;
    // Eq. 23 Poynting residual, squared (global energy term read as a mean square).
    D e = eps * (f[0] * dd(0, 2)) + f[1] * dd(1, 2) + f[2] * dd(2, 2) -
          (dd(0, 0) * f[2] + f[0] * dd(2, 0)) + (dd(0, 1) * f[1] + f[0] * dd(1, 1));
    se = se + e * e;
    if (pb.nt > 0 && pb.slice > 0) {
      int64_t k = (pb.colloc_off + b) / pb.slice;
      if (k < pb.nt) U[k] += 0.5 * (eps * f[0].v * f[0].v + f[1].v * f[1].v + f[2].v * f[2].v);
    }
  }
  D mse1v{0, 0}, mse1d{0, 0};
  if (pb.medium == 1 && pb.phys_loss == 1) {
    if (Nc > 0) mse1v = (1.0 / Nc) * s1v;   // Eq. 35: all collocation points weigh the same
  } else if (pb.medium == 1) {
    if (nv > 0) mse1v = (1.0 / nv) * s1v;
    if (nd > 0) mse1d = (1.0 / nd) * s1d;
  } else if (Nc > 0) {
    mse1v = (1.0 / Nc) * s1v;
  }
  D mse2 = Nc > 0 ? (1.0 / Nc) * s2 : D{0, 0};
  D mse3 = Nc > 0 ? (1.0 / Nc) * s3 : D{0, 0};
  D phys = mse1v + mse1d + mse2 + mse3;
  D energy = Nc > 0 ? (pb.w_energy / Nc) * se : D{0, 0};
  // Eq. 17 with a Gaussian pulse centred at (ic_x0, ic_y0): exp(-r^2 / (2 sigma^2)).
  D sic{0, 0};
  for (int64_t b = 0; b < Bi; ++b) {
    double dx = pi_[3 * b] - pb.ic_x0, dy = pi_[3 * b + 1] - pb.ic_y0;
    double e0 = std::exp(-(dx * dx + dy * dy) / (2 * pb.ic_sigma * pb.ic_sigma));
    D m0 = Fi[3 * b] - D{e0, 0};
    sic = sic + m0 * m0 + Fi[3 * b + 1] * Fi[3 * b + 1] + Fi[3 * b + 2] * Fi[3 * b + 2];
  }
  D ic = Ni > 0 ? (pb.w_ic / Ni) * sic : D{0, 0};
  // PEC boundary: tangential E vanishes, Ez = 0 on the edges.
  D sbc{0, 0};
  for (int64_t b = 0; b < Bb; ++b) sbc = sbc + Fb[3 * b] * Fb[3 * b];
  D bc = Nb > 0 ? (pb.w_bc / Nb) * sbc : D{0, 0};
  // Eq. 18 weighted as in Eq. 24, a mean over the collocation points
  D sym{0, 0};
  if (pb.w_sym > 0 && Nc > 0 && (int64_t)Fmy.size() == 3 * Bc) sym = (pb.w_sym / Nc) * sym_sum(pb, Bc, Fc, Fmx, Fmy);
  D tot = phys + ic + bc + energy + sym;
  D terms[9] = {tot, phys, ic, bc, energy, mse1v, mse1d, mse2, mse3};
  for (int i = 0; i < 9; ++i) {
    out[i] = terms[i].v;
    if (outp) outp[i] = terms[i].p;
  }
  for (int k = 0; k < pb.nt; ++k) out[9 + k] = U[k];
  if (pb.w_sym > 0) out[9 + (pb.nt > 0 ? pb.nt : 0)] = sym.v;
}

template <class F>
void parallel_for(int64_t n, int nthreads, F fn) {
  if (nthreads <= 1 || n <= 1) { for (int64_t i = 0; i < n; ++i) fn(i); return; }
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&, t] { for (int64_t i = t; i < n; i += nthreads) fn(i); });
  for (auto& x : th) x.join();
}

void to_duals(const R f[3], D* F, D* DF) {
  for (int c = 0; c < 3; ++c) {
    F[c] = {f[c].c[0], f[c].c[4]};
    if (DF)
      for (int d = 0; d < 3; ++d) DF[c * 3 + d] = {f[c].c[1 + d], f[c].c[5 + d]};
  }
}

std::vector<R> make_params(const Circ& c, const double* params, int64_t sel) {
  std::vector<R> P(c.total());
  for (int64_t i = 0; i < c.total(); ++i) P[i] = R(params[i]);
  if (sel >= 0) P[sel].c[4] = 1.0;
  return P;
}

// The point evaluations are independent, so they may run on several threads (each writes
// only its own point's entries); the loss sums of loss_terms then run in point order on one
// thread, so the result does not depend on the thread count.
void eval_loss(const Circ& c, const Prob& pb, const double* params, int64_t sel, const double* pc,
               int64_t Bc, const double* pi_, int64_t Bi, const double* pbnd, int64_t Bb, double* out,
               double* outp, int nthreads) {
  std::vector<R> P = make_params(c, params, sel);
  std::vector<D> Fc(3 * Bc), DFc(9 * Bc), Fi(3 * Bi), Fb(3 * Bb);
  // L_sym (Eq. 18): the fields at the mirrored points (-x, y, t) and (x, -y, t)
  const bool sym = pb.w_sym > 0;
  std::vector<D> Fmx(sym ? 3 * Bc : 0), Fmy(sym ? 3 * Bc : 0);
  if (sym) {
    parallel_for(2 * Bc, nthreads, [&](int64_t q) {
      const int64_t b = q % Bc;
      const bool mx = q < Bc;
      const double pt[3] = {mx ? -pc[3 * b] : pc[3 * b], mx ? pc[3 * b + 1] : -pc[3 * b + 1], pc[3 * b + 2]};
      R f[3];
      eval_point(c, P.data(), pt, f);
      to_duals(f, mx ? &Fmx[3 * b] : &Fmy[3 * b], nullptr);
    });
  }
  parallel_for(Bc + Bi + Bb, nthreads, [&](int64_t q) {
    R f[3];
    if (q < Bc) {
      eval_point(c, P.data(), pc + 3 * q, f);
      to_duals(f, &Fc[3 * q], &DFc[9 * q]);
    } else if (q < Bc + Bi) {
      const int64_t b = q - Bc;
      eval_point(c, P.data(), pi_ + 3 * b, f);
      to_duals(f, &Fi[3 * b], nullptr);
    } else {
      const int64_t b = q - Bc - Bi;
      eval_point(c, P.data(), pbnd + 3 * b, f);
      to_duals(f, &Fb[3 * b], nullptr);
    }
  });
  loss_terms(pb, pc, Bc, Fc, DFc, pi_, Bi, Fi, pbnd, Bb, Fb, out, outp, Fmx, Fmy);
}

}  // namespace

extern "C" {

int qpo_version() { return 1; }

int64_t qpo_param_count(const int* ci) {
  Circ c = read_circ(ci);
  if (!circ_ok(c)) return -1;
  return c.total();
}

// Offsets of the parameter blocks: out[0] circuit offset, out[1] head offset,
// out[2] total, out[3] number of fixed (Omega) entries at the front.
int qpo_param_layout(const int* ci, int64_t* out) {
  Circ c = read_circ(ci);
  if (!circ_ok(c)) return 1;
  out[0] = c.circuit_offset(); out[1] = c.head_offset(); out[2] = c.total();
  out[3] = c.premap == 1 ? (int64_t)c.in_dim() * c.F : 0;
  return 0;
}

// Encoding angles and their input Jacobian: theta[B][n], J[B][n][3].
int qpo_premap(const int* ci, const double* params, const double* pts, int64_t B, double* theta,
               double* J) {
  Circ c = read_circ(ci);
  if (!circ_ok(c)) return 1;
  std::vector<R> P = make_params(c, params, -1);
  for (int64_t b = 0; b < B; ++b) {
    R v[3];
    for (int d = 0; d < 3; ++d) { v[d] = R(pts[3 * b + d]); v[d].c[1 + d] = 1.0; }
    std::vector<R> th;
    premap(c, P.data(), v, th);
    for (int j = 0; j < c.n; ++j) {
      theta[b * c.n + j] = th[j].c[0];
      for (int d = 0; d < 3; ++d) J[(b * c.n + j) * 3 + d] = th[j].c[1 + d];
    }
  }
  return 0;
}

// Fields f[B][3] = (Ez, Hx, Hy) and input derivatives df[B][3][3] (c, d).
int qpo_forward(const int* ci, const double* params, const double* pts, int64_t B, double* f,
                double* df, int nthreads) {
  Circ c = read_circ(ci);
  if (!circ_ok(c)) return 1;
  std::vector<R> P = make_params(c, params, -1);
  parallel_for(B, nthreads, [&](int64_t b) {
    R o[3];
    eval_point(c, P.data(), pts + 3 * b, o);
    for (int cc = 0; cc < 3; ++cc) {
      f[3 * b + cc] = o[cc].c[0];
      if (df)
        for (int d = 0; d < 3; ++d) df[9 * b + 3 * cc + d] = o[cc].c[1 + d];
    }
  });
  return 0;
}

// Final state after embedding + layers for given embedding angles theta[n].
int qpo_state(const int* ci, const double* params, const double* theta, double* re_out,
              double* im_out) {
  Circ c = read_circ(ci);
  if (!circ_ok(c)) return 1;
  std::vector<R> P = make_params(c, params, -1);
  std::vector<R> th(c.n);
  for (int j = 0; j < c.n; ++j) th[j] = R(theta[j]);
  std::vector<C> s;
  run_circuit(c, P.data() + c.circuit_offset(), th, s);
  for (size_t k = 0; k < s.size(); ++k) { re_out[k] = s[k].c[0].real(); im_out[k] = s[k].c[0].imag(); }
  return 0;
}

// Matrix of ansatz layer l (rotations + CNOT ring), column k = layer |k>.
int qpo_layer_unitary(const int* ci, const double* params, int layer, double* re_out,
                      double* im_out) {
  Circ c = read_circ(ci);
  if (!circ_ok(c) || layer < 0 || layer >= c.L) return 1;
  std::vector<R> P = make_params(c, params, -1);
  const int64_t dim = 1LL << c.n;
  for (int64_t col = 0; col < dim; ++col) {
    std::vector<C> s(dim, C());
    s[col] = C(cd(1.0, 0.0));
    apply_layer(s, c, P.data() + c.circuit_offset(), layer);
    for (int64_t r = 0; r < dim; ++r) {
      re_out[r * dim + col] = s[r].c[0].real();
      im_out[r * dim + col] = s[r].c[0].imag();
    }
  }
  return 0;
}

// Loss terms. out layout: [0] total, [1] L_phys, [2] weighted L_IC, [3] weighted
// L_BC, [4] weighted L_energy, [5] MSE res1 (vacuum set), [6] MSE res1 (dielectric
// set), [7] MSE res2, [8] MSE res3, [9 .. 9+nt) energy slice sums U(t_k).
int qpo_loss(const int* ci, const int* pi, const double* pd, const double* params, const double* pc,
             int64_t Bc, const double* pi_, int64_t Bi, const double* pbnd, int64_t Bb, double* out,
             int nthreads) {
  Circ c = read_circ(ci);
  if (!circ_ok(c)) return 1;
  Prob pb = read_prob(pi, pd);
  eval_loss(c, pb, params, -1, pc, Bc, pi_, Bi, pbnd, Bb, out, nullptr, nthreads);
  return 0;
}

// d(total loss)/d(param) for the listed parameter indices; fixed Omega entries get 0.
int qpo_grad(const int* ci, const int* pi, const double* pd, const double* params, const double* pc,
             int64_t Bc, const double* pi_, int64_t Bi, const double* pbnd, int64_t Bb,
             const int64_t* idx, int64_t nidx, double* grad, int nthreads) {
  Circ c = read_circ(ci);
  if (!circ_ok(c)) return 1;
  Prob pb = read_prob(pi, pd);
  const int64_t nfixed = c.premap == 1 ? (int64_t)c.in_dim() * c.F : 0;
  for (int64_t i = 0; i < nidx; ++i)
    if (idx[i] < 0 || idx[i] >= c.total()) return 2;
  // threads over the listed parameters, or over the points of each evaluation when there are
  // fewer parameters than threads (same arithmetic either way)
  const bool outer = nidx >= nthreads;
  parallel_for(nidx, outer ? nthreads : 1, [&](int64_t i) {
    if (idx[i] < nfixed) { grad[i] = 0.0; return; }
    std::vector<double> out(10 + (pb.nt > 0 ? pb.nt : 0)), outp(9);
    eval_loss(c, pb, params, idx[i], pc, Bc, pi_, Bi, pbnd, Bb, out.data(), outp.data(),
              outer ? 1 : nthreads);
    grad[i] = outp[0];
  });
  return 0;
}

// Loss terms from externally given fields (no circuit): f_c[Bc][3], df_c[Bc][3][3],
// f_i[Bi][3], f_b[Bb][3]. Used to pin the residual and energy formulas.
// Number of points of pts[n][3] inside the dielectric disk (the in_diel test of the loss).
int64_t qpo_count_diel(const int* pi, const double* pd, const double* pts, int64_t n) {
  Prob pb = read_prob(pi, pd);
  int64_t c = 0;
  if (pb.medium != 1) return 0;
  for (int64_t b = 0; b < n; ++b) c += in_diel(pb, pts[3 * b], pts[3 * b + 1]) ? 1 : 0;
  return c;
}

int qpo_loss_from_fields(const int* pi, const double* pd, const double* pc, int64_t Bc,
                         const double* fc, const double* dfc, const double* pi_, int64_t Bi,
                         const double* fi, const double* pbnd, int64_t Bb, const double* fb,
                         double* out) {
  Prob pb = read_prob(pi, pd);
  std::vector<D> Fc(3 * Bc), DFc(9 * Bc), Fi(3 * Bi), Fb(3 * Bb);
  for (int64_t i = 0; i < 3 * Bc; ++i) Fc[i] = {fc[i], 0};
  for (int64_t i = 0; i < 9 * Bc; ++i) DFc[i] = {dfc[i], 0};
  for (int64_t i = 0; i < 3 * Bi; ++i) Fi[i] = {fi[i], 0};
  for (int64_t i = 0; i < 3 * Bb; ++i) Fb[i] = {fb[i], 0};
  loss_terms(pb, pc, Bc, Fc, DFc, pi_, Bi, Fi, pbnd, Bb, Fb, out, nullptr, {}, {});
  return 0;
}

// w_sym L_sym (Eq. 18 as weighted in Eq. 24) from given fields: f_c, f(-x,y,t), f(x,-y,t), each
// [Bc][3]; the mean runs over Bc points (or the sharding count).
double qpo_sym_from_fields(const int* pi, const double* pd, int64_t Bc, const double* fc, const double* fmx,
                           const double* fmy) {
  Prob pb = read_prob(pi, pd);
  std::vector<D> Fc(3 * Bc), Fmx(3 * Bc), Fmy(3 * Bc);
  for (int64_t i = 0; i < 3 * Bc; ++i) { Fc[i] = {fc[i], 0}; Fmx[i] = {fmx[i], 0}; Fmy[i] = {fmy[i], 0}; }
  const int64_t Nc = pb.norm_c > 0 ? pb.norm_c : Bc;
  return Nc > 0 ? pb.w_sym / Nc * sym_sum(pb, Bc, Fc, Fmx, Fmy).v : 0.0;
}

}  // extern "C"
